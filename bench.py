"""Benchmark: GPU solves of the locally compressed MFS on one GB300.

Default workload: P = 10^4 unit disks in a random close packing at area
fraction 0.65 (square lattice, Metropolis sweeps at minimum gap 1e-3, the
closest pair snapped to 1e-3; ~10^4 close pairs), mobility problem with
seeded N(0,1) forces (net force shifted to zero) and torques, 72 vector
unknowns per body (N_c = 60, M_c = 72, about 1.44M scalar unknowns), fine
pair parameters N_fp = 150, N_ell = 80, M_p = 200, tolerance 1e-6 on the FP64
residual.  One step = one complete solve of that batch on the device: contact
detection, one-body factors and every pair block (batched FP64 QR), the FP64
completion-flow right-hand side, mixed-precision GMRES (FP32 far field,
graph-captured iterations) refined against the FP64 operator, and the
velocity post-processing.  Inputs are resident in device memory before the
timed region; `e2e` repeats the measurement through the host API (geometry
and forces copied in from pinned host memory, velocities copied out).

Also reported: the dominant kernel's roofline (the batched FP64 QR, from CUDA
events on the handle's stream inside the library), the oracle's checks of
the timed solution on sampled rows (its residual and the matvec), the
P = 100 packing's solves (with the oracle's solve), both Stokeslet tile
kernels at the P = 10^4 size (Gpair/s against the FP32 peak), a bounded
serving stream (served mixed precision against one-at-a-time FP64 on the same
requests, p50/p99 request latency), SM clocks sampled during the timed region,
and the CPU oracle's time for this workload, extrapolated from timed samples.

--impl reference times the CPU oracle itself (plain FP64 numpy) on bounded
samples of the same workload (pair precomputes and matvec rows), extrapolated
to one solve.  Multi-GPU: the solve does not shard, so N ranks run
independent replicas (weak scaling; value = all ranks' solves / max-over-ranks
time).
"""
import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "Stokeslet Gpair-evals/s vs FP32 peak; batched solves/s & p99 latency at 1e-5 err"
WORKLOAD = "p10000_phi065_mobility"


def peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return {}


class Clocks:
    """Sample nvidia-smi SM clocks and throttle reasons in the background."""
    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index=0):
        self.index = index
        self.rows = []
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.Q,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append([x.strip() for x in line.split(",")])

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        sm = [float(r[0]) for r in self.rows if len(r) >= 8 and r[0].replace(".", "").isdigit()]
        mx = [float(r[1]) for r in self.rows if len(r) >= 8 and r[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[j] for r in self.rows if len(r) >= 8 for j in range(4) if r[4 + j] == "Active"})
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(sm)}


# Counters of the blocked QR kernel (rqr_kernel, trailing updates on the
# tensor cores) from one ncu capture of its launch on the 398 fine half
# systems of `bench.py --profile-case qr_mid` (P = 160, area fraction 0.65,
# one CTA per system as in the P = 10^4 launches): DRAM bytes
# (dram__bytes_read.sum + dram__bytes_write.sum) per system, and the launch's
# algorithmic FP64 flops per ALU-pipe warp instruction
# (sm__inst_executed_pipe_alu.sum), the pipe that carries the digit work.
# Valid only for the kernel source they were taken on (lmfs_rqr.cu and
# lmfs_emu64.cuh): reported as null once either changes.
RQR_TRAFFIC_PER_MATRIX = (80.89e9 + 40.48e9) / 398.0
RQR_FLOPS_PER_ALU_INST = 1.481730e11 / 1.2765068e10
RQR_SRC_SHA256 = "a2a29986564be4e7d583bf76d76ce2cae6d9c529f2da6d5be8c65efb76e31f1b"
ALU_WARP_INST_PER_CLK = 2          # 64 results per clock per SM for 32-bit integer add, logic and shift


def rqr_counters_valid():
    import hashlib
    h = hashlib.sha256()
    try:
        for f in ("lmfs_rqr.cu", "lmfs_emu64.cuh"):
            h.update(open(os.path.join(ROOT, "paper_2606_11273_gb300", "csrc", f), "rb").read())
    except OSError:
        return False
    return h.hexdigest() == RQR_SRC_SHA256


def rqr_traffic_per_matrix():
    return RQR_TRAFFIC_PER_MATRIX if rqr_counters_valid() else None


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def job_time_ms(t_ms, ws, device="cpu"):
    """Duration of the whole job's timed region: the maximum over ranks (the
    replicas start together after a barrier; the job ends with the slowest)."""
    if ws == 1:
        return float(t_ms)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(t_ms)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_value(steps, ws, t_ms):
    """Whole-job throughput: every rank's solves over the max-over-ranks time."""
    return ws * steps / (t_ms * 1e-3)


WORKLOADS = {
    # name: (problem, extra Params, tol)
    "p100_phi040_mobility": ("mobility", {}, 1e-7),
    "pair_gap1e-3_resistance": ("resistance", {"Nc": 36, "Mc": 72, "Rc": 0.7, "Nfp": 400}, 1e-10),
    "p1000_poly_phi060_mobility": ("mobility", {"delta_c": 0.1}, 1e-7),
    "p10000_phi065_mobility": ("mobility", {}, 1e-6),
}


def workload(name=WORKLOAD):
    import workloads as w
    if name == "p100_phi040_mobility":
        pk = w.packing_p100()
        data = w.forces_torques(pk.P, 5)
    elif name == "pair_gap1e-3_resistance":
        pk = w.two_disks(1e-3)
        data = w.rigid_velocities(2, 11)
    elif name == "p1000_poly_phi060_mobility":
        pk = w.packing_p1000_poly()
        data = w.forces_torques(pk.P, 6)
    elif name == "p10000_phi065_mobility":
        pk = w.packing_p10000()
        data = w.forces_torques(pk.P, 7)
    else:
        raise ValueError(name)
    return pk, data


def oracle_solve(pk, ft):
    from oracle.params import PACKING
    from oracle.system import System
    s = System(pk.centres, pk.radii, PACKING, "mobility")
    return s.solve(ft)


# GMRES iterations of the refined mixed solve of the P = 10^4 workload on a
# GB300 (all rounds), for the reference arm's extrapolation when it runs alone
P10K_MATVECS_PER_SOLVE = 44


def oracle_extrapolated(pk, n_matvec, seed=0):
    """The oracle's time for one solve of the P = 10^4 workload, extrapolated
    from timed samples of its own steps: the pair precompute of 2 sampled
    pairs (x C pairs), and its matvec of Algorithm 3 on 1 and on 3 target
    disks over all sources (the difference is the per-target-disk cost, x P
    disks; the intercept is Steps 1a-1b for all disks, paid once per matvec),
    times n_matvec matvecs (the right-hand side costs about one more).
    Returns (seconds per solve, sample description, measured parts)."""
    import numpy as np
    from oracle.geometry import contacts
    from oracle.pairs import pair_blocks
    from oracle.params import PACKING
    from oracle.system import System
    import workloads as w
    pairs = contacts(pk.centres, pk.radii, PACKING.delta_c)
    n4 = 4 * PACKING.Nc
    zero = {"A": np.zeros((n4, n4)), "E": np.zeros((6, n4))}   # same cost as real blocks
    so = System(pk.centres, pk.radii, PACKING, "mobility", blocks=[zero] * len(pairs), dense_limit=0)
    rng = np.random.default_rng(seed)
    picks = rng.choice(len(pairs), 2, replace=False)
    t0 = time.perf_counter()
    for q in picks:
        i, k = pairs[q]
        pair_blocks(pk.centres[i], pk.radii[i], pk.centres[k], pk.radii[k], so.ob[i], so.ob[k], PACKING,
                    "mobility", so.rho)
    t_pair = (time.perf_counter() - t0) / len(picks)
    mu = w.smooth_surface_vector(pk.P, PACKING.Mc, seed + 1).reshape(pk.P, -1)
    tg = rng.choice(pk.P, 3, replace=False)
    t0 = time.perf_counter()
    so.matvec(mu, targets=tg[:1])
    t1 = time.perf_counter()
    so.matvec(mu, targets=tg)
    t2 = time.perf_counter()
    per_disk = max(((t2 - t1) - (t1 - t0)) / 2, 1e-9)
    base = max((t1 - t0) - per_disk, 0.0)
    t_matvec = base + pk.P * per_disk
    total = len(pairs) * t_pair + (n_matvec + 1) * t_matvec
    sample = (f"extrapolated: pair precompute timed on 2 of {len(pairs)} pairs (x {len(pairs)}), matvec timed on "
              f"1 and 3 of {pk.P} target disks (x {pk.P}) over all {pk.P * PACKING.Nc} sources, x {n_matvec + 1} "
              f"matvecs per solve; numpy FP64")
    return total, sample, {"pair_s": t_pair, "matvec_s": t_matvec, "matvec_per_target_disk_s": per_disk,
                           "strengths_s": base, "n_pairs": len(pairs), "matvecs_per_solve": n_matvec + 1}


def oracle_checks(L, torch, s, pk, ft, n_disks=4, seed=11):
    """The timed solve checked by the oracle (not timed).  With the device's
    own pair blocks and one-body factors given to the oracle, on n_disks
    sampled target disks (the first the disk with the most contacts): the
    oracle's residual b - A x of the device solution x (the oracle's FP64
    right-hand side and its exclusion form of Algorithm 3), relative to |b| on
    those rows; and the device's FP64 and mixed matvecs of x on those rows
    against the oracle's."""
    import numpy as np
    from oracle.params import PACKING
    from oracle.system import System
    P = pk.P
    n = P * PACKING.Mc * 2
    x = torch.zeros(n, dtype=torch.float64, device="cuda")
    s.solution(x)
    torch.cuda.synchronize()
    A, E = s.pair_blocks(L.MOBILITY)
    so = System(pk.centres, pk.radii, PACKING, "mobility", blocks=[{"A": A[q], "E": E[q]} for q in range(len(A))],
                dense_limit=0)
    deg = np.zeros(P, dtype=int)
    for i, k in so.pairs:
        deg[i] += 1
        deg[k] += 1
    rng = np.random.default_rng(seed)
    tg = np.unique(np.concatenate([[int(np.argmax(deg))], rng.choice(P, n_disks - 1, replace=False)]))
    # the oracle's factors are its own truncated SVDs, the device's its QR: to
    # compare matvecs, both must use one of them -- give the device the SVD
    ob = so.ob[0]
    ns = 2 * PACKING.Nc
    r = ob.pinv.rank
    Ut = np.zeros((1, ns, ob.pinv.Ut.shape[1])); Ut[0, :r] = ob.pinv.Ut
    sg = np.ones((1, ns)); sg[0, :r] = ob.pinv.s[:r]
    V = np.zeros((1, ns, ns)); V[0, :, :r] = ob.pinv.VSi * ob.pinv.s[:r]
    xs = x.cpu().numpy().reshape(P, -1)
    # residual of the device's solution under the device's own operator (FP64)
    b = torch.zeros_like(x)
    s.rhs(L.MOBILITY, torch.tensor(ft.ravel(), dtype=torch.float64, device="cuda"), b, L.FP64)
    ax = torch.zeros_like(x)
    s.matvec(L.MOBILITY, x, ax, L.FP64)
    torch.cuda.synchronize()
    res_dev = float((b - ax).norm() / b.norm())
    b_or = so.rhs_mobility(ft, tg)
    s.set_onebody(L.MOBILITY, Ut, sg, V, np.array([r]))
    u_or = so.matvec_exclusion(xs, tg)
    out = {}
    for prec in (L.FP64, L.MIXED):
        ud = torch.zeros_like(x)
        s.matvec(L.MOBILITY, x, ud, prec)
        torch.cuda.synchronize()
        out[prec] = ud.cpu().numpy().reshape(P, -1)[tg]
    rel = lambda a, c: float(np.linalg.norm(a - c) / np.linalg.norm(c))
    return {"target_disks": [int(t) for t in tg], "rows": int(len(tg) * 2 * PACKING.Mc),
            "fp64_residual_all_rows_device": res_dev,
            "residual_sampled_rows_oracle_svd_factors": rel(u_or, b_or),
            "matvec_fp64_vs_oracle": rel(out[L.FP64], u_or), "matvec_mixed_vs_oracle": rel(out[L.MIXED], u_or),
            "note": "oracle: FP64 exclusion form of Algorithm 3 with the device's pair blocks and the oracle's "
                    "one-body SVD factors (the device solution x was computed with its QR factors, so the sampled "
                    "residual measures x against the SVD-factor operator)"}


def stokeslet_kernel_rate(L, torch, stream, precision):
    """Direct FP32 tile kernel at the P = 10^4 problem's size: 10^4 source
    disks x 60 sources on a square lattice (spacing 4.4) and 72 targets per
    lattice cell on a radius-0.5 circle about the cell centre (every target
    at least 4 ring radii from every disk centre)."""
    n = 100
    h = 4.4
    g = (np.arange(n) + 0.5) * h
    cx, cy = np.meshgrid(g, g)
    centres = np.stack([cx.ravel(), cy.ravel()], -1)
    th = 2 * np.pi * np.arange(60) / 60
    off = np.broadcast_to(np.stack([0.54 * np.cos(th), 0.54 * np.sin(th)], -1), (n * n, 60, 2)).copy()
    rng = np.random.default_rng(0)
    s = rng.standard_normal((n * n, 60, 2)) / 60
    tc = centres + h / 2
    ph = 2 * np.pi * np.arange(72) / 72
    targets = (tc[:, None, :] + 0.5 * np.stack([np.cos(ph), np.sin(ph)], -1)[None]).reshape(-1, 2)
    d = lambda x: torch.tensor(np.ascontiguousarray(x), dtype=torch.float64, device="cuda")
    T, Cc, O, S = d(targets), d(centres), d(off), d(s)
    out = torch.zeros_like(T)
    pairs = T.shape[0] * S.shape[0] * S.shape[1]
    l2_flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")   # L2 is 129 MB
    reps = 3
    evs = []
    with torch.cuda.stream(stream):
        for _ in range(3):   # warm-up; the first call of a size class also autotunes
            L.stokeslet_sum(T, Cc, O, S, precision=precision, stream=stream.cuda_stream, out=out)
        for _ in range(reps):
            l2_flush.zero_()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            L.stokeslet_sum(T, Cc, O, S, precision=precision, stream=stream.cuda_stream, out=out)
            e1.record(stream)
            evs.append((e0, e1))
    torch.cuda.synchronize()
    ms = sum(a.elapsed_time(b) for a, b in evs) / reps
    # sampled targets for an FP64 check (rank 0, beside the CPU baseline)
    idx = np.random.default_rng(1).choice(T.shape[0], 12, replace=False)
    sample = {"targets": targets[idx], "sources": (centres[:, None, :] + off).reshape(-1, 2), "s": s.reshape(-1),
              "gpu": out.cpu().numpy()[idx]}
    return {"targets": int(T.shape[0]), "sources": int(S.shape[0] * S.shape[1]), "ms_per_sum": ms,
            "gpair_per_s": pairs / (ms * 1e-3) / 1e9,
            "l2": "flushed before each timed sum (256 MiB write, not timed); 3 warm-up sums"}, sample


def stokeslet_sample_error(sample):
    """Relative 2-norm error of the sampled targets against FP64 direct summation."""
    from oracle.kernel import stokeslet
    ref = (stokeslet(sample["targets"], sample["sources"]) @ sample["s"]).reshape(-1, 2)
    return float(np.linalg.norm(sample["gpu"] - ref) / np.linalg.norm(ref))


def p100_side(L, torch, stream, local, n=10):
    """The P = 100 packing at area fraction 0.40 (mobility, tol 1e-7): device
    solves/s (each a full solve, precompute included) and the velocities'
    error against the oracle's solve of the same workload."""
    import numpy as np
    pk, ft = workload("p100_phi040_mobility")
    s = L.Solver(pk.centres, pk.radii, L.Params(precision=L.MIXED, tol=1e-7, stream=stream.cuda_stream, device=local))
    ft_d = torch.tensor(ft, dtype=torch.float64, device="cuda")
    out_d = torch.zeros_like(ft_d)
    for _ in range(3):
        s.invalidate()
        info = s.solve_device(L.MOBILITY, ft_d, out_d)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(n):
        s.invalidate()
        info = s.solve_device(L.MOBILITY, ft_d, out_d)
    e1.record(stream)
    e1.synchronize()
    ms = e0.elapsed_time(e1) / n
    v = out_d.cpu().numpy()
    tune = tune_summary(s.tune_report())
    s.close()
    t0 = time.perf_counter()
    ref, oinfo = oracle_solve(pk, ft)
    t_or = time.perf_counter() - t0
    return {"workload": "p100_phi040_mobility", "P": pk.P, "solves_per_s": 1e3 / ms, "ms_per_solve": ms,
            "gmres_iters": info["iters"], "refine_rounds": info["refine_rounds"], "fp64_relres": info["relres"],
            "velocity_err_vs_oracle": float(np.linalg.norm(v - ref) / np.linalg.norm(ref)),
            "oracle_solve_s": t_or, "oracle_gmres_iters": oinfo["iters"], "autotune": tune}


def serving_side(L, n=24, pmax=600, slots=8, seed=0):
    """A bounded serving stream (the serving workload's recipe with P
    log-uniform in [50, pmax] instead of [50, 5000], n requests): served in
    mixed precision (continuous batching, interleaved engine, refinement
    against the FP64 operator) at the stream's arrival times, and the SAME
    requests solved one at a time in FP64 on the GPU, first come first
    served.  Reports solves/s, request latency (arrival to result) p50/p99,
    and the served results' distance from the FP64 ones."""
    import numpy as np
    import workloads as w
    stream = w.serving_stream(n, seed=seed, pmax=pmax)
    prm = lambda: L.Params(tol=1e-7)
    srv = L.Server(hbm_budget_bytes=150 << 30, max_slots=slots, precision=L.MIXED, engine=0)
    pending, done, lat = {}, {}, {}
    q = 0
    start = time.perf_counter()
    while q < len(stream) or pending:
        now = time.perf_counter() - start
        while q < len(stream) and stream[q][0] <= now:
            _, pk, problem, data = stream[q]
            tk, P = srv.submit(pk.centres, pk.radii, problem, data, prm())
            pending[q] = (tk, P, start + stream[q][0])
            q += 1
        for k in list(pending):
            tk, P, t_arr = pending[k]
            rc, out, info = srv.poll(tk, P, timeout_us=0)
            if rc != L._lib.LMFS_PENDING:
                lat[k] = time.perf_counter() - t_arr
                done[k] = (rc, out, info)
                srv.forget(tk)
                del pending[k]
        time.sleep(0.0005)
    served_s = time.perf_counter() - start
    srv.close()
    ref, ref_info, solve_s = {}, {}, []
    t1 = time.perf_counter()
    for k, (_, pk, problem, data) in enumerate(stream):
        ts = time.perf_counter()
        so = L.Solver(pk.centres, pk.radii, L.Params(tol=1e-7, precision=L.FP64))
        ref[k], ref_info[k] = so.solve(problem, data)
        so.close()
        solve_s.append(time.perf_counter() - ts)
    seq_s = time.perf_counter() - t1
    seq_done, seq_lat = 0.0, []
    for k, (t_arr, _, _, _) in enumerate(stream):
        seq_done = max(seq_done, t_arr) + solve_s[k]
        seq_lat.append(seq_done - t_arr)
    both = [k for k in done if done[k][0] == 0 and ref_info[k]["converged"]]
    errs = [float(np.linalg.norm(done[k][1] - ref[k]) / np.linalg.norm(ref[k])) for k in both]
    lat_ms = np.array([lat[k] for k in sorted(lat)]) * 1e3
    return {"requests": n, "P_range": [min(x[1].P for x in stream), max(x[1].P for x in stream)],
            "recipe": f"serving stream, P log-uniform in [50, {pmax}], Poisson arrivals 20 ms apart, 50/50 "
                      "resistance/mobility, HBM budget 150 GB", "slots": slots, "tol": 1e-7,
            "served_mixed": {"solves_per_s": n / served_s, "wall_s": served_s,
                             "latency_ms": {"p50": float(np.percentile(lat_ms, 50)),
                                            "p99": float(np.percentile(lat_ms, 99))},
                             "not_converged": sum(done[k][0] != 0 for k in done)},
            "one_at_a_time_fp64": {"solves_per_s": n / seq_s, "wall_s": seq_s,
                                   "latency_ms": {"p50": float(np.percentile(seq_lat, 50) * 1e3),
                                                  "p99": float(np.percentile(seq_lat, 99) * 1e3)},
                                   "not_converged": sum(not ref_info[k]["converged"] for k in ref_info)},
            "solves_per_s_ratio": (n / served_s) / (n / seq_s),
            "served_vs_fp64_rel_2norm": {"both_converged": len(errs),
                                         "median": float(np.median(errs)) if errs else None,
                                         "max": float(np.max(errs)) if errs else None,
                                         "above_1e-5": int(sum(e > 1e-5 for e in errs))}}


def run_ours(args):
    import numpy as np
    import torch
    import torch.distributed as dist
    ws, rank, local = dist_env()
    if ws > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    from paper_2606_11273_gb300 import build as b
    b.build()
    import paper_2606_11273_gb300 as L
    from paper_2606_11273_gb300 import _lib
    problem, extra, tol = WORKLOADS[WORKLOAD]
    pk, ft = workload()
    stream = torch.cuda.Stream()
    prm = L.Params(precision=L.MIXED, tol=tol, stream=stream.cuda_stream, device=local, keep_fine=1, **extra)
    s = L.Solver(pk.centres, pk.radii, prm)
    ft_d = torch.tensor(ft, dtype=torch.float64, device="cuda")
    out_d = torch.zeros_like(ft_d)

    def step():
        s.invalidate()
        return s.solve_device(L.MOBILITY, ft_d, out_d)

    for _ in range(args.warmup):
        info = step()
    torch.cuda.synchronize()
    lat, infos, qr = [], [], []
    # L2 flush between timed steps: a 256 MiB write (L2 is 129 MB) on the
    # step's stream, inside the timed region
    l2_flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    if ws > 1:
        dist.barrier()
    torch.cuda.synchronize()
    n0 = _lib.launch_count()
    ev_all0, ev_all1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with Clocks(local) as clk:
        ev_all0.record(stream)
        for _ in range(args.steps):
            with torch.cuda.stream(stream):
                l2_flush.zero_()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            info = step()
            e1.record(stream)
            e1.synchronize()
            lat.append(e0.elapsed_time(e1))
            infos.append(info)
            qr.append(s.stats(L.MOBILITY))
        ev_all1.record(stream)
        torch.cuda.synchronize()
    if ws > 1:
        dist.barrier()
    launches = _lib.launch_count() - n0
    t_ms = job_time_ms(ev_all0.elapsed_time(ev_all1), ws, device="cuda")
    value = job_value(args.steps, ws, t_ms)
    vel_gpu = out_d.cpu().numpy()

    # end to end through the public host API: create + solve + destroy, inputs
    # from pinned host memory, the velocities read back every step
    e2e = None
    if rank == 0:
        n_e2e = max(1, min(args.steps, 2))
        c_h = torch.from_numpy(np.ascontiguousarray(pk.centres)).pin_memory().numpy()
        r_h = torch.from_numpy(np.ascontiguousarray(pk.radii)).pin_memory().numpy()
        f_h = torch.from_numpy(np.ascontiguousarray(ft)).pin_memory().numpy()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(n_e2e):
            s2 = L.Solver(c_h, r_h, L.Params(precision=L.MIXED, tol=tol, device=local, **extra))
            vel_e2e, info_e2e = s2.solve(L.MOBILITY, f_h)
            s2.close()
        e2e_ms = (time.perf_counter() - t0) * 1e3 / n_e2e
        e2e = {"value": 1e3 / e2e_ms, "unit": "solves/s", "h2d_bytes_per_step": int(c_h.nbytes + r_h.nbytes + f_h.nbytes),
               "d2h_bytes_per_step": int(pk.P * 3 * 8), "steps": n_e2e,
               "path": "lmfs_create + lmfs_solve (host in/out) + lmfs_destroy",
               "velocity_rel_diff_vs_timed_solve": float(np.linalg.norm(vel_e2e - vel_gpu) / np.linalg.norm(vel_gpu))}

    result = None
    if rank == 0:
        pk_ = peaks()
        sm_max = pk_.get("sm_max_mhz", 2070.0)
        fp64_peak_tf = 152 * 2 * 2 * sm_max * 1e6 / 1e12
        fp32_peak_tf = 152 * 128 * 2 * sm_max * 1e6 / 1e12
        fac_ms = float(np.mean([q["factor_ms"] for q in qr]))
        fac_tf = float(np.mean([q["factor_flops"] for q in qr])) / (fac_ms * 1e-3) / 1e12
        rhs_ms = float(np.mean([q["rhs_ms"] for q in qr]))
        rhs_tf = float(np.mean([q["rhs_flops"] for q in qr])) / (rhs_ms * 1e-3) / 1e12 if rhs_ms > 0 else None
        fine_ms = float(np.mean([q["fine_ms"] for q in qr]))
        fine_tf = float(np.mean([q["fine_flops"] for q in qr])) / (fine_ms * 1e-3) / 1e12
        fine_blocked = all(q["fine_blocked"] > 0 for q in qr)
        fine_emu = all(q["fine_blocked"] == 2 for q in qr)
        pre_ms = float(np.mean([q["precompute_ms"] for q in qr]))
        clocks = clk.summary()
        n_pairs = int(s.n_pairs)
        iters = int(np.median([x["iters"] for x in infos]))
        rounds = int(np.median([x["refine_rounds"] for x in infos]))
        # the timed solution's relative boundary residual (eq. (residual)) at
        # 144 new nodes per boundary, then the oracle's checks of it
        t0 = time.perf_counter()
        res_disk, rel_res = s.flow_boundary(L.MOBILITY, 144)
        flow = {"relative_boundary_residual": rel_res, "max_disk": float(res_disk.max()),
                "median_disk": float(np.median(res_disk)), "m_eval": 144, "eval_s": time.perf_counter() - t0,
                "definition": "max |u - g| over 144 new nodes per boundary / max |g| (u: two-body flow with each "
                              "pair's fine sources; g: v + omega (x - c)^perp)"}
        tune = tune_summary(s.tune_report())
        checks = oracle_checks(L, torch, s, pk, ft)
        dyn = dynamic_side(L, s, pk, ft, pre_ms)
        s.close()
        side = p100_side(L, torch, stream, local)
        stk, stk_sample = stokeslet_kernel_rate(L, torch, stream, L.FP32_FAST)
        stk_series, stk_series_sample = stokeslet_kernel_rate(L, torch, stream, L.MIXED_DIRECT)
        serving = serving_side(L) if not args.no_serving else None
        t_or, or_sample, or_parts = oracle_extrapolated(pk, iters + rounds)
        # DRAM traffic of rqr_kernel per step: the per-system figure of the
        # P = 160 capture times the step's fine half systems (two per pair)
        tr = rqr_traffic_per_matrix()
        traffic = tr * 2 * n_pairs if (tr is not None and fine_blocked) else None
        result = {
            "metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": t_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64+f32",
            "data": "synthetic (seeded packing and forces)",
            "config": {"workload": WORKLOAD, "P": int(pk.P), "n_pairs": n_pairs, "phi": 0.65, "min_gap": 1e-3,
                       "Nc": 60, "Mc": 72, "Nfp": 150, "Nell": 80, "Mp": 200, "tol": tol,
                       "precision": "mixed (FP32 far field), refined against the FP64 operator",
                       "far_field": "cells (one-level FMM)", "keep_fine": 1,
                       "l2": "flushed before every timed step (256 MiB write, counted in the time); the step "
                             "streams terabytes of pair-system QR traffic through DRAM and recomputes every "
                             "pair block",
                       "parallelism": f"replicas x{ws}"},
            "latency_ms": {"p50": float(np.percentile(lat, 50)), "p99": float(np.percentile(lat, 99)),
                           "mean": float(np.mean(lat)), "note": "per timed step (one solve each)"},
            "breakdown_ms": {"precompute": pre_ms, "qr_fine_systems": fine_ms, "qr_factor": fac_ms, "qr_rhs": rhs_ms,
                             "rest": float(np.mean(lat)) - pre_ms},
            "gmres_iters": iters, "refine_rounds": rounds,
            "fp64_relres": float(np.max([x["relres"] for x in infos])),
            "err_vs_oracle": checks,
            "boundary_residual": flow,
            "dynamic_geometry": dyn,
            "autotune": tune,
            "e2e": e2e,
            "gpu_launches": int(launches),
            "roofline": rqr_roofline(fine_emu, fine_blocked, fine_tf, fp64_peak_tf, sm_max, traffic,
                                     float(np.mean([q["fine_flops"] for q in qr])), fine_ms, t_ms / args.steps),
            "qr_all_stages": {"factor_ms": fac_ms, "factor_tflops": fac_tf, "rhs_ms": rhs_ms, "rhs_tflops": rhs_tf,
                              "note": "all pair QR launches of a step, fine and peanut systems: the blocked form "
                                      "(rqr_kernel, launches of >= 1216 systems; counted as factorization) or the "
                                      "pivoted cluster form (qrcp_kernel + apply_qt_kernel)"},
            "p100": side,
            "stokeslet_tile_kernel": {**stk, "kernel": "far32_lean_kernel (LMFS_FP32_FAST)", "flops_per_pair": 17,
                                      "achieved_tflops_17": stk["gpair_per_s"] * 17 / 1e3,
                                      "fp32_peak_tflops": fp32_peak_tf,
                                      "frac_17": stk["gpair_per_s"] * 17 / 1e3 / fp32_peak_tf,
                                      "err_vs_fp64_sampled": stokeslet_sample_error(stk_sample)},
            "stokeslet_series_kernel": {**stk_series, "kernel": "far32_kernel<2> (LMFS_MIXED_DIRECT)",
                                        "frac_17": stk_series["gpair_per_s"] * 17 / 1e3 / fp32_peak_tf,
                                        "err_vs_fp64_sampled": stokeslet_sample_error(stk_series_sample)},
            "serving": serving,
            "clocks": clocks,
            "cpu_baseline": {"value": 1.0 / t_or, "unit": "solves/s", "cores": os.cpu_count(),
                             "kind": "oracle", "sample": or_sample, "parts": or_parts,
                             "threads_note": "numpy elementwise sums run on one thread, BLAS on all cores"},
        }
        print(json.dumps(result))
    if ws > 1:
        dist.destroy_process_group()
    return result


def rqr_roofline(fine_emu, fine_blocked, fine_tf, fp64_peak_tf, sm_max, traffic, flops, fine_ms, step_ms):
    """Roofline of the fine systems' QR.  With FP64 trailing updates it is
    bound by the FP64 pipe; with the updates as exact bf16 digit products on
    the tensor cores the FP64 pipe no longer bounds it (it runs above that
    pipe's peak in FP64-equivalent flops), and the bound is the ALU pipe,
    which carries the digit extraction and the integer assembly of the
    products: the ceiling is the algorithm's flops per ALU warp instruction
    (from the capture) at the ALU pipe's full rate."""
    base = {"achieved": fine_tf, "traffic": traffic, "algorithmic_flops_per_step": flops,
            "traffic_note": "DRAM bytes per step: the ncu capture of rqr_kernel on 398 fine half systems "
                            "(P = 160), per system, times the 20940 of the step; null if the kernel changed since",
            "kernel_ms_per_step": fine_ms, "share_of_step": fine_ms / step_ms}
    if fine_emu:
        fpi = RQR_FLOPS_PER_ALU_INST if rqr_counters_valid() else None
        peak = fpi * 152 * ALU_WARP_INST_PER_CLK * sm_max * 1e6 / 1e12 if fpi else None
        return {"bound": "alu", "kernel": "rqr_kernel (blocked QR of the fine pair systems, pivots from a random "
                                          "sketch; trailing updates as exact bf16 digit products on the tensor "
                                          "cores, FP64-class)",
                "unit": "TFLOP/s (FP64-equivalent: the algorithm's FP64 flops)", "peak": peak,
                "frac": fine_tf / peak if peak else None, **base,
                "vs_fp64_pipe_peak": fine_tf / fp64_peak_tf,
                "peak_note": "derived: the launch's algorithmic flops per ALU-pipe warp instruction (ncu, P = 160 "
                             "capture) x 152 SMs x 2 ALU warp instructions per clock x max SM clock; "
                             "vs_fp64_pipe_peak compares with the FP64 pipe (152 x 2 FMA/clk x 2 x max clock)"}
    return {"bound": "alu", "kernel": ("rqr_kernel (blocked FP64 QR of the fine pair systems, pivots from a random "
                                       "sketch, right-hand sides in the same sweep)" if fine_blocked else
                                       "qrcp_kernel + apply_qt_kernel (pivoted FP64 QR of the fine pair systems)"),
            "unit": "TFLOP/s (FP64)", "peak": fp64_peak_tf, "frac": fine_tf / fp64_peak_tf, **base,
            "peak_note": "derived: 152 SMs x 2 FP64 FMA/clk x 2 flop x max SM clock (no FP64 figure in the "
                         "measured peaks)"}


def tune_summary(rows):
    """Per (kernel, precision): candidates timed, the occupancy model's shape
    and time, the chosen shape and time (the handle's first solve tunes)."""
    out = {}
    for r in rows:
        key = f"{r['kind']}_{'fp64' if r['precision'] == 0 else 'mixed'}"
        g = out.setdefault(key, {"candidates": 0})
        g["candidates"] += 1
        if r["model"]:
            g["model"] = [r["p1"], r["p2"], r["ms"]]
        if r["chosen"]:
            g["chosen"] = [r["p1"], r["p2"], r["ms"]]
    for g in out.values():
        if "model" in g and "chosen" in g and g["chosen"][2] > 0:
            g["speedup_vs_model"] = g["model"][2] / g["chosen"][2]
    return out or None


def dynamic_side(L, s, pk, ft, pre_ms):
    """One step of a moving geometry on the timed handle (after the timed
    region): 1% of the disks move by 0.3 of their smallest gap, the handle
    keeps the blocks of every pair whose relative position is unchanged and
    precomputes the others, then solves again."""
    import workloads as w
    newc, moved = w.move_disks(pk, pk.P // 100, seed=21)
    t0 = time.perf_counter()
    n = s.update_geometry(newc)
    t_upd = (time.perf_counter() - t0) * 1e3
    t0 = time.perf_counter()
    _, info = s.solve(L.MOBILITY, ft)
    t_solve = (time.perf_counter() - t0) * 1e3
    return {"moved_disks": int(len(moved)), "recomputed_pairs": int(n), "n_pairs": int(s.n_pairs),
            "update_ms": t_upd, "full_precompute_ms": pre_ms, "solve_after_ms": t_solve,
            "iters": info["iters"], "relres": info["relres"], "converged": info["converged"],
            "note": "update = contact detection, far-field tables and the recomputed pairs' blocks (kept "
                    "blocks gathered on the device); host wall time, one sample"}


def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    pk, ft = workload()
    vals, sample = [], ""
    for _ in range(args.warmup):
        oracle_extrapolated(pk, P10K_MATVECS_PER_SOLVE, seed=100)
    t0 = time.perf_counter()
    for k in range(args.steps):
        t_solve, sample, _ = oracle_extrapolated(pk, P10K_MATVECS_PER_SOLVE, seed=k)
        vals.append(t_solve)
    wall = time.perf_counter() - t0
    v = 1.0 / (sum(vals) / len(vals))
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": v, "unit": "solves/s", "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 / v, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic (seeded packing and forces)",
        "config": {"workload": WORKLOAD, "P": int(pk.P)},
        "sample_wall_s": wall,
        "cpu_baseline": {"value": v, "unit": "solves/s", "cores": os.cpu_count(), "kind": "oracle",
                         "sample": sample + f" ({P10K_MATVECS_PER_SOLVE} GMRES iterations per solve, as the GPU "
                                            "solve of this workload takes)"},
        "e2e": {"value": v, "unit": "solves/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}))


def run_large(args):
    """Non-default workloads: timings and full-size properties (no oracle solve)."""
    import torch
    from paper_2606_11273_gb300 import build as b
    b.build()
    import paper_2606_11273_gb300 as L
    problem, extra, tol = WORKLOADS[args.workload]
    code = L.MOBILITY if problem == "mobility" else L.RESISTANCE
    t0 = time.perf_counter()
    pk, data = workload(args.workload)
    t_geom = time.perf_counter() - t0
    stream = torch.cuda.Stream()
    res = {"workload": args.workload, "P": int(pk.P), "geometry_s": t_geom}
    for prec in (L.MIXED, L.FP64) if args.workload != "p10000_phi065_mobility" else (L.MIXED,):
        prm = L.Params(precision=prec, tol=tol, stream=stream.cuda_stream, **extra)
        s = L.Solver(pk.centres, pk.radii, prm)
        d_in = torch.tensor(data, dtype=torch.float64, device="cuda")
        d_out = torch.zeros_like(d_in)
        info = s.solve_device(code, d_in, d_out)          # includes the pair precompute
        st = s.stats(code)
        t1 = time.perf_counter()
        info2 = s.solve_device(code, d_in, d_out)         # blocks resident
        t_solve = time.perf_counter() - t1
        n = pk.P * prm.Mc * 2
        mu = torch.randn(n, dtype=torch.float64, device="cuda")
        u = torch.zeros_like(mu)
        s.matvec(code, mu, u, prec)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(3):
            s.matvec(code, mu, u, prec)
        e1.record(stream)
        e1.synchronize()
        r = {"n_pairs": s.n_pairs, "precompute_ms": st["precompute_ms"], "qr_ms": st["qr_ms"],
             "qr_tflops": st["qr_flops"] / (st["qr_ms"] * 1e-3) / 1e12, "rank_F": [st["min_rank_F"], st["max_rank_F"]],
             "iters": info["iters"], "relres": info["relres"], "converged": info["converged"],
             "solve_s_blocks_resident": t_solve, "matvec_ms": e0.elapsed_time(e1) / 3}
        if prec == L.MIXED:
            # full-size property: the mixed solution's residual under the FP64 operator
            x = torch.zeros(n, dtype=torch.float64, device="cuda")
            s.solution(x)
            bvec = torch.zeros_like(x)
            s.rhs(code, d_in, bvec, L.FP64)
            ax = torch.zeros_like(x)
            t2 = time.perf_counter()
            s.matvec(code, x, ax, L.FP64)
            torch.cuda.synchronize()
            r["fp64_matvec_s"] = time.perf_counter() - t2
            r["fp64_true_relres_of_mixed_solution"] = float((ax - bvec).norm() / bvec.norm())
            mixed_out = d_out.cpu().numpy()
        else:
            r["rel_diff_fp64_vs_mixed"] = float(np.linalg.norm(d_out.cpu().numpy() - mixed_out) / np.linalg.norm(d_out.cpu().numpy()))
        res["mixed" if prec == L.MIXED else "fp64"] = r
        s.close()
    print(json.dumps(res))


def _stats(xs):
    xs = [float(x) for x in xs]
    return {"mean": float(np.mean(xs)), "min": float(np.min(xs)), "max": float(np.max(xs))}


def _solve_case(L, pk, prm, code, data, m_eval):
    """One solve through the library: iterations, the relative boundary
    residual at m_eval new nodes per boundary, close pairs, solve time."""
    s = L.Solver(pk.centres, pk.radii, prm)
    t0 = time.perf_counter()
    out, info = s.solve(code, data)
    t = time.perf_counter() - t0
    _, rel_res = s.flow_boundary(code, m_eval)
    r = {"iters": info["iters"], "converged": info["converged"], "residual": rel_res, "n_pairs": int(s.n_pairs),
         "solve_s": t}
    return s, out, r


def experiment_delta(L, w, runs):
    """Sec. 6.1: random clusters with every disk at separation delta from a
    neighbour; the two-body solver against one-body preconditioning at the
    same coarse discretization (no pair blocks: delta_c = 0), and the
    two-way error (mobility output fed to the resistance solve)."""
    # peanut nodes: Mp = 10 N_c / 3 (rounded to even) keeps the peanut fit as
    # overdetermined as Sec. 6.2's M_p = 200 at N_c = 60; at N_c = 128 the
    # default 200 nodes give fewer equations (400) than unknowns (512)
    cases = {
        "mobility": (50, dict(Nc=80, Mc=96, Nfp=60, Nell=100, Mp=268), L.MOBILITY, (1e-1, 1e-2, 1e-3, 1e-4)),
        "resistance": (20, dict(Nc=128, Mc=154, Nfp=120, Nell=100, Mp=428), L.RESISTANCE, (1e-1, 1e-2, 1e-3)),
    }
    out = {}
    for name, (P, kw, code, deltas) in cases.items():
        rows = []
        for delta in deltas:
            agg = {"two_body": [], "one_body": [], "two_way": [], "pairs_per_body": []}
            for q in range(runs):
                pk = w.cluster(P, delta, seed=100 * q + 7)
                data = w.forces_torques(P, q) if code == L.MOBILITY else w.rigid_velocities(P, q)
                m_eval = 2 * kw["Mc"]
                prm = L.Params(precision=L.FP64, tol=1e-7, keep_fine=1, **kw)
                s, res, r2 = _solve_case(L, pk, prm, code, data, m_eval)
                s.close()
                if code == L.MOBILITY:
                    # two-way error (Sec. 6.1): the resistance output (forces
                    # of N(0, 1) velocities) fed to the mobility solve, against
                    # those velocities; GMRES at 1e-11 so that its tolerance
                    # does not hide the discretization's share, and both
                    # solves' boundary residuals beside it
                    s2 = L.Solver(pk.centres, pk.radii,
                                  L.Params(precision=L.FP64, tol=1e-11, maxit=1000, keep_fine=1, **kw))
                    uv = w.rigid_velocities(P, 50 + q)
                    f, i_r = s2.solve(L.RESISTANCE, uv)
                    _, res_r = s2.flow_boundary(L.RESISTANCE, m_eval)
                    v2, i_m = s2.solve(L.MOBILITY, f)
                    _, res_m = s2.flow_boundary(L.MOBILITY, m_eval)
                    s2.close()
                    agg["two_way"].append({"error": float(np.linalg.norm(v2 - uv) / np.linalg.norm(uv)),
                                           "residual_resistance": res_r, "residual_mobility": res_m,
                                           "iters": [i_r["iters"], i_m["iters"]],
                                           "converged": bool(i_r["converged"] and i_m["converged"])})
                s1, _, r1 = _solve_case(L, pk, L.Params(precision=L.FP64, tol=1e-7, keep_fine=1, delta_c=0.0, **kw),
                                        code, data, m_eval)
                s1.close()
                agg["two_body"].append(r2)
                agg["one_body"].append(r1)
                agg["pairs_per_body"].append(2.0 * r2["n_pairs"] / P)
            row = {"delta": delta, "runs": runs, "pairs_per_body": _stats(agg["pairs_per_body"])}
            for k in ("two_body", "one_body"):
                row[k] = {"iters": _stats([r["iters"] for r in agg[k]]),
                          "residual": _stats([r["residual"] for r in agg[k]]),
                          "solve_s": _stats([r["solve_s"] for r in agg[k]]),
                          "not_converged": sum(1 for r in agg[k] if not r["converged"])}
            if agg["two_way"]:
                tw = agg["two_way"]
                row["two_way"] = {"error": _stats([r["error"] for r in tw]),
                                  "over_residual": _stats([r["error"] / max(r["residual_resistance"],
                                                                            r["residual_mobility"]) for r in tw]),
                                  "tol": 1e-11, "per_run": tw}
            row["per_run"] = {k: [{"iters": r["iters"], "residual": r["residual"]} for r in agg[k]]
                              for k in ("two_body", "one_body")}
            rows.append(row)
        out[name] = {"P": P, "params": kw, "tol": 1e-7, "precision": "fp64", "m_eval": 2 * kw["Mc"], "rows": rows}
    return out


def experiment_packing(L, w, sweep, runs):
    """Sec. 6.2: mobility on random packings (square lattice + Metropolis
    sweeps, minimum gap 1e-3), GMRES tol 1e-7: iterations, close neighbours
    per body and the relative boundary residual, over `runs` packings per
    point; sweep "phi" fixes P = 500, sweep "P" fixes phi = 0.65."""
    pts = ([(500, phi) for phi in (0.30, 0.40, 0.50, 0.60, 0.65)] if sweep == "phi"
           else [(P, 0.65) for P in (100, 300, 1000, 3000, 10000)])
    rows = []
    for P, phi in pts:
        n = runs if P <= 1000 else max(1, runs // (3 if P <= 3000 else 10))
        rs = []
        for q in range(n):
            pk = w.packing(P, phi, seed=1000 + q, gmin=1e-3, nsweep=10 if P <= 3000 else 6)
            ft = w.forces_torques(P, q)
            prm = L.Params(precision=L.FP64, tol=1e-7, keep_fine=1)
            s, _, r = _solve_case(L, pk, prm, L.MOBILITY, ft, 144)
            s.close()
            r["pairs_per_body"] = 2.0 * r["n_pairs"] / P
            rs.append(r)
        rows.append({"P": P, "phi": phi, "runs": n, "iters": _stats([r["iters"] for r in rs]),
                     "pairs_per_body": _stats([r["pairs_per_body"] for r in rs]),
                     "residual": _stats([r["residual"] for r in rs]),
                     "solve_s": _stats([r["solve_s"] for r in rs]),
                     "not_converged": sum(1 for r in rs if not r["converged"])})
    return {"sweep": sweep, "precision": "fp64", "tol": 1e-7, "m_eval": 144, "rows": rows}


def run_experiment(args):
    """The paper's experiments through the library on the GPU (side reports,
    one JSON line): --experiment delta (Sec. 6.1), phi or P (Sec. 6.2)."""
    from paper_2606_11273_gb300 import build as b
    b.build()
    import paper_2606_11273_gb300 as L
    import workloads as w
    t0 = time.perf_counter()
    if args.experiment == "delta":
        res = experiment_delta(L, w, args.runs if args.runs else 5)
    else:
        res = experiment_packing(L, w, args.experiment, args.runs if args.runs else 10)
    res["experiment"] = args.experiment
    res["wall_s"] = time.perf_counter() - t0
    print(json.dumps(res))


def run_serving(args):
    """Serving stream (Poisson arrivals, mixed disk counts and problems)
    through the continuous-batching server in the mixed-precision form,
    against the same requests solved one at a time in FP64 on the GPU.
    Prints one JSON line (a side report; the contract line is the default run)."""
    import torch
    from paper_2606_11273_gb300 import build as b
    b.build()
    import paper_2606_11273_gb300 as L
    import workloads as w
    t0 = time.perf_counter()
    stream = w.serving_stream(args.requests, seed=0, pmax=args.pmax)
    t_gen = time.perf_counter() - t0
    prm = lambda: L.Params(tol=1e-7)
    # warm-up: load the library, first-use costs of CUDA
    pk0 = w.packing(20, 0.4, 1, gmin=1e-2, start="square", nsweep=2)
    s0 = L.Solver(pk0.centres, pk0.radii, prm()); s0.solve(L.MOBILITY, w.forces_torques(20, 1)); s0.close()
    torch.cuda.synchronize()
    # served, mixed precision: submit at the arrival times, poll without blocking
    srv = L.Server(hbm_budget_bytes=150 << 30, max_slots=args.slots, precision=L.MIXED, engine=args.engine)
    pending, done, lat = {}, {}, {}
    q = 0
    start = time.perf_counter()
    with Clocks(0) as clk:
        while q < len(stream) or pending:
            now = time.perf_counter() - start
            while q < len(stream) and stream[q][0] <= now:
                t_arr, pk, problem, data = stream[q]
                tk, P = srv.submit(pk.centres, pk.radii, problem, data, prm())
                pending[q] = (tk, P, time.perf_counter())
                q += 1
            for k in list(pending):
                tk, P, ts = pending[k]
                rc, out, info = srv.poll(tk, P, timeout_us=0)
                if rc != L._lib.LMFS_PENDING:
                    lat[k] = time.perf_counter() - ts
                    done[k] = (rc, out, info)
                    del pending[k]
            time.sleep(0.0005)
    served_s = time.perf_counter() - start
    srv.close()
    # one at a time, FP64, on the first nb requests of the same stream
    nb = min(len(stream), args.baseline_requests)
    ref, ref_info, seq_lat = {}, {}, []
    t1 = time.perf_counter()
    for k, (t_arr, pk, problem, data) in enumerate(stream[:nb]):
        ts = time.perf_counter()
        so = L.Solver(pk.centres, pk.radii, L.Params(tol=1e-7, precision=L.FP64))
        out, info = so.solve(problem, data)
        so.close()
        ref[k] = out
        ref_info[k] = info
        seq_lat.append(time.perf_counter() - ts)
    seq_s = time.perf_counter() - t1
    # the same arrivals served first come, first served by the one-at-a-time form
    seq_done, seq_queue_lat = 0.0, []
    for k, (t_arr, _, _, _) in enumerate(stream[:nb]):
        seq_done = max(seq_done, t_arr) + seq_lat[k]
        seq_queue_lat.append(seq_done - t_arr)
    ok = [k for k in ref if done[k][0] == 0 and ref_info[k]["converged"]]
    errs = {k: float(np.linalg.norm(done[k][1] - ref[k]) / np.linalg.norm(ref[k])) for k in ok}
    bad = [k for k in done if done[k][0] != 0]
    desc = lambda k: {"P": stream[k][1].P, "problem": "mobility" if stream[k][2] else "resistance",
                      "phi": round(float(stream[k][1].meta.get("phi", 0.0)), 3),
                      "gmin": float(stream[k][1].meta.get("gmin", 0.0)), "iters": int(done[k][2]["iters"])}
    lat_ms = np.array([lat[k] for k in sorted(lat)]) * 1e3
    Ps = [x[1].P for x in stream]
    print(json.dumps({
        "serving": {"requests": len(stream), "P_range": [min(Ps), max(Ps)], "P_median": float(np.median(Ps)),
                    "mean_arrival_gap_ms": 20.0, "hbm_budget_gb": 150, "slots": args.slots, "engine": ["interleaved", "streams"][args.engine], "tol": 1e-7,
                    "generation_s": t_gen},
        "served_mixed": {"solves_per_s": len(stream) / served_s, "wall_s": served_s,
                         "latency_ms": {"p50": float(np.percentile(lat_ms, 50)), "p99": float(np.percentile(lat_ms, 99)),
                                        "max": float(lat_ms.max())}},
        "one_at_a_time_fp64": {"requests": nb, "solves_per_s": nb / seq_s, "wall_s": seq_s,
                               "latency_ms": {"p50": float(np.percentile(seq_queue_lat, 50) * 1e3),
                                              "p99": float(np.percentile(seq_queue_lat, 99) * 1e3),
                                              "note": "same arrival times, first come first served"},
                               "solve_ms": {"p50": float(np.percentile(seq_lat, 50) * 1e3),
                                            "p99": float(np.percentile(seq_lat, 99) * 1e3)}},
        "solves_per_s_ratio": (len(stream) / served_s) / (nb / seq_s),
        "served_not_converged": {"count": len(bad),
                                 "by_problem": {"resistance": sum(stream[k][2] == 0 for k in bad),
                                                "mobility": sum(stream[k][2] == 1 for k in bad)},
                                 "fp64_not_converged_of_baseline": sum(not ref_info[k]["converged"] for k in ref_info)},
        "iters_median": {"served": float(np.median([done[k][2]["iters"] for k in done])),
                         "fp64": float(np.median([ref_info[k]["iters"] for k in ref_info]))},
        "served_vs_fp64_rel_2norm": {"both_converged": len(errs),
                                     "median": float(np.median(list(errs.values()))) if errs else None,
                                     "max": float(np.max(list(errs.values()))) if errs else None,
                                     "above_1e-5": [dict(desc(k), err=errs[k]) for k in errs if errs[k] > 1e-5]},
        "clocks": clk.summary()}))


def run_profile_case(case):
    """Small, bounded cases for ncu captures (a few launches of one kernel)."""
    import torch
    from paper_2606_11273_gb300 import build as b
    b.build()
    import paper_2606_11273_gb300 as L
    stream = torch.cuda.Stream()
    if case in ("m2p_large", "matvec_large"):
        # P = 10^4 packing with zero pair blocks (no precompute): far field only
        pk, _ = workload("p10000_phi065_mobility")
        s = L.Solver(pk.centres, pk.radii, L.Params(precision=L.MIXED, stream=stream.cuda_stream))
        C = s.n_pairs
        s.set_pair_blocks(L.MOBILITY, np.zeros((C, 240, 240)), np.zeros((C, 6, 240)))
        mu = torch.randn(pk.P * 144, dtype=torch.float64, device="cuda")
        u = torch.zeros_like(mu)
        for _ in range(2):
            s.matvec(L.MOBILITY, mu, u, L.MIXED)
        if case == "matvec_large":
            s.matvec(L.MOBILITY, mu, u, L.FP64)
        torch.cuda.synchronize()
    elif case == "qr_large":
        # the P = 10^4 pair precompute (23 chunks of <= 456 pairs)
        pk, _ = workload("p10000_phi065_mobility")
        s = L.Solver(pk.centres, pk.radii, L.Params(precision=L.MIXED, stream=stream.cuda_stream))
        s.precompute(L.MOBILITY)
        torch.cuda.synchronize()
    elif case == "qr_mid":
        # P = 160 at area fraction 0.65: 398 fine half systems, one launch
        import workloads as w
        pk = w.packing(160, 0.65, 5, gmin=1e-3)
        s = L.Solver(pk.centres, pk.radii, L.Params(precision=L.MIXED, stream=stream.cuda_stream))
        s.precompute(L.MOBILITY)
        torch.cuda.synchronize()
        st = s.stats(L.MOBILITY)
        print(f"qr_mid: {2 * s.n_pairs} fine half systems, fine QR {st['fine_ms']:.2f} ms, "
              f"{st['fine_flops']:.6e} algorithmic flops, form {st['fine_blocked']:.0f}")
    elif case in ("qr", "matvec"):
        pk, ft = workload("p100_phi040_mobility")
        s = L.Solver(pk.centres, pk.radii, L.Params(precision=L.MIXED, stream=stream.cuda_stream))
        s.precompute(L.MOBILITY)
        if case == "qr":
            s.invalidate()
            s.precompute(L.MOBILITY)
        else:
            n = pk.P * 72 * 2
            mu = torch.randn(n, dtype=torch.float64, device="cuda")
            u = torch.zeros_like(mu)
            for _ in range(3):
                s.matvec(L.MOBILITY, mu, u, L.MIXED)
        torch.cuda.synchronize()
    elif case in ("stokeslet", "stokeslet_fast"):
        # 2000 source disks x 60 sources, 2000 x 72 targets (1.7e10 pairs)
        n = 45
        h = 4.4
        g = (np.arange(n) + 0.5) * h
        cx, cy = np.meshgrid(g, g)
        centres = np.stack([cx.ravel(), cy.ravel()], -1)[:2000]
        th = 2 * np.pi * np.arange(60) / 60
        off = np.broadcast_to(np.stack([0.54 * np.cos(th), 0.54 * np.sin(th)], -1), (2000, 60, 2)).copy()
        s = np.random.default_rng(0).standard_normal((2000, 60, 2)) / 60
        ph = 2 * np.pi * np.arange(72) / 72
        targets = ((centres + h / 2)[:, None, :] + 0.5 * np.stack([np.cos(ph), np.sin(ph)], -1)[None]).reshape(-1, 2)
        d = lambda x: torch.tensor(np.ascontiguousarray(x), dtype=torch.float64, device="cuda")
        T, Cc, O, S = d(targets), d(centres), d(off), d(s)
        prec = L.FP32_FAST if case == "stokeslet_fast" else L.MIXED_DIRECT
        for _ in range(2):
            L.stokeslet_sum(T, Cc, O, S, precision=prec, stream=stream.cuda_stream)
        torch.cuda.synchronize()
    print(f"profile case {case} done")


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--profile-case", default=None, choices=["qr", "qr_mid", "qr_large", "matvec", "stokeslet", "stokeslet_fast", "m2p_large", "matvec_large"],
                    help="run one small bounded case for an ncu capture and exit")
    ap.add_argument("--serving", action="store_true",
                    help="serving stream: served mixed precision against one-at-a-time FP64 (side report)")
    ap.add_argument("--requests", type=int, default=64, help="serving: requests in the stream (the full stream has 256)")
    ap.add_argument("--pmax", type=int, default=5000, help="serving: largest disk count")
    ap.add_argument("--slots", type=int, default=8, help="serving: concurrent request slots")
    ap.add_argument("--engine", type=int, default=0, choices=[0, 1],
                    help="serving: 0 = interleaved (one far-field launch for all ready requests), 1 = a stream per request")
    ap.add_argument("--baseline-requests", type=int, default=24,
                    help="serving: requests (from the start of the stream) solved one at a time in FP64")
    ap.add_argument("--no-serving", action="store_true", help="default run: leave out the bounded serving key")
    ap.add_argument("--workload", default=WORKLOAD, choices=sorted(WORKLOADS),
                    help="non-default workloads print timings and full-size checks, not the contract line")
    ap.add_argument("--experiment", default=None, choices=["delta", "phi", "P"],
                    help="the paper's experiments on the GPU: delta-sweep clusters (Sec. 6.1), phi- or P-sweep "
                         "packings (Sec. 6.2); prints one JSON line")
    ap.add_argument("--runs", type=int, default=0, help="experiment: runs per point (default 5 delta, 10 sweeps)")
    args = ap.parse_args()
    if args.experiment:
        run_experiment(args)
        return
    if args.profile_case:
        run_profile_case(args.profile_case)
        return
    if args.serving:
        run_serving(args)
        return
    if args.workload != WORKLOAD:
        run_large(args)
        return
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
