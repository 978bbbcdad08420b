"""Benchmark: batched GPU solves of the locally compressed MFS on one GB300.

Default workload: P = 100 unit disks at area fraction 0.40 (random sequential
placement, minimum gap 1e-2), mobility problem with per-disk N(0,1) forces
(net force shifted to zero) and torques, 72 vector unknowns per body
(N_c = 60, M_c = 72), fine pair parameters N_fp = 150, N_ell = 80, M_p = 200,
GMRES tol 1e-7.  One step = one complete solve of that batch on the device:
contact detection, one-body factors and every pair block (batched QR), the
completion-flow right-hand side, GMRES with the two-body matvec, and the
velocity post-processing.  Inputs are resident in device memory before the
timed region; `e2e` repeats the measurement through the host API (geometry
and forces copied in, velocities copied out, every step).

Also reported: the dominant kernel's roofline (the batched FP64 QR, from CUDA
events on the handle's stream inside the library), the Stokeslet direct-tile
kernel's pair rate at the P = 10^4 problem's size (7.2e5 targets x 6e5
sources), per-step p50/p99 latency, SM clocks sampled during the timed
region, and the CPU oracle's time for the same solve on this host.

--impl reference times the CPU oracle itself (plain FP64 numpy) on the same
workload.  Multi-GPU: the solve does not shard, so N ranks run independent
replicas (weak scaling; value = all ranks' solves / max-over-ranks time).
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
WORKLOAD = "p100_phi040_mobility"


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


# DRAM traffic of the pivoted-QR kernel (qrcp_kernel) per timed step -- its two
# launches, the fine pair systems and the peanut systems of the P = 100 batch --
# from one ncu capture (dram__bytes_read.sum + dram__bytes_write.sum; command
# and figures in profiles/qrcp_kernel_p100_mobility.md).  Valid only for the
# kernel source it was taken on: reported as null once lmfs_qr.cu changes.
QRCP_TRAFFIC_BYTES = 23436956160 + 25761400320 + 14299136 + 2100224
QRCP_TRAFFIC_SRC_SHA256 = "3ce04c663094e62340580234a338a11233c67842ce496f69c0fbeeff384884f9"


def qrcp_traffic():
    import hashlib
    src = os.path.join(ROOT, "paper_2606_11273_gb300", "csrc", "lmfs_qr.cu")
    try:
        h = hashlib.sha256(open(src, "rb").read()).hexdigest()
    except OSError:
        return None
    return QRCP_TRAFFIC_BYTES if h == QRCP_TRAFFIC_SRC_SHA256 else None


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


def run_ours(args):
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
    pk, ft = workload()
    stream = torch.cuda.Stream()
    prm = L.Params(precision=L.MIXED, tol=1e-7, stream=stream.cuda_stream, device=local)
    s = L.Solver(pk.centres, pk.radii, prm)
    ft_d = torch.tensor(ft, dtype=torch.float64, device="cuda")
    out_d = torch.zeros_like(ft_d)

    def step():
        s.invalidate()
        return s.solve_device(L.MOBILITY, ft_d, out_d)

    for _ in range(args.warmup):
        info = step()
    torch.cuda.synchronize()
    vel_gpu = out_d.cpu().numpy()
    lat, qr_ms, qr_flops, fac, rhs = [], [], [], [], []
    iters = []
    # L2 flush between timed steps: a 256 MiB write (L2 is 129 MB) on the
    # step's stream, inside the timed region (about 40 us per step)
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
            st = s.stats(L.MOBILITY)
            qr_ms.append(st["qr_ms"])
            qr_flops.append(st["qr_flops"])
            fac.append((st["factor_ms"], st["factor_flops"]))
            rhs.append((st["rhs_ms"], st["rhs_flops"]))
            iters.append(info["iters"])
        ev_all1.record(stream)
        torch.cuda.synchronize()
    if ws > 1:
        dist.barrier()
    launches = _lib.launch_count() - n0
    t_ms = job_time_ms(ev_all0.elapsed_time(ev_all1), ws, device="cuda")
    value = job_value(args.steps, ws, t_ms)

    # end to end through the public host API: create + solve (host in/out) + destroy
    e2e_ms = None
    if rank == 0:
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(args.steps):
            s2 = L.Solver(pk.centres, pk.radii, L.Params(precision=L.MIXED, tol=1e-7, device=local))
            vel_e2e, _ = s2.solve(L.MOBILITY, ft)
            s2.close()
        e2e_ms = (time.perf_counter() - t0) * 1e3 / args.steps

    result = None
    if rank == 0:
        pk_ = peaks()
        # FP64 peak of this part from unit counts and clocks: 152 SMs x 2 DFMA/clk x 2 flop
        sm_max = pk_.get("sm_max_mhz", 2070.0)
        fp64_peak_tf = 152 * 2 * 2 * sm_max * 1e6 / 1e12
        qr_t = float(np.mean(qr_ms))
        fac_ms = float(np.mean([f[0] for f in fac])); fac_tf = float(np.mean([f[1] for f in fac])) / (fac_ms * 1e-3) / 1e12
        rhs_ms = float(np.mean([f[0] for f in rhs])); rhs_tf = float(np.mean([f[1] for f in rhs])) / (rhs_ms * 1e-3) / 1e12
        stk, stk_sample = stokeslet_kernel_rate(L, torch, stream, L.FP32_FAST)
        stk_series, stk_series_sample = stokeslet_kernel_rate(L, torch, stream, L.MIXED_DIRECT)
        fp32_peak_tf = 152 * 128 * 2 * sm_max * 1e6 / 1e12
        # accuracy of the timed result against the oracle (not timed)
        t0 = time.perf_counter()
        vel_ref, oinfo = oracle_solve(pk, ft)
        oracle_s = time.perf_counter() - t0
        err = float(np.linalg.norm(vel_gpu - vel_ref) / np.linalg.norm(vel_ref))
        err_e2e = float(np.linalg.norm(vel_e2e - vel_ref) / np.linalg.norm(vel_ref))
        clocks = clk.summary()
        nbytes_in = (pk.P * 2 + pk.P + pk.P * 3) * 8
        result = {
            "metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": t_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64+f32",
            "data": "synthetic (seeded packing and forces)",
            "config": {"workload": WORKLOAD, "P": int(pk.P), "n_pairs": int(s.n_pairs), "Nc": 60, "Mc": 72,
                       "Nfp": 150, "Nell": 80, "Mp": 200, "tol": 1e-7, "precision": "mixed (FP32 far field)",
                       "l2": "flushed before every timed step (256 MiB write, counted in the time); each step also streams ~49 GB of pair-system QR traffic through DRAM and recomputes every pair block",
                       "parallelism": f"replicas x{ws}"},
            "latency_ms": {"p50": float(np.percentile(lat, 50)), "p99": float(np.percentile(lat, 99)),
                           "mean": float(np.mean(lat))},
            "gmres_iters": int(np.median(iters)),
            "err_vs_oracle": {"velocity_rel_2norm": err, "e2e_velocity_rel_2norm": err_e2e},
            "e2e": {"value": 1e3 / e2e_ms, "unit": "solves/s", "h2d_bytes_per_step": nbytes_in,
                    "d2h_bytes_per_step": pk.P * 3 * 8},
            "gpu_launches": int(launches),
            "roofline": {"bound": "alu", "kernel": "qrcp_kernel (pivoted FP64 QR of the pair systems, 2 launches/step)",
                         "achieved": fac_tf, "peak": fp64_peak_tf, "unit": "TFLOP/s (FP64)",
                         "frac": fac_tf / fp64_peak_tf, "traffic": qrcp_traffic(),
                         "traffic_note": "DRAM bytes of the step's qrcp launches from ncu, null if the kernel changed",
                         "peak_note": "derived: 152 SMs x 2 FP64 FMA/clk x 2 flop x max SM clock",
                         "kernel_ms_per_step": fac_ms, "share_of_step": fac_ms / (t_ms / args.steps)},
            "roofline_rhs": {"bound": "alu", "kernel": "apply_qt_kernel (Q^T B and back substitution)",
                             "achieved": rhs_tf, "peak": fp64_peak_tf, "unit": "TFLOP/s (FP64)",
                             "frac": rhs_tf / fp64_peak_tf, "kernel_ms_per_step": rhs_ms},
            "qr_ms_per_step": qr_t,
            "stokeslet_tile_kernel": {**stk, "kernel": "far32_lean_kernel (LMFS_FP32_FAST)", "flops_per_pair": 17,
                                      "achieved_tflops_17": stk["gpair_per_s"] * 17 / 1e3,
                                      "fp32_peak_tflops": fp32_peak_tf,
                                      "frac_17": stk["gpair_per_s"] * 17 / 1e3 / fp32_peak_tf,
                                      "err_vs_fp64_sampled": stokeslet_sample_error(stk_sample)},
            "stokeslet_series_kernel": {**stk_series, "kernel": "far32_kernel<2> (LMFS_MIXED_DIRECT)",
                                        "frac_17": stk_series["gpair_per_s"] * 17 / 1e3 / fp32_peak_tf,
                                        "err_vs_fp64_sampled": stokeslet_sample_error(stk_series_sample)},
            "clocks": clocks,
            "cpu_baseline": {"value": 1.0 / oracle_s, "unit": "solves/s", "cores": os.cpu_count(),
                             "kind": "oracle", "sample": "one full solve of the same workload (numpy FP64)",
                             "gmres_iters": oinfo["iters"]},
        }
        print(json.dumps(result))
    if ws > 1:
        dist.destroy_process_group()
    return result


def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    pk, ft = workload()
    for _ in range(args.warmup):
        oracle_solve(pk, ft)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        oracle_solve(pk, ft)
    t = time.perf_counter() - t0
    v = args.steps / t
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": v, "unit": "solves/s", "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": t * 1e3 / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic (seeded packing and forces)",
        "config": {"workload": WORKLOAD, "P": int(pk.P)},
        "cpu_baseline": {"value": v, "unit": "solves/s", "cores": os.cpu_count(), "kind": "oracle",
                         "sample": "full solves of the workload, numpy FP64 on the host cores"},
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
        torch.cuda.synchronize()
    elif case in ("qr", "matvec"):
        pk, ft = workload()
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
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--profile-case", default=None, choices=["qr", "matvec", "stokeslet", "stokeslet_fast", "m2p_large", "matvec_large"],
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
    ap.add_argument("--workload", default=WORKLOAD, choices=sorted(WORKLOADS),
                    help="non-default workloads print timings and full-size checks, not the contract line")
    args = ap.parse_args()
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
