"""The pair precompute's two QR forms through the C ABI: the blocked QR with
pivots chosen on a random sketch (one matrix per CTA, the form large batches
use, with its trailing updates as exact digit products on the tensor cores or
in FP64; two CTAs per matrix in FP64) and the column-pivoted cluster form
(small batches).  LMFS_QR_PATH, LMFS_QR_CS and LMFS_QR_EMU force a form.  Both truncate at the same level and differ only in
numerically null directions, so the unique parts of the blocks -- E and C A
-- are compared with the oracle's SVD-truncated blocks, and the solves with
each other."""
import numpy as np
import pytest

import workloads as w
from oracle.onebody import OneBody
from oracle.pairs import pair_blocks
from oracle.params import PACKING

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def L():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    from paper_2606_11273_gb300 import build
    build.build()
    import paper_2606_11273_gb300 as lib
    return lib


def gparams(L, p, **kw):
    base = dict(Nc=p.Nc, Mc=p.Mc, Rc=p.Rc, Nfp=p.Nfp, Nell=p.Nell, Mp=p.Mp, delta_c=p.delta_c, tol=p.tol,
                gamma=p.gamma, af=p.af, r_mob=p.r_mob, aell=p.aell, eps_trunc=p.eps_trunc,
                eps_trunc_fine=p.eps_trunc_fine, mu=p.mu)
    base.update(kw)
    return L.Params(**base)


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b)))


def solver(L, monkeypatch, path, pk, problem, cs=None, emu=None, **kw):
    monkeypatch.setenv("LMFS_QR_PATH", path)
    if cs:
        monkeypatch.setenv("LMFS_QR_CS", cs)
    if emu is not None:
        monkeypatch.setenv("LMFS_QR_EMU", emu)
    s = L.Solver(pk.centres, pk.radii, gparams(L, PACKING, **kw))
    s.precompute(problem)
    monkeypatch.delenv("LMFS_QR_PATH")
    if cs:
        monkeypatch.delenv("LMFS_QR_CS")
    if emu is not None:
        monkeypatch.delenv("LMFS_QR_EMU")
    return s


@pytest.mark.parametrize("cs,emu", [("1", "1"), ("1", "0"), ("2", None)])
@pytest.mark.parametrize("problem", ["mobility", "resistance"])
def test_blocked_qr_pair_blocks_against_oracle(L, monkeypatch, problem, cs, emu):
    """P = 100 packing (37 close pairs): on 8 sampled pairs E and C A of the
    blocked form -- one CTA per system with the trailing updates on the tensor
    cores or in FP64, and two CTAs (a cluster) per system in FP64, the form of
    mid-size batches without the tensor-core updates -- against the oracle's
    SVD blocks within 1e-5, as the cluster form's are; the fine ranks of the
    forms within a few columns."""
    code = L.MOBILITY if problem == "mobility" else L.RESISTANCE
    pk = w.packing_p100()
    sb = solver(L, monkeypatch, "blocked", pk, code, cs=cs, emu=emu)
    sc = solver(L, monkeypatch, "cluster", pk, code)
    Ab, Eb = sb.pair_blocks(code)
    Ac, Ec = sc.pair_blocks(code)
    stb, stc = sb.stats(code), sc.stats(code)
    ob = OneBody(1.0, PACKING, problem)
    pairs = sb.pairs()
    worst = {"blocked": [0.0, 0.0], "cluster": [0.0, 0.0]}
    for q in np.linspace(0, len(pairs) - 1, 8).astype(int):
        i, k = pairs[q]
        b = pair_blocks(pk.centres[i], 1.0, pk.centres[k], 1.0, ob, ob, PACKING, problem, 1.0, keep=True)
        for name, A, E in (("blocked", Ab, Eb), ("cluster", Ac, Ec)):
            worst[name][0] = max(worst[name][0], rel(E[q], b["E"]))
            worst[name][1] = max(worst[name][1], rel(b["C"] @ A[q], b["C"] @ b["A"]))
    print(f"{problem}, {cs} CTA(s) per system, tensor-core updates {emu}: E, C A vs oracle: blocked {worst['blocked'][0]:.2e} {worst['blocked'][1]:.2e}, "
          f"cluster {worst['cluster'][0]:.2e} {worst['cluster'][1]:.2e}; rank F blocked "
          f"[{stb['min_rank_F']:.0f}, {stb['max_rank_F']:.0f}] cluster [{stc['min_rank_F']:.0f}, {stc['max_rank_F']:.0f}]; "
          f"QR ms blocked {stb['qr_ms']:.1f} cluster {stc['qr_ms']:.1f}")
    assert worst["blocked"][0] < 1e-5 and worst["blocked"][1] < 1e-5
    assert abs(stb["min_rank_F"] - stc["min_rank_F"]) <= 8 and abs(stb["max_rank_F"] - stc["max_rank_F"]) <= 8
    sb.close()
    sc.close()


def test_blocked_qr_solves_like_the_cluster_form(L, monkeypatch):
    """The P = 100 mobility solve (FP64) on blocks from either form: the
    velocities agree within 1e-6 (each is within ~3e-7 of the oracle)."""
    pk = w.packing_p100()
    ft = w.forces_torques(pk.P, 5)
    out = {}
    for path in ("blocked", "cluster"):
        s = solver(L, monkeypatch, path, pk, L.MOBILITY, precision=L.FP64)
        out[path], info = s.solve(L.MOBILITY, ft)
        assert info["converged"]
        s.close()
    d = rel(out["blocked"], out["cluster"])
    print(f"velocities blocked vs cluster {d:.2e}")
    assert d < 1e-6


@pytest.mark.parametrize("problem", ["mobility", "resistance"])
def test_tensor_core_updates_match_fp64_updates(L, monkeypatch, problem):
    """The blocked form with its trailing updates as exact digit products on
    the tensor cores against the same form with FP64 updates, P = 100: the
    same fine ranks on every pair, every E within 1e-9 (measured 1.9e-11 and
    3.6e-13: the two differ by rounding, the digit products being exact), and
    the FP64 mobility solve on either set of blocks within 1e-6."""
    code = L.MOBILITY if problem == "mobility" else L.RESISTANCE
    pk = w.packing_p100()
    se = solver(L, monkeypatch, "blocked", pk, code, cs="1", emu="1", precision=L.FP64)
    sf = solver(L, monkeypatch, "blocked", pk, code, cs="1", emu="0", precision=L.FP64)
    Ae, Ee = se.pair_blocks(code)
    Af, Ef = sf.pair_blocks(code)
    ste, stf = se.stats(code), sf.stats(code)
    assert ste["min_rank_F"] == stf["min_rank_F"] and ste["max_rank_F"] == stf["max_rank_F"]
    dE = max(rel(Ee[q], Ef[q]) for q in range(len(Ee)))
    print(f"{problem}: E tensor-core vs FP64 updates, worst pair {dE:.2e}; fine QR ms {ste['fine_ms']:.1f} "
          f"against {stf['fine_ms']:.1f}")
    assert dE < 1e-9
    if code == L.MOBILITY:
        ft = w.forces_torques(pk.P, 5)
        ve, ie = se.solve(code, ft)
        vf, if_ = sf.solve(code, ft)
        assert ie["converged"] and if_["converged"]
        assert rel(ve, vf) < 1e-6
    se.close()
    sf.close()


def test_digit_dz_matches_fp64_dz(L, monkeypatch):
    """The pair precompute's D Z product as exact digit products on the
    tensor cores (the default) against the FP64 kernel (LMFS_DZ_EMU=0),
    P = 100 mobility: C A -- the part of A the method uses, A being unique
    only up to C's null directions -- on 4 sampled pairs within 1e-8 (the two
    products differ by rounding, which the peanut system's truncated solve
    amplifies: measured 2.0e-9, against 2.2e-7 for either set of blocks
    against the oracle's), E unchanged, and the FP64 solves on either set of
    blocks within 1e-6 (measured 6.2e-7, GMRES stopping at 1e-7)."""
    pk = w.packing_p100()
    ft = w.forces_torques(pk.P, 5)
    out = {}
    for dz in ("1", "0"):
        monkeypatch.setenv("LMFS_DZ_EMU", dz)
        s = L.Solver(pk.centres, pk.radii, gparams(L, PACKING, precision=L.FP64))
        s.precompute(L.MOBILITY)
        monkeypatch.delenv("LMFS_DZ_EMU")
        A, E = s.pair_blocks(L.MOBILITY)
        v, info = s.solve(L.MOBILITY, ft)
        assert info["converged"]
        out[dz] = (A, E, v, s.pairs().copy())
        s.close()
    (Ad, Ed, vd, pairs), (Af, Ef, vf, _) = out["1"], out["0"]
    assert np.array_equal(Ed, Ef)
    ob = OneBody(1.0, PACKING, "mobility")
    worst = 0.0
    for q in np.linspace(0, len(pairs) - 1, 4).astype(int):
        i, k = pairs[q]
        b = pair_blocks(pk.centres[i], 1.0, pk.centres[k], 1.0, ob, ob, PACKING, "mobility", 1.0, keep=True)
        worst = max(worst, rel(b["C"] @ Ad[q], b["C"] @ Af[q]))
    dv = rel(vd, vf)
    print(f"C A digit vs FP64 D Z: worst sampled pair {worst:.2e}; FP64 velocities {dv:.2e}")
    assert worst < 1e-8
    assert dv < 1e-6
