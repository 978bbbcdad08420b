"""The matvec autotuner through the C ABI: before the first GMRES iteration
of a precision is captured, a handle times the near kernel's launch shapes
(and the all-pairs far field's source splits) on the solve's right-hand side
and keeps the fastest, cached per size class.  Checked: one choice per kernel
and precision, the fastest of its candidates; a second handle of the class
reuses it without timing and solves bitwise like the first; and the matvec
with the chosen shapes equals the occupancy models' shapes to rounding."""
import numpy as np
import pytest

import workloads as w
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


def matvec(L, s, x, prec):
    md = torch.tensor(x.ravel(), dtype=torch.float64, device="cuda")
    ud = torch.zeros_like(md)
    s.matvec(L.MOBILITY, md, ud, prec)
    torch.cuda.synchronize()
    return ud.cpu().numpy()


def test_autotuner_choices_reuse_and_results(L):
    # a packing of its own size class (P = 97), so that no earlier test's
    # handle has filled the cache for it
    pk = w.packing(97, 0.40, 21, gmin=1e-2, start="rsa", nsweep=10, step=0.3)
    ft = w.forces_torques(pk.P, 3)
    mu = w.smooth_surface_vector(pk.P, PACKING.Mc, 4)
    ref = L.Solver(pk.centres, pk.radii, gparams(L, PACKING))
    ref.precompute(L.MOBILITY)
    u_model = {p: matvec(L, ref, mu, p) for p in (L.FP64, L.MIXED)}
    s = L.Solver(pk.centres, pk.radii, gparams(L, PACKING))
    v1, info1 = s.solve(L.MOBILITY, ft)
    assert info1["converged"]
    rows = s.tune_report()
    print("\n".join(f"{r['kind']:4s} prec {r['precision']} ({r['p1']:2d}, {r['p2']:3d}) {r['ms']:.4f} ms"
                    f"{' *' if r['chosen'] else ''}" for r in rows))
    kinds = {(r["kind"], r["precision"]) for r in rows}
    assert ("near", L.MIXED) in kinds
    for key in kinds:
        grp = [r for r in rows if (r["kind"], r["precision"]) == key]
        chosen = [r for r in grp if r["chosen"]]
        assert len(chosen) == 1 and len(grp) >= 2
        assert chosen[0]["ms"] <= min(r["ms"] for r in grp) * (1 + 1e-9)
        assert sum(r["model"] for r in grp) == 1
    # the tuned shapes give the models' results to rounding
    # (a different split reorders the FP32 far field's partial sums: 1e-6 for mixed)
    for p, tol in ((L.FP64, 1e-13), (L.MIXED, 1e-6)):
        u = matvec(L, s, mu, p)
        d = np.linalg.norm(u - u_model[p]) / np.linalg.norm(u_model[p])
        print(f"precision {p}: tuned vs model shapes {d:.2e}")
        assert d < tol
    # a second handle of the class: no timing, the same choices, the same solve
    s2 = L.Solver(pk.centres, pk.radii, gparams(L, PACKING))
    v2, info2 = s2.solve(L.MOBILITY, ft)
    assert s2.tune_report() == []
    assert info2["iters"] == info1["iters"] and np.array_equal(v2, v1)
    for h in (ref, s, s2):
        h.close()
