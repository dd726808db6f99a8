"""Parity at the full size of the 3D elasticity workload on 64^3 vertices
(774,144 dofs), in the launch configuration bench.py times (library setup,
AMG_LAYOUT_AUTO with the kernel tuner, PCG graph with programmatic launches;
the FP64 variant re-uploads the downloaded prolongations, as the bench's
precision variants do).  The oracle runs its own solve phase on the same
prolongations (Galerkin products, smoothers, coarsest factor, V-cycle, PCG:
oracle/solve.py), and every vector is compared element by element
(max_i |gpu_i - oracle_i| <= tol * max_i |oracle_i|):

* every coarse matrix A_{l+1} = P_l^T A_l P_l built on the device against
  the oracle's Galerkin product: rowptr and colidx bit-exact, values 1e-12;
* A_0 x (FP64), whole vector: 1e-12;
* one FP64 V-cycle against the oracle V-cycle: 1e-10; the FP32 V-cycle of
  the bench's main context: 1e-4;
* FP64 PCG against the oracle PCG: iterations +-1, iterates 1e-10 at equal
  iteration counts, FP64 true residual <= 1.5e-8;
* PCG with the FP32 V-cycle: FP64 true residual <= 1.5e-8 and energy-norm
  error <= 1e-6 against the oracle's own tight solve (rtol 1e-12).
"""
import numpy as np
import pytest

from oracle import solve
from workloads import configs

torch = pytest.importorskip("torch")
pytestmark = [pytest.mark.gpu, pytest.mark.slow]

_S = {}


def _amg():
    from paper_2011_13325_gb300 import amg
    return amg


def maxrel(a, b):
    a, b = np.asarray(a), np.asarray(b)
    assert a.shape == b.shape
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))


def state():
    if not _S:
        amg = _amg()
        p = configs.cube64()
        ctx = amg.Context(0)
        ctx.setup(p, amg.AMG_PREC_FP32_VCYCLE)
        P_list = [ctx.download_prolongation(l) for l in range(ctx.n_levels - 1)]
        Ps = [solve.Mat(n, m, rp.astype(np.int64), ci.astype(np.int64), v)
              for (n, m, rp, ci, v) in P_list]
        H = solve.prepare(solve.mat_from(p.A), Ps)         # the oracle's solve phase
        c64 = amg.Context(0)
        c64.upload_hierarchy(p.A, [type("P", (), dict(n_rows=n, n_cols=m, rowptr=rp, colidx=ci,
                                                      vals=v)) for (n, m, rp, ci, v) in P_list],
                             amg.AMG_PREC_FP64)
        _S.update(p=p, ctx=ctx, c64=c64, H=H)
    return _S


def _dev(x):
    return torch.from_numpy(np.ascontiguousarray(x, dtype=np.float64)).cuda()


def test_fullsize_galerkin_matches_oracle_exactly():
    st = state()
    H = st["H"]
    for c in (st["ctx"], st["c64"]):
        assert c.n_levels == H.n_levels
        for l in range(1, H.n_levels):
            rp, ci, v = c.download_matrix(l)
            A = H.A[l]
            np.testing.assert_array_equal(rp, A.rowptr)
            np.testing.assert_array_equal(ci, A.colidx)
            assert np.abs(v - A.vals).max() <= 1e-12 * np.abs(A.vals).max(), l


def test_fullsize_spmv_whole_vector():
    st = state()
    H = st["H"]
    n = H.A[0].n_rows * H.A[0].br
    x = np.random.default_rng(0).normal(size=n)
    y = torch.zeros(n, dtype=torch.float64, device="cuda")
    st["ctx"].spmv(0, _dev(x), y)
    assert maxrel(y.cpu().numpy(), solve.spmv(H.A[0], x)) <= 1e-12


def test_fullsize_vcycle_matches_oracle():
    st = state()
    H = st["H"]
    n = H.A[0].n_rows * H.A[0].br
    rng = np.random.default_rng(3)
    for r in (st["p"].b[0], rng.normal(size=n)):
        zo = solve.vcycle(H, r)
        z = torch.zeros(n, dtype=torch.float64, device="cuda")
        st["c64"].vcycle(_dev(r), z)
        assert maxrel(z.cpu().numpy(), zo) <= 1e-10
        z.zero_()
        st["ctx"].vcycle(_dev(r), z)
        assert maxrel(z.cpu().numpy(), zo) <= 1e-4


def test_fullsize_fp64_pcg_matches_oracle():
    st = state()
    p, H, c64 = st["p"], st["H"], st["c64"]
    f = p.b[0]
    u_or, it_or, _ = solve.pcg(H, f, rtol=1e-8, maxit=1000)
    u = torch.zeros(f.shape[0], dtype=torch.float64, device="cuda")
    _, its, rr = c64.pcg_solve(_dev(f), u, rtol=1e-8, maxit=1000)
    assert abs(its[0] - it_or) <= 1, (its, it_or)
    assert rr[0] <= 1e-8
    u_k = u_or if its[0] == it_or else solve.pcg(H, f, rtol=0.0, maxit=its[0])[0]
    uh = u.cpu().numpy()
    assert maxrel(uh, u_k) <= 1e-10
    assert np.linalg.norm(f - solve.spmv(H.A[0], uh)) <= 1.5e-8 * np.linalg.norm(f)
    _S["u_or"] = u_or


def test_fullsize_mixed_pcg_residual_and_energy_vs_oracle():
    st = state()
    p, ctx, H = st["p"], st["ctx"], st["H"]
    f = p.b[0]
    u = torch.zeros(f.shape[0], dtype=torch.float64, device="cuda")
    _, its, rr = ctx.pcg_solve(_dev(f), u, rtol=1e-8, maxit=1000)
    uh = u.cpu().numpy()
    A = H.A[0]
    assert np.linalg.norm(f - solve.spmv(A, uh)) <= 1.5e-8 * np.linalg.norm(f)
    # the oracle's own tight solve, started from its 1e-8 solution if present
    ue, _, hist = solve.pcg(H, f, rtol=1e-12, maxit=2000, x0=_S.get("u_or"))
    e = uh - ue
    energy = np.sqrt(e @ solve.spmv(A, e) / (ue @ solve.spmv(A, ue)))
    assert energy <= 1e-6, energy
