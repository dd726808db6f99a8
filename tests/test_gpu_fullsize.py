"""Parity at the full size of the default bench workload (3D elasticity on
64^3 vertices, 774,144 dofs), in the launch configuration bench.py times
(library setup, AMG_LAYOUT_AUTO with the kernel tuner, PCG graph with
programmatic launches): sampled outputs the oracle computes row by row, and
properties that hold at any size.

* A_0 x (FP64) on 300 sampled block rows: 1e-12 relative;
* A_1 = P_0^T A_0 P_0 built on the device, 200 sampled block rows against
  the same rows of the sparse product on the host: pattern exact, 1e-12;
* V-cycle (FP64) symmetric and positive on random vectors;
* PCG with the FP32 V-cycle: FP64 true residual <= 1.5e-8 and energy-norm
  error <= 1e-6 against a tight FP64 solve on the same hierarchy.
"""
import numpy as np
import pytest
import scipy.sparse as sp

from oracle import solve
from workloads import configs

torch = pytest.importorskip("torch")
pytestmark = [pytest.mark.gpu, pytest.mark.slow]

_S = {}


def _amg():
    from paper_2011_13325_gb300 import amg
    return amg


def state():
    if not _S:
        amg = _amg()
        p = configs.cube64()
        ctx = amg.Context(0)
        ctx.setup(p, amg.AMG_PREC_FP32_VCYCLE)
        _S.update(p=p, ctx=ctx, A=solve.mat_from(p.A))
    return _S


def _block_rows(M, rows):
    """Dense block rows of a BSR Mat as {col: block}."""
    out = []
    for r in rows:
        s, e = M.rowptr[r], M.rowptr[r + 1]
        out.append({int(c): M.vals[q] for q, c in zip(range(s, e), M.colidx[s:e])})
    return out


def test_fullsize_spmv_sampled_rows():
    st = state()
    A, ctx = st["A"], st["ctx"]
    n = A.n_rows * 3
    x = np.random.default_rng(0).normal(size=n)
    y = torch.zeros(n, dtype=torch.float64, device="cuda")
    ctx.spmv(0, torch.from_numpy(x).cuda(), y)
    y = y.cpu().numpy()
    rows = np.random.default_rng(1).choice(A.n_rows, 300, replace=False)
    for r, blocks in zip(rows, _block_rows(A, rows)):
        want = sum(B @ x[3 * c:3 * c + 3] for c, B in blocks.items())
        got = y[3 * r:3 * r + 3]
        assert np.abs(got - want).max() <= 1e-12 * np.abs(want).max() + 1e-300


def test_fullsize_galerkin_sampled_rows():
    st = state()
    A, ctx = st["A"], st["ctx"]
    n1, m1, rp, ci, v = ctx.download_prolongation(0)
    P = sp.bsr_matrix((v, ci, rp), shape=(n1 * 3, m1 * 6)).tocsr()
    As = A.scipy()
    rp1, ci1, v1 = ctx.download_matrix(1)
    rows = np.random.default_rng(2).choice(m1, 200, replace=False)
    PT = P.T.tocsr()
    for r in rows:
        # block row r of P^T A P from the host sparse product of 6 scalar rows
        Rr = PT[6 * r:6 * r + 6]
        dense = (Rr @ As @ P).toarray()                # 6 x (6 m1)
        s, e = rp1[r], rp1[r + 1]
        cols = ci1[s:e]
        # every structurally nonzero block column of the product is stored
        nz = np.nonzero(np.abs(dense).reshape(6, m1, 6).sum(axis=(0, 2)))[0]
        assert set(nz.tolist()) <= set(cols.tolist())
        scale = np.abs(dense).max()
        for q, c in zip(range(s, e), cols):
            assert np.abs(v1[q] - dense[:, 6 * c:6 * c + 6]).max() <= 1e-12 * scale


def test_fullsize_vcycle_symmetric_positive():
    amg = _amg()
    st = state()
    p = st["p"]
    ctx = amg.Context(0)
    Ps = []
    for l in range(st["ctx"].n_levels - 1):
        n, m, rp, ci, v = st["ctx"].download_prolongation(l)
        Ps.append(type("P", (), dict(n_rows=n, n_cols=m, rowptr=rp, colidx=ci, vals=v)))
    ctx.upload_hierarchy(p.A, Ps, amg.AMG_PREC_FP64)
    n = p.A.n_rows * 3
    rng = np.random.default_rng(3)
    a, b = rng.normal(size=(2, n))
    za = torch.zeros(n, dtype=torch.float64, device="cuda")
    zb = torch.zeros_like(za)
    ctx.vcycle(torch.from_numpy(a).cuda(), za)
    ctx.vcycle(torch.from_numpy(b).cuda(), zb)
    za, zb = za.cpu().numpy(), zb.cpu().numpy()
    assert abs(b @ za - a @ zb) <= 1e-10 * abs(a @ za)
    assert a @ za > 0 and b @ zb > 0
    _S["ctx64"] = ctx


def test_fullsize_mixed_pcg_residual_and_energy():
    st = state()
    p, ctx, A = st["p"], st["ctx"], st["A"]
    f = torch.from_numpy(p.b[0]).cuda()
    u = torch.zeros_like(f)
    _, its, rr = ctx.pcg_solve(f, u, rtol=1e-8, maxit=1000)
    uh = u.cpu().numpy()
    true = np.linalg.norm(p.b[0] - solve.spmv(A, uh)) / np.linalg.norm(p.b[0])
    assert true <= 1.5e-8
    ctx64 = st.get("ctx64")
    if ctx64 is None:
        pytest.skip("needs the FP64 context of the previous test")
    ue = torch.zeros_like(f)
    ctx64.pcg_solve(f, ue, rtol=1e-13, maxit=3000, check=False)
    ue = ue.cpu().numpy()
    e = uh - ue
    energy = np.sqrt(e @ solve.spmv(A, e) / (ue @ solve.spmv(A, ue)))
    assert energy <= 1e-6
