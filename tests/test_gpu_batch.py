"""Batched solve (amg_batch_*): independent systems of uneven size with six
load cases each, solved by one graph launch, against the FP64 oracle PCG on
the same hierarchies, load case by load case.

FP64: iteration counts +-1 and iterates 1e-10 relative at equal iteration
counts (the multi-load-case kernels sum in another order than the oracle).
FP32 / BF16-storage V-cycle: FP64 true residual <= 1.5e-8 and energy-norm
error <= 1e-6 against the FP64 oracle solution.  The CG product in
double-float arithmetic (48 significant bits per value): iteration counts
+-1 and iterates 1e-8.
"""
import numpy as np
import pytest

from oracle import hierarchy, solve
from workloads import configs, make_problem

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

LOADS_2D = [[1, 0], [-1, 0], [0, 1], [0, -1], [1, 1], [-1, 1]]


def _amg():
    from paper_2011_13325_gb300 import amg
    return amg


def _systems():
    """Uneven 3D boxes (h = 1/32, per-system E and nu), one 2D square and one
    system whose hierarchy is a single (coarsest) level."""
    out = []
    for i, (shape, E, nu) in enumerate([((6, 7, 5), 2.0, 0.3), ((8, 8, 8), 0.5, 0.25),
                                        ((5, 9, 6), 7.0, 0.38), ((10, 6, 7), 1.0, 0.2)]):
        p = make_problem(shape, seed=20 + i, h=1.0 / 32, E=E, nu=nu, forces=configs.SIX_LOADS)
        out.append((p, hierarchy.setup(p, hierarchy.SetupParams(coarse_max=8))))
    p = make_problem((13, 11), seed=30, forces=LOADS_2D)
    out.append((p, hierarchy.setup(p, hierarchy.SetupParams(coarse_max=8))))
    p = make_problem((4, 3, 3), seed=31, h=1.0 / 32, forces=configs.SIX_LOADS)
    out.append((p, hierarchy.setup(p, hierarchy.SetupParams(coarse_max=10000))))
    return out


_SYS = []


def systems():
    if not _SYS:
        _SYS.extend(_systems())
    return _SYS


def _batch(prec, nrhs=6, layout=0, cg_op=None):
    amg = _amg()
    ctxs = []
    for p, H in systems():
        c = amg.Context(0)
        if layout:
            c.set_layout_policy(layout)
        c.upload_hierarchy(H.A[0], H.P, prec)
        if cg_op is not None:
            c.set_cg_operator(cg_op)
        ctxs.append(c)
    return ctxs, amg.Batch(ctxs, nrhs)


def _stack(B, loads):
    """Stacked device f from per-system (nrhs, n) arrays."""
    total = B.layout(0)[2]
    f = np.zeros(total)
    for s, F in enumerate(loads):
        off, n, _ = B.layout(s)
        f[off:off + F.size] = F.reshape(-1)
    return torch.from_numpy(f).cuda()


def _unstack(B, u, nrhs):
    torch.cuda.synchronize()
    uh = u.cpu().numpy()
    out = []
    for s in range(len(B.contexts)):
        off, n, _ = B.layout(s)
        out.append(uh[off:off + nrhs * n].reshape(nrhs, n))
    return out


def maxrel(a, b):
    """Element-wise error: max_i |a_i - b_i| / max_i |b_i|."""
    a, b = np.asarray(a), np.asarray(b)
    assert a.shape == b.shape
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))


def test_single_level_hierarchy_present():
    assert systems()[-1][1].n_levels == 1
    assert all(H.n_levels >= 2 for _, H in systems()[:-1])


def test_layout_is_stacked_per_system():
    ctxs, B = _batch(0)
    off = 0
    for s, (p, H) in enumerate(systems()):
        o, n, total = B.layout(s)
        assert o == off and n == H.A[0].n_rows * H.A[0].br
        off += 6 * n
    assert total == off
    with pytest.raises(_amg().AmgError):
        B.layout(len(systems()))


@pytest.mark.parametrize("layout", [0, 2, 1], ids=["auto", "warp", "sell"])
def test_batch_fp64_matches_oracle(layout):
    ctxs, B = _batch(0, layout=layout)
    f = _stack(B, [p.b for p, _ in systems()])
    u = torch.zeros_like(f)
    s, its, rr, ms = B.pcg_solve(f, u, rtol=1e-8, maxit=500)
    assert ms > 0
    us = _unstack(B, u, 6)
    for si, (p, H) in enumerate(systems()):
        for j in range(6):
            it = its[si * 6 + j]
            _, it_or, _ = solve.pcg(H, p.b[j], rtol=1e-8, maxit=500)
            assert abs(it - it_or) <= 1, (si, j, it, it_or)
            assert rr[si * 6 + j] <= 1e-8
            u_k, _, _ = solve.pcg(H, p.b[j], rtol=0.0, maxit=it)
            assert maxrel(us[si][j], u_k) <= 1e-10, (si, j)
            true = np.linalg.norm(p.b[j] - solve.spmv(H.A[0], us[si][j])) / np.linalg.norm(p.b[j])
            assert true <= 1.5e-8


def test_batch_double_float_cg_product_matches_oracle():
    """The batched CG product q = A_0 p in double-float arithmetic (contexts
    set to AMG_CG_DOUBLE_FLOAT before the batch is created; FP64 V-cycle, so
    the rest is as in the FP64 test): every load case within +-1 iteration
    of the oracle's PCG, its iterate within 1e-8 of the oracle's at the same
    count, true residual <= 1.5e-8; with the FP64 V-cycle and AMG_CG_AUTO the
    product stays FP64, with the FP32 V-cycle AUTO takes the double-float
    one."""
    amg = _amg()
    ctxs, B = _batch(0, cg_op=amg.AMG_CG_DOUBLE_FLOAT)
    assert "q = A_0 p (double-float)" in B.describe()
    f = _stack(B, [p.b for p, _ in systems()])
    u = torch.zeros_like(f)
    s, its, rr, ms = B.pcg_solve(f, u, rtol=1e-8, maxit=500)
    us = _unstack(B, u, 6)
    for si, (p, H) in enumerate(systems()):
        for j in range(6):
            it = its[si * 6 + j]
            _, it_or, _ = solve.pcg(H, p.b[j], rtol=1e-8, maxit=500)
            assert abs(it - it_or) <= 1, (si, j, it, it_or)
            u_k, _, _ = solve.pcg(H, p.b[j], rtol=0.0, maxit=it)
            assert maxrel(us[si][j], u_k) <= 1e-8, (si, j)
            true = np.linalg.norm(p.b[j] - solve.spmv(H.A[0], us[si][j])) / np.linalg.norm(p.b[j])
            assert true <= 1.5e-8
    _, B64 = _batch(0)
    assert "double-float" not in B64.describe()
    _, B32 = _batch(1)
    assert "q = A_0 p (double-float)" in B32.describe()


def test_batch_single_load_case_matches_context_solve():
    """nrhs = 1: each system's load case 0 agrees with the single-system
    amg_pcg_solve (same iteration counts +-1, iterates 1e-10)."""
    ctxs, B = _batch(0, nrhs=1)
    f = _stack(B, [p.b[:1] for p, _ in systems()])
    u = torch.zeros_like(f)
    s, its, rr, ms = B.pcg_solve(f, u, rtol=1e-8)
    us = _unstack(B, u, 1)
    for si, (p, H) in enumerate(systems()):
        ud = torch.zeros(p.b.shape[1], dtype=torch.float64, device="cuda")
        _, it1, _ = ctxs[si].pcg_solve(torch.from_numpy(p.b[0]).cuda(), ud, rtol=1e-8)
        assert abs(its[si] - it1[0]) <= 1
        u_k, _, _ = solve.pcg(H, p.b[0], rtol=0.0, maxit=its[si])
        assert maxrel(us[si][0], u_k) <= 1e-10


@pytest.mark.parametrize("prec", [1, 2], ids=["fp32", "bf16"])
def test_batch_mixed_precision_reaches_fp64_tolerance(prec):
    ctxs, B = _batch(prec)
    f = _stack(B, [p.b for p, _ in systems()])
    u = torch.zeros_like(f)
    s, its, rr, ms = B.pcg_solve(f, u, rtol=1e-8, maxit=500)
    us = _unstack(B, u, 6)
    for si, (p, H) in enumerate(systems()):
        A = H.A[0]
        for j in range(6):
            uh = us[si][j]
            true = np.linalg.norm(p.b[j] - solve.spmv(A, uh)) / np.linalg.norm(p.b[j])
            assert true <= 1.5e-8, (si, j, true)
            u_ex, it64, _ = solve.pcg(H, p.b[j], rtol=1e-13, maxit=1000)
            e = uh - u_ex
            energy = np.sqrt(e @ solve.spmv(A, e) / (u_ex @ solve.spmv(A, u_ex)))
            assert energy <= 1e-6, (si, j, energy)
            _, it8, _ = solve.pcg(H, p.b[j], rtol=1e-8)
            assert its[si * 6 + j] <= it8 + 10


def test_batch_deterministic_and_restart():
    ctxs, B = _batch(0)
    f = _stack(B, [p.b for p, _ in systems()])
    u1, u2 = torch.zeros_like(f), torch.zeros_like(f)
    _, it1, r1, _ = B.pcg_solve(f, u1, rtol=1e-8)
    _, it2, r2, _ = B.pcg_solve(f, u2, rtol=1e-8)
    assert it1 == it2 and r1 == r2 and torch.equal(u1, u2)
    # started from its own solution every load case needs no iteration
    _, it3, _, _ = B.pcg_solve(f, u2, rtol=1e-6)
    assert max(it3) == 0 and torch.equal(u1, u2)


def test_batch_frozen_and_unconverged_load_cases():
    amg = _amg()
    ctxs, B = _batch(0)
    loads = []
    for p, _ in systems():
        F = p.b.copy()
        F[2] = 0.0  # a load case with f = 0 is done before the first iteration
        loads.append(F)
    f = _stack(B, loads)
    u = torch.zeros_like(f)
    s, its, rr, _ = B.pcg_solve(f, u, rtol=1e-8)
    assert s == amg.AMG_OK
    us = _unstack(B, u, 6)
    for si in range(len(systems())):
        assert its[si * 6 + 2] == 0 and not us[si][2].any()
        assert min(its[si * 6 + j] for j in (0, 1, 3, 4, 5)) > 0
    s, its, rr, _ = B.pcg_solve(_stack(B, [p.b for p, _ in systems()]), torch.zeros_like(f),
                                rtol=1e-8, maxit=2, check=False)
    assert s == amg.AMG_ERR_NO_CONVERGENCE
    assert all(it == 2 for it in its[:6 * (len(systems()) - 1)])


def test_batch_rejects_bad_arguments():
    amg = _amg()
    ctxs, B = _batch(0)
    with pytest.raises(amg.AmgError):
        amg.Batch(ctxs, 4)  # nrhs must be 1 or 6
    empty = amg.Context(0)
    with pytest.raises(amg.AmgError) as e:
        amg.Batch([ctxs[0], empty], 6)
    assert e.value.code == amg.AMG_ERR_STATE
    other = amg.Context(0)
    p, H = systems()[0]
    other.upload_hierarchy(H.A[0], H.P, 1)
    with pytest.raises(amg.AmgError) as e:
        amg.Batch([ctxs[0], other], 6)
    assert e.value.code == amg.AMG_ERR_ARG


def test_batch_host_entry_point_matches_device():
    ctxs, B = _batch(1)
    f = _stack(B, [p.b for p, _ in systems()])
    u = torch.zeros_like(f)
    _, it1, r1, ms1 = B.pcg_solve(f, u, rtol=1e-8)
    fh = f.cpu().pin_memory()
    uh = torch.zeros_like(fh).pin_memory()
    _, it2, r2, ms2 = B.pcg_solve_host(fh, uh, rtol=1e-8)
    assert it1 == it2 and r1 == r2 and ms2 > 0
    assert torch.equal(u.cpu(), uh)


def test_batch_schedule_is_grouped_and_tuned():
    """One grouped launch per step for all systems: the launches per
    iteration do not grow with the number of systems, and every product
    stage carries the tile the autotuner chose."""
    amg = _amg()
    ctxs, B = _batch(1)
    per_it, fixed = B.launches()
    d = B.describe()
    prods = [ln for ln in d.splitlines() if "lanes/row" in ln or "SELL-32" in ln]
    assert prods and all(any(f"{l} lanes/row" in ln for l in (32, 16, 8)) or "SELL-32" in ln
                         for ln in prods)
    # the FP64 CG product of every system is one of the tuned stages
    assert any("q = A_0 p" in ln for ln in prods)
    assert len([ln for ln in d.splitlines() if ln.startswith("iteration")]) == per_it
    ctx1, B1 = ctxs[:2], amg.Batch(ctxs[:2], 6)
    assert B1.launches()[0] <= per_it <= 40
