"""The block-l1 hybrid Gauss-Seidel smoother on the GPU
(AMG_SMOOTHER_HYBRID_GS) against the oracle's (oracle/solve.py: the same
greedy colouring, smoother blocks and sweeps) on the same hierarchies:
colourings identical, smoother blocks 1e-10, V-cycle 1e-10 element by
element, PCG iterations +-1 and iterates 1e-10; the FP32 / BF16-storage
V-cycles reach the FP64 residual with an energy error <= 1e-6 against the
oracle's tight solve."""
import numpy as np
import pytest

from oracle import hierarchy, solve
from workloads import configs, make_problem

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

CASES = {
    "square32": lambda: (configs.square32(), hierarchy.SetupParams()),
    "cube10": lambda: (make_problem((10, 10, 10), seed=2), hierarchy.SetupParams(coarse_max=8)),
    "box_jump": lambda: (make_problem((9, 7, 8), seed=3, jump_boxes=6, nu_range=(0.25, 0.45)),
                         hierarchy.SetupParams(coarse_max=6)),
    "jump11": lambda: (configs.jump11(12), hierarchy.SetupParams(coarse_max=8, passes_first=4,
                                                                  passes_later=3)),
    "poisson": lambda: (configs.poisson(14), hierarchy.SetupParams(coarse_max=12,
                                                                    **configs.SETUP["poisson"])),
}
_H = {}


def _amg():
    from paper_2011_13325_gb300 import amg
    return amg


def _case(name):
    if name not in _H:
        p, prm = CASES[name]()
        H = hierarchy.setup(p, prm)
        _H[name] = (p, solve.prepare(H.A[0], H.P, "hybrid_gs"))
    return _H[name]


def maxrel(a, b):
    a, b = np.asarray(a), np.asarray(b)
    assert a.shape == b.shape
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))


def dev(x):
    return torch.from_numpy(np.ascontiguousarray(x, dtype=np.float64)).cuda()


def _ctx(H, prec=0, layout=0):
    amg = _amg()
    ctx = amg.Context(0)
    ctx.set_layout_policy(layout)
    ctx.upload_hierarchy(H.A[0], H.P, prec, smoother=amg.AMG_SMOOTHER_HYBRID_GS)
    return ctx


@pytest.mark.parametrize("name", sorted(CASES))
def test_gs_setup_matches_oracle(name):
    p, H = _case(name)
    ctx = _ctx(H)
    for l in range(H.n_levels - 1):
        col, nc = ctx.smoother_colouring(l)
        np.testing.assert_array_equal(col, H.colour[l])
        assert nc == int(H.colour[l].max()) + 1
        m = ctx.download_smoother(l)
        assert np.abs(m - H.Minv[l]).max() <= 1e-10 * np.abs(H.Minv[l]).max(), l
    ctx.close()


@pytest.mark.parametrize("layout", [0, 1])
@pytest.mark.parametrize("name", sorted(CASES))
def test_gs_vcycle_and_pcg_match_oracle(name, layout):
    p, H = _case(name)
    ctx = _ctx(H, layout=layout)
    n = H.A[0].n_rows * H.A[0].br
    rng = np.random.default_rng(8)
    for r in (p.b[0], rng.normal(size=n)):
        z = dev(np.zeros(n))
        ctx.vcycle(dev(r), z)
        assert maxrel(z.cpu().numpy(), solve.vcycle(H, r)) <= 1e-10
    f = p.b[0]
    u = dev(np.zeros_like(f))
    _, its, rr = ctx.pcg_solve(dev(f), u, rtol=1e-8, maxit=500)
    u_or, it_or, _ = solve.pcg(H, f, rtol=1e-8)
    assert abs(its[0] - it_or) <= 1 and rr[0] <= 1e-8
    u_k = u_or if its[0] == it_or else solve.pcg(H, f, rtol=0.0, maxit=its[0])[0]
    assert maxrel(u.cpu().numpy(), u_k) <= 1e-10
    # the host-driven loop launches the same kernels
    ctx.set_pcg_graph(False)
    u2 = dev(np.zeros_like(f))
    _, its2, _ = ctx.pcg_solve(dev(f), u2, rtol=1e-8, maxit=500)
    assert its2 == its and torch.equal(u, u2)
    ctx.close()


@pytest.mark.parametrize("prec", [1, 2])
def test_gs_mixed_precision_reaches_fp64_tolerance(prec):
    p, H = _case("box_jump")
    ctx = _ctx(H, prec=prec, layout=1)
    f = p.b[0]
    u = dev(np.zeros_like(f))
    _, its, _ = ctx.pcg_solve(dev(f), u, rtol=1e-8, maxit=500)
    uh = u.cpu().numpy()
    A = H.A[0]
    assert np.linalg.norm(f - solve.spmv(A, uh)) <= 1.5e-8 * np.linalg.norm(f)
    ue, _, _ = solve.pcg(H, f, rtol=1e-13, maxit=1000)
    e = uh - ue
    assert np.sqrt(e @ solve.spmv(A, e) / (ue @ solve.spmv(A, ue))) <= 1e-6
    ctx.close()


def test_gs_vcycle_symmetric_positive_and_counted():
    p, H = _case("cube10")
    ctx = _ctx(H)
    n = H.A[0].n_rows * H.A[0].br
    rng = np.random.default_rng(9)
    x, y = rng.normal(size=(2, n))
    bx, by = dev(np.zeros(n)), dev(np.zeros(n))
    ctx.vcycle(dev(x), bx)
    ctx.vcycle(dev(y), by)
    bx, by = bx.cpu().numpy(), by.cpu().numpy()
    assert abs(y @ bx - x @ by) <= 1e-10 * abs(x @ bx)
    assert x @ bx > 0 and y @ by > 0
    per_it, fixed = ctx.pcg_launches()
    want = 1 + 6 + sum(3 + 2 * (int(c.max()) + 1) for c in H.colour)
    assert per_it == want
    prof = ctx.profile_vcycle(reps=2)
    assert len(prof) == 5 * (H.n_levels - 1) + 1 and all(us > 0 for _, _, us, _ in prof)
    ctx.close()


def test_gs_is_refused_where_it_is_not_built():
    amg = _amg()
    p, H = _case("cube10")
    ctx = _ctx(H)
    with pytest.raises(amg.AmgError) as e:
        ctx.vcycle_static(dev(p.b[0]), dev(np.zeros_like(p.b[0])))
    assert e.value.code == amg.AMG_ERR_ARG
    with pytest.raises(amg.AmgError) as e:
        ctx.set_learned_smoother(amg.Mlp(0, seed=1), p.coords[p.free])
    assert e.value.code == amg.AMG_ERR_STATE and "Gauss-Seidel" in str(e.value)
    with pytest.raises(amg.AmgError):
        amg.Batch([ctx], 6)
    # the context stays usable
    u = dev(np.zeros_like(p.b[0]))
    ctx.pcg_solve(dev(p.b[0]), u, rtol=1e-8)
    ctx.close()
