"""The library's own setup (amg_setup: host Algorithm 1 + auxiliary smoothed
prolongation, device Galerkin) against the oracle's setup on the same
seeded problems: same levels, same prolongation patterns, values to 1e-10,
same PCG iteration counts."""
import numpy as np
import pytest

from oracle import hierarchy, solve
from workloads import configs, make_problem

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

CASES = {
    "square32": (lambda: configs.square32(), {}),
    "cube10": (lambda: make_problem((10, 10, 10), seed=2), {"coarse_max": 8}),
    "box_jump": (lambda: make_problem((9, 7, 8), seed=3, jump_boxes=6, nu_range=(0.25, 0.45)),
                 {"coarse_max": 6}),
}


@pytest.mark.parametrize("name", sorted(CASES))
def test_library_setup_matches_oracle_setup(name):
    from paper_2011_13325_gb300 import amg
    make, kw = CASES[name]
    p = make()
    H = hierarchy.setup(p, hierarchy.SetupParams(**kw))
    ctx = amg.Context(0)
    ctx.setup(p, amg.AMG_PREC_FP64, **kw)
    assert ctx.n_levels == H.n_levels
    for l, P in enumerate(H.P):
        n, m, rp, ci, v = ctx.download_prolongation(l)
        assert (n, m) == (P.n_rows, P.n_cols), l
        np.testing.assert_array_equal(rp, P.rowptr)
        np.testing.assert_array_equal(ci, P.colidx)
        assert np.abs(v - P.vals).max() <= 1e-10 * np.abs(P.vals).max(), l
    f = p.b[0]
    u = torch.zeros(f.shape[0], dtype=torch.float64, device="cuda")
    _, its, rr = ctx.pcg_solve(torch.from_numpy(f).cuda(), u, rtol=1e-8)
    _, it_or, _ = solve.pcg(H, f, rtol=1e-8)
    assert abs(its[0] - it_or) <= 1
    ctx.close()


def test_setup_rejects_bad_problem():
    from paper_2011_13325_gb300 import amg
    p = configs.square32()
    p.A_full.colidx[3] = p.A_full.n_cols + 1
    ctx = amg.Context(0)
    with pytest.raises(amg.AmgError) as e:
        ctx.setup(p)
    assert e.value.code == amg.AMG_ERR_ARG
    ctx.close()
