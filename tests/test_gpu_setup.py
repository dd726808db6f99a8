"""The library's own setup (amg_setup: Algorithm 1 on the host; the coarse
edge / vertex matrices of Thm. cemats and the auxiliary smoothed
prolongation of Def. aux_sp on the device, or on the host with
device_setup=0; device Galerkin products) against the oracle's setup on the
same seeded problems: same levels, same prolongation patterns, values to
1e-10, same PCG iteration counts; the device-built coarse topologies against
the oracle's (edges exact, edge / vertex matrices 1e-12)."""
import numpy as np
import pytest

from oracle import hierarchy, solve, topology
from workloads import configs, make_problem

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

CASES = {
    "square32": (lambda: configs.square32(), {}),
    "cube10": (lambda: make_problem((10, 10, 10), seed=2), {"coarse_max": 8}),
    "box_jump": (lambda: make_problem((9, 7, 8), seed=3, jump_boxes=6, nu_range=(0.25, 0.45)),
                 {"coarse_max": 6}),
    "beam": (lambda: configs.beam(4), {"coarse_max": 8}),
    "jump11": (lambda: configs.jump11(12), {"coarse_max": 8, "passes_first": 4, "passes_later": 3}),
    "poisson": (lambda: configs.poisson(14), dict(configs.SETUP["poisson"], coarse_max=12)),
}
_OR = {}


def _oracle(name):
    if name not in _OR:
        make, kw = CASES[name]
        p = make()
        _OR[name] = (p, kw, hierarchy.setup(p, hierarchy.SetupParams(**kw)))
    return _OR[name]


@pytest.mark.parametrize("device_setup", [1, 0])
@pytest.mark.parametrize("name", sorted(CASES))
def test_library_setup_matches_oracle_setup(name, device_setup):
    from paper_2011_13325_gb300 import amg
    p, kw, H = _oracle(name)
    ctx = amg.Context(0)
    # device_setup = 1 with every device stage, mu_p included
    ctx.setup(p, amg.AMG_PREC_FP64, device_setup=device_setup, device_pair_measure=device_setup, **kw)
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


@pytest.mark.parametrize("name", sorted(CASES))
def test_device_coarse_topology_matches_oracle(name):
    """Thm. cemats on the device (one direct transfer from the level's
    topology to the final agglomerates) against the oracle's coarse_topology
    on the same agglomerates, and against the topology the oracle's own
    Algorithm 1 built pass by pass (the Q transfers compose)."""
    from paper_2011_13325_gb300 import amg
    p, kw, H = _oracle(name)
    if p.k == 1:
        pytest.skip("the scalar problem builds its coarse topology on the host")
    ctx = amg.Context(0)
    ctx.setup(p, amg.AMG_PREC_FP64, keep_topology=1, **kw)
    recs = H.info["records"]
    for l, rec in enumerate(recs):
        pos, edges, E, M = ctx.download_topology(l + 1)
        want = topology.coarse_topology(rec["topo"], rec["agg"], rec["xc"].shape[0], rec["xc"])
        np.testing.assert_array_equal(edges, want.edges)
        assert np.abs(pos - want.pos).max() <= 1e-14 * max(1.0, np.abs(want.pos).max())
        assert np.abs(E - want.E).max() <= 1e-12 * np.abs(want.E).max(), l
        if np.abs(want.M).max() > 0:
            assert np.abs(M - want.M).max() <= 1e-12 * np.abs(want.M).max(), l
        else:
            assert not M.any()
        if l + 1 < len(recs):
            seq = recs[l + 1]["topo"]
            np.testing.assert_array_equal(edges, seq.edges)
            assert np.abs(E - seq.E).max() <= 1e-12 * np.abs(seq.E).max(), l
    with pytest.raises(amg.AmgError):
        ctx.download_topology(len(recs) + 1)
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


def test_device_pair_measure_gives_the_host_hierarchy():
    """Algorithm 1 with mu_p evaluated on the device (batches of candidate
    pairs) takes the decisions of the host evaluation: on a 3D jump problem
    large enough for many device batches, the setups with mu_p on the device,
    with mu_p on the host (other device stages on), and all on the host give
    prolongations with identical patterns and values to 1e-12; only the
    first reports device time for mu_p."""
    from paper_2011_13325_gb300 import amg
    p = make_problem((20, 19, 18), seed=9, jump_boxes=30, nu_range=(0.25, 0.45))
    out = []
    for dev, dpm in ((1, 1), (1, 0), (0, 1)):
        ctx = amg.Context(0)
        ctx.setup(p, amg.AMG_PREC_FP64, device_setup=dev, device_pair_measure=dpm)
        out.append(([ctx.download_prolongation(l) for l in range(ctx.n_levels - 1)], ctx.setup_times()))
        ctx.close()
    (Pd, td), (Pm, tm), (Ph, th) = out
    assert td["device_pair_measure_s"] > 0.0
    assert tm["device_pair_measure_s"] == 0.0 and th["device_pair_measure_s"] == 0.0
    for Px in (Pd, Pm):
        assert len(Px) == len(Ph)
        for (n, m, rp, ci, v), (n2, m2, rp2, ci2, v2) in zip(Px, Ph):
            assert (n, m) == (n2, m2)
            np.testing.assert_array_equal(rp, rp2)
            np.testing.assert_array_equal(ci, ci2)
            assert np.abs(v - v2).max() <= 1e-12 * np.abs(v2).max()
