"""Pins of the oracle's auxiliary topology (Sec. 3-4) against facts the paper
and the mathematics fix, independent of the oracle's own formulas."""
import numpy as np
import pytest

from oracle import coarsening, topology as T
from workloads import make_problem


def _cross2(t, r):
    # 2D: rotation r about the z axis applied to t, i.e. e_z x t * r
    return np.array([-t[1] * r[0], t[0] * r[0]])


@pytest.mark.parametrize("d", [2, 3])
def test_skew_is_cross_product(d):
    rng = np.random.default_rng(0)
    for _ in range(5):
        t = rng.normal(size=d)
        r = rng.normal(size=T.kdim(d) - d)
        got = T.skew(t) @ r
        want = np.cross(t, r) if d == 3 else _cross2(t, r)
        np.testing.assert_allclose(got, want, rtol=0, atol=1e-15)


@pytest.mark.parametrize("d", [2, 3])
def test_rigid_mode_transfer(d):
    """u(y) = u(x) + Skew(y - x) r for u(x) = d + Skew(x) r (Sec. 3): the
    nodal coordinates (u(x_i), r) map to (u(x_j), r) by Q^{v_i -> v_j}."""
    rng = np.random.default_rng(1)
    k = T.kdim(d)
    dv = rng.normal(size=d)
    r = rng.normal(size=k - d)

    def u(x):  # rigid motion written with numpy's cross product
        return dv + (np.cross(x, r) if d == 3 else _cross2(x, r))

    xi, xj = rng.normal(size=d), rng.normal(size=d)
    vi = np.concatenate([u(xi), r])
    vj = np.concatenate([u(xj), r])
    np.testing.assert_allclose(T.Q_transfer(xi, xj) @ vi, vj, atol=1e-14)
    # Q^{ij} squared is Q^{v_i -> v_j}; transfers compose (Def. deng)
    np.testing.assert_allclose(T.Q_half(xi, xj) @ T.Q_half(xi, xj), T.Q_transfer(xi, xj), atol=1e-14)
    xl = rng.normal(size=d)
    np.testing.assert_allclose(T.Q_transfer(xj, xl) @ T.Q_transfer(xi, xj), T.Q_transfer(xi, xl),
                               atol=1e-14)


def test_coarse_transfer_closed_form():
    """Q^{IJ->ij} Q^{IJ} = Q^{ij} Q^{v_I->v_i} (proof of Thm. cemats); with
    Q^{IJ->ij} = Q^{ij} Q^{v_I->v_i} Q^{JI} it is the shift by
    (x_i + x_j)/2 - (x_I + x_J)/2."""
    rng = np.random.default_rng(2)
    xi, xj, xI, xJ = (rng.normal(size=3) for _ in range(4))
    qt = T.Q_half(xi, xj) @ T.Q_transfer(xI, xi) @ T.Q_half(xJ, xI)
    np.testing.assert_allclose(qt @ T.Q_half(xI, xJ), T.Q_half(xi, xj) @ T.Q_transfer(xI, xi),
                               atol=1e-14)
    shift = 0.5 * (xi + xj) - 0.5 * (xI + xJ)
    want = np.eye(6)
    want[:3, 3:] = np.array([[0, -shift[2], shift[1]], [shift[2], 0, -shift[0]],
                             [-shift[1], shift[0], 0]])
    np.testing.assert_allclose(qt, want, atol=1e-14)


def test_edge_form_equals_pair_matrix():
    """Proof of Thm. deng_elast: with E = c [[t t^T, 0],[0, 0]] the edge energy
    of (u_i, 0), (u_j, 0) is c (t . (u_i - u_j))^2."""
    rng = np.random.default_rng(3)
    xi, xj = rng.normal(size=3), rng.normal(size=3)
    t = xj - xi
    c = 0.7
    E = np.zeros((6, 6))
    E[:3, :3] = c * np.outer(t, t)
    F = T.edge_form(xi, xj, E)
    for _ in range(5):
        ui, uj = rng.normal(size=3), rng.normal(size=3)
        v = np.concatenate([ui, np.zeros(3), uj, np.zeros(3)])
        assert abs(v @ F @ v - c * (t @ (ui - uj)) ** 2) <= 1e-13 * (1 + abs(v @ F @ v))


def test_edge_form_rotations_drop_out():
    """t . (t x r) = 0: a finest-level edge matrix sees neither rotation dof."""
    rng = np.random.default_rng(4)
    xi, xj = rng.normal(size=3), rng.normal(size=3)
    t = xj - xi
    E = np.zeros((6, 6))
    E[:3, :3] = np.outer(t, t)
    F = T.edge_form(xi, xj, E)
    v = np.concatenate([np.zeros(3), rng.normal(size=3), np.zeros(3), rng.normal(size=3)])
    assert abs(v @ F @ v) < 1e-14


def _topo(shape, seed=5, clamp=True):
    p = make_problem(shape, seed=seed, clamp=clamp)
    return p, T.finest_topology(p.coords, p.A_full.rowptr, p.A_full.colidx, p.A_full.vals,
                                p.dirichlet)


@pytest.mark.parametrize("shape", [(5, 5), (4, 4, 3)])
def test_aux_matrix_annihilates_rigid_modes(shape):
    """Def. deng: every edge term vanishes on a rigid mode, on the finest level
    (rank-one edges) and on a coarse Neumann level (full-rank edges)."""
    _, topo = _topo(shape, clamp=False)
    agg, nc, xc, tc, D = coarsening.successive_matching(topo, coarsening.CoarsenParams(passes=1))
    for tp in (topo, tc):
        Ah = T.aux_matrix_dense(tp)
        W = T.rigid_modes(tp.pos, with_rotations=True)
        assert np.abs(Ah @ W).max() <= 1e-13 * np.abs(Ah).max()
        np.testing.assert_allclose(Ah, Ah.T, atol=1e-15 * np.abs(Ah).max())
        assert np.linalg.eigvalsh(Ah).min() >= -1e-13 * np.abs(Ah).max()


def test_finest_edge_weight_is_mean_abs_block():
    """Remark after Thm. deng_elast: c^{ij} = (1/d^2) sum |(A_ij)_lm|."""
    p, topo = _topo((4, 4))
    e = 3
    i, j = topo.edges[e]
    row = p.A_full.colidx[p.A_full.rowptr[i]:p.A_full.rowptr[i + 1]]
    blk = p.A_full.vals[p.A_full.rowptr[i] + np.nonzero(row == j)[0][0]]
    t = p.coords[j] - p.coords[i]
    c = np.abs(blk).mean()
    np.testing.assert_allclose(topo.E[e][:2, :2], c * np.outer(t, t), rtol=1e-14)
    assert np.all(topo.E[e][2:, :] == 0) and np.all(topo.M == 0)


@pytest.mark.parametrize("shape,clamp", [((7, 6), True), ((7, 6), False), ((4, 4, 4), True)])
def test_galerkin_of_aux_matrix_is_coarse_aux_matrix(shape, clamp):
    """Proof of Thm. cemats: P^T A-hat P = A-hat_c exactly, with edges inside an
    agglomerate cancelling and edges to D folded into M^I."""
    _, topo = _topo(shape, clamp=clamp)
    for passes in (1, 2):
        agg, nc, xc, tc, D = coarsening.successive_matching(
            topo, coarsening.CoarsenParams(passes=passes))
        k = topo.k
        P = np.zeros((topo.n * k, nc * k))
        for i in range(topo.n):
            if agg[i] >= 0:
                P[i * k:(i + 1) * k, agg[i] * k:(agg[i] + 1) * k] = T.Q_transfer(xc[agg[i]], topo.pos[i])
        Ah = T.aux_matrix_dense(topo)
        Ac = T.aux_matrix_dense(tc)
        assert np.abs(P.T @ Ah @ P - Ac).max() <= 1e-12 * np.abs(Ac).max()
        if clamp:
            assert np.abs(tc.M).max() > 0  # Dirichlet edges became vertex matrices
        else:
            assert np.abs(tc.M).max() == 0


@pytest.mark.parametrize("shape,kw", [((13, 11), {"coarse_max": 3}), ((7, 6, 5), {"coarse_max": 4}),
                                      ((9, 7, 8), {"coarse_max": 6})])
def test_coarse_topology_in_one_step_equals_pass_by_pass(shape, kw):
    """Kernel transfers compose (Q(a) Q(b) = Q(a + b)), so Thm. cemats applied
    once from a level's topology to the final agglomerates of Algorithm 1
    gives the coarse topology Algorithm 1 built pass by pass (edges exact,
    matrices to rounding)."""
    from oracle import hierarchy
    p = make_problem(shape, seed=3, jump_boxes=4 if len(shape) == 3 else 0)
    H = hierarchy.setup(p, hierarchy.SetupParams(**kw), factor=False)
    recs = H.info["records"]
    assert len(recs) >= 2
    for l in range(len(recs) - 1):
        rec, seq = recs[l], recs[l + 1]["topo"]
        one = T.coarse_topology(rec["topo"], rec["agg"], rec["xc"].shape[0], rec["xc"])
        np.testing.assert_array_equal(one.edges, seq.edges)
        assert np.abs(one.E - seq.E).max() <= 1e-12 * np.abs(seq.E).max()
        assert np.abs(one.M - seq.M).max() <= 1e-12 * max(np.abs(seq.M).max(), 1e-300)
