"""Pins of the oracle on the paper's scalar problem (Problem gg, Sec. 2;
scalar model problem of Sec. 7): the edge / vertex weights of Sec. 4
(E^{ij} = |A_ij|, M^i = max{0, A_ii - sum |A_ij|}) split an M-matrix
exactly, the prolongations reproduce the constants (the kernel of the
scalar operator, k = 1), the coarse Neumann matrices annihilate them, and the
V-cycle is an SPD preconditioner whose PCG recovers a manufactured
solution."""
import numpy as np
import pytest

from oracle import hierarchy, solve, topology
from workloads.poisson import make_poisson


def _dense(M):
    return M.scipy().toarray()


def _scalar_params(**kw):
    base = dict(passes_first=4, passes_later=3, scalar_only=True, cap_S_first=4, cap_S_later=4)
    base.update(kw)
    return hierarchy.SetupParams(**base)


def test_weights_split_an_m_matrix_exactly():
    """On the plain grid the P1 Laplacian of the Kuhn / SW-NE splits is an
    M-matrix; then A-hat of eq. (auxa) equals the full matrix."""
    import scipy.sparse as sp
    for shape in ((7, 6), (5, 5, 4)):
        q = make_poisson(shape, seed=0, amp=0.0)
        Af = q.A_full
        A = sp.bsr_matrix((Af.vals, Af.colidx, Af.rowptr)).toarray()
        off = A - np.diag(np.diag(A))
        assert off.max() <= 1e-14 * np.abs(A).max()          # an M-matrix
        T = topology.finest_topology_scalar(q.coords, Af.rowptr, Af.colidx, Af.vals, q.dirichlet)
        Ahat = topology.aux_matrix_dense(T)
        assert np.abs(Ahat - A).max() <= 1e-13 * np.abs(A).max()


@pytest.mark.parametrize("shape", [(13, 11), (9, 8, 7)])
def test_prolongations_reproduce_constants_and_coarse_kernel(shape):
    p = make_poisson(shape, seed=2)
    H = hierarchy.setup(p, _scalar_params(coarse_max=4))
    assert H.n_levels >= 2
    for l, rec in enumerate(H.info["records"]):
        P = H.P[l]
        ok = ~rec["D"][rec["rowmap"]]
        one = _dense(P) @ np.ones(P.n_cols)
        assert np.abs(one[ok] - 1.0).max() <= 1e-12
        # tentative P: every non-D row is one 1 in its agglomerate's column
        rows = [r for r in rec["tentative"]]
        assert all(len(r) == (0 if rec["D"][v] else 1) for r, v in zip(rows, rec["rowmap"]))
    # Neumann version: coarse matrices annihilate the constants
    q = make_poisson(shape, seed=2)
    q.dirichlet[:] = False
    q.free = np.arange(q.n_all)
    q.A = q.A_full
    Hn = hierarchy.setup(q, _scalar_params(coarse_max=4), factor=False)
    scale = np.abs(_dense(Hn.A[0])).max()
    for Al in Hn.A[1:]:
        Ad = _dense(Al)
        assert np.abs(Ad @ np.ones(Ad.shape[0])).max() <= 1e-11 * scale


def test_scalar_vcycle_spd_two_grid_contracts_and_pcg_recovers_solution():
    p = make_poisson((10, 9, 8), seed=3)
    H = hierarchy.setup(p, _scalar_params(coarse_max=30, max_levels=2))
    n = H.A[0].n_rows
    rng = np.random.default_rng(4)
    x, y = rng.normal(size=(2, n))
    bx, by = solve.vcycle(H, x), solve.vcycle(H, y)
    assert abs(y @ bx - x @ by) <= 1e-11 * abs(x @ bx) and x @ bx > 0
    A = _dense(H.A[0])
    B = np.column_stack([solve.vcycle(H, e) for e in np.eye(n)])
    assert np.abs(np.linalg.eigvals(np.eye(n) - B @ A)).max() < 1.0
    u_star = rng.normal(size=n)
    u, it, _ = solve.pcg(H, A @ u_star, rtol=1e-12, maxit=500)
    e = u - u_star
    assert np.sqrt(e @ A @ e / (u_star @ A @ u_star)) <= 1e-9
