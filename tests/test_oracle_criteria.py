"""Pins of the coarsening measures (Sec. 5): harmonic-mean identities, the
generalised eigenproblem, mu_p = mu_g for pairs, mu_g's left side as a
least-squares infimum, and Algorithm 1's output invariants."""
import numpy as np
import pytest
import scipy.linalg as sla

from oracle import coarsening, criteria as C, topology as T
from workloads import make_problem


def _psd(rng, n, rank=None):
    rank = n if rank is None else rank
    G = rng.normal(size=(n, rank))
    return G @ G.T


def test_harmonic_pinv_identity():
    """eq. (harm_pinv): A(A+B)^+B(A+B)^+A + B(A+B)^+A(A+B)^+B = A(A+B)^+B."""
    rng = np.random.default_rng(0)
    for rank_a, rank_b in [(6, 6), (2, 3), (1, 1), (4, 2)]:
        A, B = _psd(rng, 6, rank_a), _psd(rng, 6, rank_b)
        S = C.pinv_sym(A + B)
        lhs = A @ S @ B @ S @ A + B @ S @ A @ S @ B
        np.testing.assert_allclose(lhs, A @ S @ B, rtol=0, atol=1e-12 * (np.abs(A).max() + np.abs(B).max()))


def test_harmonic_is_parallel_sum():
    """x^T H(A,B) x = inf_y ||y||_A^2 + ||x-y||_B^2 (textbook parallel sum)."""
    rng = np.random.default_rng(1)
    A, B = _psd(rng, 5), _psd(rng, 5)
    x = rng.normal(size=5)
    y = np.linalg.solve(A + B, B @ x)
    brute = y @ A @ y + (x - y) @ B @ (x - y)
    assert abs(x @ C.harmonic(A, B) @ x - brute) < 1e-10 * abs(brute)
    # two rank-one matrices with different directions: series sum is zero
    a, b = rng.normal(size=5), rng.normal(size=5)
    assert np.abs(C.harmonic(np.outer(a, a), np.outer(b, b))).max() < 1e-12


def test_gen_lambda_max_against_scipy():
    rng = np.random.default_rng(2)
    L, R = _psd(rng, 6), _psd(rng, 6)
    assert abs(C.gen_lambda_max(L, R) - sla.eigh(L, R, eigvals_only=True).max()) < 1e-9
    # singular right side: restricted to its range; energy on ker(R) -> inf
    v = rng.normal(size=(6, 3))
    R3 = v @ v.T
    Pr = v @ np.linalg.pinv(v)
    L_in = Pr @ _psd(rng, 6) @ Pr
    w = sla.eigh(v.T @ L_in @ v, v.T @ R3 @ v, eigvals_only=True).max()
    assert abs(C.gen_lambda_max(L_in, R3) - w) < 1e-8 * w
    assert C.gen_lambda_max(_psd(rng, 6), R3) == np.inf


def _topo(shape, seed=3, clamp=True):
    p = make_problem(shape, seed=seed, clamp=clamp)
    return T.finest_topology(p.coords, p.A_full.rowptr, p.A_full.colidx, p.A_full.vals, p.dirichlet)


@pytest.mark.parametrize("shape", [(6, 5), (4, 4, 4)])
def test_mu_p_equals_mu_g_for_pairs_without_vertex_weights(shape):
    """Remark after Lemma mu2: mu_p = mu_g({v_i, v_j}) when M^i = M^j = 0."""
    topo = _topo(shape)
    nb, Dh = topo.adjacency(), T.aux_diagonal(topo)
    n_checked = 0
    for i, j in topo.edges:
        if topo.dirichlet[i] or topo.dirichlet[j]:
            continue
        mp = C.mu_p(topo, Dh, nb, i, j)
        mg = C.mu_g(topo, Dh, nb, [i, j])
        if np.isfinite(mg):
            assert abs(mp - mg) <= 1e-8 * mg
            n_checked += 1
        else:
            assert not np.isfinite(mp)
        if n_checked >= 12:
            break
    assert n_checked >= 6


def test_mu_p_bounds_mu_g_with_vertex_weights():
    """Lemma mu2: mu_g({v_i, v_j}) <= mu_p(v_i, v_j) (coarse level with M != 0)."""
    topo = _topo((8, 7))
    agg, nc, xc, tc, D = coarsening.successive_matching(topo, coarsening.CoarsenParams(passes=1))
    nb, Dh = tc.adjacency(), T.aux_diagonal(tc)
    checked = 0
    for i, j in tc.edges:
        if np.trace(tc.M[i]) + np.trace(tc.M[j]) == 0:
            continue
        mp = C.mu_p(tc, Dh, nb, i, j)
        mg = C.mu_g(tc, Dh, nb, [i, j])
        assert mg <= mp * (1 + 1e-8) or not np.isfinite(mp)
        checked += 1
    assert checked > 0


def test_mu_g_left_side_is_least_squares_infimum():
    """Left side of eq. (mu_a): inf_w ||v_C - P_C w||^2_{D_C} by brute force."""
    topo = _topo((6, 6))
    nb, Dh = topo.adjacency(), T.aux_diagonal(topo)
    Cset = [7, 8, 13, 14]
    left, right = C.mu_g_matrices(topo, Dh, nb, Cset)
    k = topo.k
    xH = topo.pos[Cset].mean(axis=0)
    PC = np.vstack([T.Q_transfer(xH, topo.pos[v]) for v in Cset])
    DC = sla.block_diag(*[Dh[v] for v in Cset])
    rng = np.random.default_rng(4)
    for _ in range(4):
        v = rng.normal(size=len(Cset) * k)
        # minimise (v - P w)^T D (v - P w) over w by least squares on D^(1/2)
        w_, V = np.linalg.eigh(DC)
        Dh2 = V @ np.diag(np.sqrt(np.clip(w_, 0, None))) @ V.T
        wopt = np.linalg.lstsq(Dh2 @ PC, Dh2 @ v, rcond=None)[0]
        brute = (v - PC @ wopt) @ DC @ (v - PC @ wopt)
        assert abs(v @ left @ v - brute) <= 1e-10 * max(1.0, abs(brute))
    # the right side is PSD and the agglomerate's rigid modes have zero energy
    Wc = np.vstack([T.Q_transfer(xH, topo.pos[v]) for v in Cset])
    assert np.abs(right @ Wc).max() < 1e-12 * np.abs(right).max()


@pytest.mark.parametrize("shape,passes", [((9, 9), 3), ((5, 5, 4), 2)])
def test_algorithm1_invariants(shape, passes):
    """Algorithm 1 output: a partition of V \\ D whose agglomerates all satisfy
    mu_g(C) < sigma (Thm. mu1), with D containing the Dirichlet vertices."""
    topo = _topo(shape)
    p = coarsening.CoarsenParams(passes=passes)
    agg, nc, xc, tc, D = coarsening.successive_matching(topo, p)
    assert np.all(D[topo.dirichlet])
    assert np.all((agg >= 0) == ~D)
    assert set(np.unique(agg[agg >= 0])) == set(range(nc))
    assert nc < (~D).sum()
    sizes = np.bincount(agg[agg >= 0])
    assert sizes.max() <= 2 ** passes
    nb, Dh = topo.adjacency(), T.aux_diagonal(topo)
    for I in range(nc):
        members = np.nonzero(agg == I)[0]
        if members.size >= 2:
            assert C.mu_g(topo, Dh, nb, members) < p.sigma
        np.testing.assert_allclose(xc[I], topo.pos[members].mean(axis=0), atol=1e-15)


def test_cuthill_mckee_is_permutation_of_active():
    topo = _topo((6, 6))
    order = coarsening.cuthill_mckee(topo, ~topo.dirichlet)
    assert sorted(order) == sorted(np.nonzero(~topo.dirichlet)[0].tolist())


def test_mu_p_equals_mu_g_on_coarse_neumann_level():
    """Remark after Lemma mu2 on a coarse level (full-rank edge matrices, M = 0):
    exercises the delta-term of eq. (mub_ineq), which vanishes on the finest level."""
    topo = _topo((9, 8), clamp=False)
    agg, nc, xc, tc, D = coarsening.successive_matching(topo, coarsening.CoarsenParams(passes=1))
    assert np.abs(tc.M).max() == 0
    nb, Dh = tc.adjacency(), T.aux_diagonal(tc)
    checked = 0
    for i, j in tc.edges[:15]:
        common = set(nb[i]) & set(nb[j])
        if not common:
            continue
        mp = C.mu_p(tc, Dh, nb, i, j)
        mg = C.mu_g(tc, Dh, nb, [i, j])
        if not np.isfinite(mg):
            assert not np.isfinite(mp)
            continue
        assert np.isfinite(mp) and abs(mp - mg) <= 1e-7 * mg
        checked += 1
    assert checked >= 5


def test_robust_criteria_keep_two_grid_conditioned_across_jumps():
    """Sec. 5, the coefficient-jump figures: on 2D elasticity with stiff
    (10^4) and soft (1) boxes and a clamped left side, Algorithm 1 with the
    robust measures mu_p, mu_g gives a well-conditioned two-grid method,
    while the scalar measure mu_s alone merges across the jumps and the
    condition number grows by orders of magnitude (the paper reports about
    2.84 against about 270 on its own mesh).  Here: a 4 x 4 checkerboard of
    boxes on a 17 x 17 mesh, one coarsening step, the block-l1 Jacobi
    two-grid preconditioner, kappa from a dense eigen-solve."""
    from oracle import hierarchy, solve
    from workloads import make_problem

    def checker(c, nb=4):
        i = np.floor(c[:, 0] * nb).clip(0, nb - 1)
        j = np.floor(c[:, 1] * nb).clip(0, nb - 1)
        return np.where((i + j) % 2 == 1, 1e4, 1.0)

    p = make_problem((17, 17), seed=1, nu=0.25, E_fn=checker)
    kappas = []
    for scalar_only in (False, True):
        H = hierarchy.setup(p, hierarchy.SetupParams(max_levels=2, coarse_max=1,
                                                     scalar_only=scalar_only))
        assert H.n_levels == 2
        n = H.A[0].n_rows * H.A[0].br
        V = np.column_stack([solve.vcycle(H, e) for e in np.eye(n)])
        A = np.column_stack([solve.spmv(H.A[0], e) for e in np.eye(n)])
        ev = np.linalg.eigvals(V @ A).real
        assert ev.min() > 0
        kappas.append(ev.max() / ev.min())
    robust, scalar = kappas
    assert robust < 30.0
    assert scalar > 50.0 * robust


def _hand_topology(pos, edges, weights):
    """A topology written out by hand: edge matrices w_e I_k, no vertex
    weights (so mu_D = +inf and no vertex joins D)."""
    pos = np.asarray(pos, dtype=np.float64)
    k = T.kdim(pos.shape[1])
    E = np.array([w * np.eye(k) for w in weights])
    return T.Topology(pos=pos, edges=np.asarray(edges, dtype=np.int64), E=E,
                      M=np.zeros((pos.shape[0], k, k)), dirichlet=np.zeros(pos.shape[0], bool))


def _groups(agg):
    return sorted(sorted(np.nonzero(agg == g)[0].tolist()) for g in set(agg.tolist()))


def test_algorithm1_tries_the_candidate_of_minimal_mu_s_first():
    """Algorithm 1 (Sec. 5.2), candidate choice, derived by hand on a 4-cycle
    0-1-2-3-0 with edge traces 3 w (k = 3) for w01 = 1, w12 = w23 = w30 = 2;
    sigma = 1e6 lets every mu_p / mu_g test pass, so only the choice and the
    order decide.  Every vertex has degree 2: the Cuthill-McKee order starts
    at vertex 0 (lowest id), then its neighbours by (degree, id): 1, 3, then 2.
    The trace maxima are max over incident edges: 6 at every vertex, so
    mu_s(0,1) = sqrt(6*6)/3 = 2 and mu_s(0,3) = sqrt(6*6)/6 = 1.  The minimal
    mu_s pairs 0 with 3; vertex 1 is visited next and its only unmatched
    neighbour is 2: agglomerates {0,3}, {1,2}.  Choosing the maximal mu_s
    would give {0,1}, {2,3}."""
    t = _hand_topology([(0, 0), (1, 0), (1, 1), (0, 1)], [(0, 1), (1, 2), (2, 3), (0, 3)],
                       [1.0, 2.0, 2.0, 2.0])
    tmax = C.trace_max(t, t.adjacency())
    assert np.allclose(tmax, 6.0)
    assert C.mu_s(tmax, 3.0, 0, 1) == 2.0 and C.mu_s(tmax, 6.0, 0, 3) == 1.0
    agg, nc, _, _, D = coarsening.successive_matching(t, coarsening.CoarsenParams(sigma=1e6,
                                                                                    passes=1))
    assert not D.any() and nc == 2
    assert _groups(agg) == [[0, 3], [1, 2]]


def test_algorithm1_later_pass_visits_in_reverse_insertion_order():
    """Algorithm 1 (Sec. 5.2), pass order, derived by hand on a zig-zag path
    0-1-2-3-4-5 with equal edges (E = I), sigma = 1e6.  Pass 1 (Cuthill-McKee
    from vertex 0, the lowest-id vertex of degree 1: 0,1,...,5) forms {0,1},
    {2,3}, {4,5} in that order.  Pass 2 visits them in reverse insertion
    order: {4,5} first, whose only neighbour is {2,3}, giving {2,3,4,5};
    {0,1} is then left alone.  Visiting in insertion order would give
    {0,1,2,3} and {4,5}.  Pairs are numbered before singletons, so the
    merged agglomerate is coarse vertex 0."""
    pos = [(i, 0.3 * (i % 2)) for i in range(6)]
    t = _hand_topology(pos, [(i, i + 1) for i in range(5)], [1.0] * 5)
    agg1, nc1, _, _, _ = coarsening.successive_matching(t, coarsening.CoarsenParams(sigma=1e6,
                                                                                      passes=1))
    assert agg1.tolist() == [0, 0, 1, 1, 2, 2]
    agg2, nc2, _, _, _ = coarsening.successive_matching(t, coarsening.CoarsenParams(sigma=1e6,
                                                                                      passes=2))
    assert agg2.tolist() == [1, 1, 0, 0, 0, 0]
