"""Pins of the oracle's solve phase: Galerkin product, explicit transpose,
block-l1 smoother, coarsest regularisation (Sec. 3 after Lemma eet_is_diag), two-grid convergence
(Sec. 3, Algorithm tg), V-cycle symmetry and PCG on manufactured solutions."""
import numpy as np
import pytest

from oracle import hierarchy, solve
from workloads import make_problem


@pytest.fixture(scope="module")
def h2d():
    p = make_problem((11, 10), seed=21)
    H = hierarchy.setup(p, hierarchy.SetupParams(coarse_max=6, passes_first=2, passes_later=2))
    return p, H


@pytest.fixture(scope="module")
def h3d():
    p = make_problem((5, 5, 6), seed=22)
    H = hierarchy.setup(p, hierarchy.SetupParams(coarse_max=6, passes_first=2, passes_later=2))
    return p, H


def _dense(M):
    return M.scipy().toarray()


@pytest.mark.parametrize("which", ["h2d", "h3d"])
def test_galerkin_pattern_and_values_brute_force(which, request):
    p, H = request.getfixturevalue(which)
    assert H.n_levels >= 3
    for lev, P in enumerate(H.P):
        A = H.A[lev]
        C = H.A[lev + 1]
        # values: dense triple product
        np.testing.assert_allclose(_dense(C), _dense(P).T @ _dense(A) @ _dense(P),
                                   rtol=0, atol=1e-13 * np.abs(_dense(C)).max())
        # pattern: every coarse block pair (I, J) reached by P_iI A_ij P_jJ
        Prow = [set(P.colidx[P.rowptr[i]:P.rowptr[i + 1]]) for i in range(P.n_rows)]
        want = set()
        for i in range(A.n_rows):
            for j in A.colidx[A.rowptr[i]:A.rowptr[i + 1]]:
                for I in Prow[i]:
                    for J in Prow[j]:
                        want.add((int(I), int(J)))
        got = {(int(I), int(J)) for I in range(C.n_rows)
               for J in C.colidx[C.rowptr[I]:C.rowptr[I + 1]]}
        assert got == want
        for I in range(C.n_rows):
            cols = C.colidx[C.rowptr[I]:C.rowptr[I + 1]]
            assert np.all(np.diff(cols) > 0)


def test_explicit_transpose(h3d):
    _, H = h3d
    for P, R in zip(H.P, H.R):
        np.testing.assert_array_equal(_dense(R), _dense(P).T)


@pytest.mark.parametrize("which", ["h2d", "h3d"])
def test_block_l1_smoother_dominates_A(which, request):
    """l1 property (Sec. 7, smoother of [UPSM]): blockdiag(M_v) - A is PSD, so
    the block Jacobi sweep is convergent in the energy norm."""
    _, H = request.getfixturevalue(which)
    for lev in range(H.n_levels - 1):
        A = H.A[lev]
        Ad = _dense(A)
        k = A.br
        Md = np.zeros_like(Ad)
        for i in range(A.n_rows):
            blk = Ad[i * k:(i + 1) * k, i * k:(i + 1) * k].copy()
            off = np.abs(Ad[i * k:(i + 1) * k, :]).sum(axis=1) - np.abs(blk).sum(axis=1)
            Md[i * k:(i + 1) * k, i * k:(i + 1) * k] = blk + np.diag(off)
        assert np.linalg.eigvalsh(Md - Ad).min() >= -1e-12 * np.abs(Ad).max()
        # the stored blocks are the (pseudo-)inverses of these M_v
        Minv = solve.block_diag_dense(H.Minv[lev])
        Pr = Minv @ Md
        np.testing.assert_allclose(Pr @ Pr, Pr, atol=1e-9)
        np.testing.assert_allclose(Md @ Minv @ Md, Md, atol=1e-9 * np.abs(Md).max())
        # error propagation of the sweep contracts the A-norm
        E = np.eye(Ad.shape[0]) - Minv @ Ad
        w = np.linalg.eigvals(E)
        assert np.abs(w).max() <= 1 + 1e-10


def test_coarsest_regularisation_identity(h3d):
    """Sec. 3 after Lemma eet_is_diag: (E A~ E^T + (I - E E^T))^{-1} = E A~^{-1} E^T + (I - E E^T)
    with A~ = E^T A_L E and E spanning the complement of the block kernels."""
    _, H = h3d
    A = H.A[-1]
    k = A.br
    n = A.n_rows * k
    Kb = solve.diag_kernels(A)
    K = np.zeros((n, sum(b.shape[1] for b in Kb)))
    c = 0
    for i, b in enumerate(Kb):
        K[i * k:(i + 1) * k, c:c + b.shape[1]] = b
        c += b.shape[1]
    Pk = K @ K.T
    w, V = np.linalg.eigh(np.eye(n) - Pk)
    E = V[:, w > 0.5]
    At = E.T @ _dense(A) @ E
    lhs = np.linalg.inv(solve.coarsest_matrix(A))
    rhs = E @ np.linalg.inv(At) @ E.T + Pk
    np.testing.assert_allclose(lhs, rhs, atol=1e-8 * np.abs(rhs).max())


@pytest.mark.parametrize("which", ["h2d", "h3d"])
def test_two_grid_spectral_radius(which, request):
    """Sec. 3: rho(E_TG) < 1; power iteration agrees with a dense eigen-solve."""
    _, H = request.getfixturevalue(which)
    A = _dense(H.A[0])
    Minv = solve.block_diag_dense(H.Minv[0])
    P = _dense(H.P[0])
    Acp = np.linalg.pinv(P.T @ A @ P, rcond=1e-12, hermitian=True)
    E = solve.two_grid_matrix(A, Minv, P)
    rho_dense = np.abs(np.linalg.eigvals(E)).max()
    rho_pow = solve.spectral_radius_power(lambda x: solve.two_grid_apply(A, Minv, P, Acp, x),
                                          A.shape[0], iters=2000)
    assert rho_dense < 1.0
    assert abs(rho_pow - rho_dense) <= 1e-8


def test_two_level_vcycle_is_two_grid_formula(h2d):
    """A 2-level V-cycle equals B_TG^{-1} = M~^{-1} + (I - M^{-T}A) P A_c^+ P^T (I - A M^{-1})
    with M~^{-1} = M^{-T}(M + M^T - A)M^{-1} (Sec. 3)."""
    p, H = h2d
    H2 = solve.prepare(H.A[0], H.P[:1])
    A = _dense(H2.A[0])
    Minv = solve.block_diag_dense(H2.Minv[0])
    M = np.linalg.pinv(Minv)
    P = _dense(H2.P[0])
    n = A.shape[0]
    I = np.eye(n)
    Acp = np.linalg.pinv(P.T @ A @ P, rcond=1e-12, hermitian=True)
    Binv = Minv.T @ (M + M.T - A) @ Minv + (I - Minv.T @ A) @ P @ Acp @ P.T @ (I - A @ Minv)
    V = np.column_stack([solve.vcycle(H2, e) for e in I])
    np.testing.assert_allclose(V, Binv, atol=1e-9 * np.abs(Binv).max())


@pytest.mark.parametrize("which", ["h2d", "h3d"])
def test_vcycle_is_spd(which, request):
    _, H = request.getfixturevalue(which)
    n = H.A[0].n_rows * H.A[0].br
    V = np.column_stack([solve.vcycle(H, e) for e in np.eye(n)])
    np.testing.assert_allclose(V, V.T, atol=1e-12 * np.abs(V).max())
    assert np.linalg.eigvalsh(0.5 * (V + V.T)).min() > 0
    A = _dense(H.A[0])
    assert np.abs(np.linalg.eigvals(np.eye(n) - V @ A)).max() < 1.0


@pytest.mark.parametrize("which", ["h2d", "h3d"])
def test_pcg_recovers_manufactured_solution(which, request):
    p, H = request.getfixturevalue(which)
    A = H.A[0]
    rng = np.random.default_rng(5)
    x = p.coords[p.free]
    smooth = np.stack([np.sin(3 * x[:, 0]) * np.cos(2 * x[:, 1]) for _ in range(p.dim)], axis=1)
    for ustar in (rng.normal(size=A.n_rows * A.br), smooth.ravel()):
        f = solve.spmv(A, ustar)
        u, it, hist = solve.pcg(H, f, rtol=1e-12, maxit=500)
        e = u - ustar
        err = np.sqrt(e @ solve.spmv(A, e)) / np.sqrt(ustar @ solve.spmv(A, ustar))
        assert err <= 1e-7
        assert hist[-1] <= 1e-12


def test_pcg_degenerate_right_sides(h2d):
    """f = 0 from x0 = 0: the stopping rule ||r|| <= rtol ||f|| holds at once
    (0 iterations, x = 0).  A start at the solution of a manufactured
    problem needs no iteration either, and a start on one side of the
    solution converges to it."""
    p, H = h2d
    A = H.A[0]
    n = A.n_rows * A.br
    x, it, hist = solve.pcg(H, np.zeros(n), rtol=1e-8)
    assert it == 0 and not x.any() and hist == [0.0]
    ustar = np.random.default_rng(7).normal(size=n)
    f = solve.spmv(A, ustar)
    u, it, hist = solve.pcg(H, f, rtol=1e-8, x0=ustar)
    assert it == 0 and hist[0] <= 1e-12
    u, it, hist = solve.pcg(H, f, rtol=1e-10, x0=ustar + 1e-3)
    assert 0 < it < 60 and np.abs(u - ustar).max() <= 1e-6


def test_one_level_hierarchy_is_an_exact_solve():
    """A problem at or below the coarse size keeps one level: the V-cycle is
    the regularised coarsest solve, which for an SPD A_0 (no kernel to
    regularise) is A_0^{-1}, so PCG stops after one iteration."""
    p = make_problem((4, 3), seed=1)
    H = hierarchy.setup(p)
    assert H.n_levels == 1
    n = H.A[0].n_rows * H.A[0].br
    V = np.column_stack([solve.vcycle(H, e) for e in np.eye(n)])
    A = _dense(H.A[0])
    np.testing.assert_allclose(V @ A, np.eye(n), atol=1e-12)
    _, it, hist = solve.pcg(H, p.b[0], rtol=1e-12)
    assert it == 1 and hist[-1] <= 1e-12


def test_galerkin_many_coarse_rows_keeps_block_keys():
    """P = I on 50,000 block rows (nc^2 > 2^31): P^T A P must return A itself
    (the block keys of the scatter need 64-bit arithmetic)."""
    n, k = 50_000, 3
    rng = np.random.default_rng(0)
    rp = np.arange(n + 1, dtype=np.int64)
    ci = np.arange(n, dtype=np.int64)
    eye = np.tile(np.eye(k), (n, 1, 1))
    P = solve.Mat(n, n, rp, ci, eye)
    # A: diagonal blocks plus a coupling of row i to row n-1-i
    rows, cols = [], []
    for i in range(n):
        j = n - 1 - i
        rows += [i] * (1 if i == j else 2)
        cols += sorted({i, j})
    rows, cols = np.array(rows), np.array(cols)
    Arp = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(np.bincount(rows, minlength=n), out=Arp[1:])
    vals = rng.normal(size=(cols.shape[0], k, k))
    A = solve.Mat(n, n, Arp, cols, vals)
    C = solve.galerkin(P, A)
    assert np.array_equal(C.rowptr, A.rowptr) and np.array_equal(C.colidx, A.colidx)
    assert np.array_equal(C.vals, A.vals)
