"""Pins of the oracle's block-l1 hybrid Gauss-Seidel smoother (the other
form of the l1 smoothers Sec. 7 cites; on one device: block Gauss-Seidel
over the colour classes of a distance-1 colouring) against the matrix
splitting it must equal, the symmetry the V-cycle needs, and the two-grid
robustness experiment of Sec. 5 (which the paper runs with Gauss-Seidel)."""
import numpy as np
import pytest

from oracle import hierarchy, solve
from workloads import configs, make_problem


def _gs_hier(p, **kw):
    H = hierarchy.setup(p, hierarchy.SetupParams(**kw))
    return H, solve.prepare(H.A[0], H.P, "hybrid_gs")


def test_colouring_is_distance_one_and_greedy_bounded():
    p = make_problem((9, 8, 7), seed=3, jump_boxes=4)
    H, Hg = _gs_hier(p, coarse_max=6)
    for A, col in zip(Hg.A[:-1], Hg.colour):
        rows = np.repeat(np.arange(A.n_rows), np.diff(A.rowptr))
        off = A.colidx != rows
        assert not np.any(col[rows[off]] == col[A.colidx[off]])     # no coupled pair shares a colour
        deg = np.diff(A.rowptr).max() - 1
        assert col.min() == 0 and col.max() <= deg                   # greedy: at most max degree + 1
        assert set(np.unique(col).tolist()) == set(range(int(col.max()) + 1))


def _path_in_bad_order():
    """The path a - b - c - d stored as rows a = 0, d = 1, b = 2, c = 3 (1x1
    blocks): in index order the greedy colouring takes a = 0, d = 0, b = 1
    and c, next to b = 1 and d = 0, needs a third colour."""
    edges = {0: [2], 1: [3], 2: [0, 3], 3: [1, 2]}
    rowptr, colidx = [0], []
    for i in range(4):
        colidx.extend(sorted(edges[i] + [i]))
        rowptr.append(len(colidx))
    return solve.Mat(n_rows=4, n_cols=4, rowptr=np.array(rowptr), colidx=np.array(colidx),
                     vals=np.ones((len(colidx), 1, 1)))


def test_colouring_follows_smallest_last_order_by_hand():
    """Smallest-last on the path above, derived by hand: degrees a 1, d 1,
    b 2, c 2; remove a (least degree, smallest index), then d (b and d have
    degree 1, d has the smaller index), then b, then c.  The order is the
    reverse, c, b, d, a; greedy: c = 0, b = 1, d = 1, a = 0 -- two colours
    where the index order needs three."""
    A = _path_in_bad_order()
    assert solve.smallest_last_order(A) == [3, 2, 1, 0]
    assert solve.greedy_colouring(A).tolist() == [0, 1, 1, 0]


def test_sweep_equals_block_triangular_splitting():
    """A forward sweep is x + (L + D)^{-1}(b - A x) with the matrix ordered by
    colour (classes in order, rows by index inside a class), L its strictly
    block-lower part and D the block diagonal of the M_v; a backward sweep
    uses the block-upper part.  Checked against a dense triangular solve."""
    p = make_problem((7, 6), seed=5, nu=0.3)
    H, Hg = _gs_hier(p, coarse_max=4)
    A, col, Minv = Hg.A[0], Hg.colour[0], Hg.Minv[0]
    n, k = A.n_rows, A.br
    Ad = A.scipy().toarray()
    perm = np.lexsort((np.arange(n), col))                 # by colour, then row
    rank = np.empty(n, dtype=np.int64)
    rank[perm] = np.arange(n)
    rng = np.random.default_rng(1)
    b, x = rng.normal(size=(2, n * k))
    for forward in (True, False):
        M = np.zeros_like(Ad)
        for i in range(n):
            for j in range(n):
                blk = Ad[i * k:(i + 1) * k, j * k:(j + 1) * k]
                if i == j:
                    M[i * k:(i + 1) * k, i * k:(i + 1) * k] = np.linalg.pinv(Minv[i])
                elif (rank[j] < rank[i]) == forward:
                    M[i * k:(i + 1) * k, j * k:(j + 1) * k] = blk
        want = x + np.linalg.solve(M, b - Ad @ x)
        got = solve.gs_sweep(A, Minv, col, b, x, forward=forward)
        assert np.abs(got - want).max() <= 1e-10 * np.abs(want).max(), forward


def test_gs_vcycle_symmetric_positive_and_two_grid_contracts():
    p = make_problem((8, 7, 6), seed=4)
    H, Hg = _gs_hier(p, coarse_max=20, max_levels=2)
    n = Hg.A[0].n_rows * Hg.A[0].br
    rng = np.random.default_rng(2)
    x, y = rng.normal(size=(2, n))
    bx, by = solve.vcycle(Hg, x), solve.vcycle(Hg, y)
    assert abs(y @ bx - x @ by) <= 1e-11 * abs(x @ bx)
    assert x @ bx > 0 and y @ by > 0
    # two-grid error propagation I - B A has spectral radius < 1
    Ad = Hg.A[0].scipy().toarray()
    B = np.column_stack([solve.vcycle(Hg, e) for e in np.eye(n)])
    rho = np.abs(np.linalg.eigvals(np.eye(n) - B @ Ad)).max()
    assert rho < 1.0


def test_gs_needs_fewer_iterations_than_jacobi():
    p = configs.square32()
    H, Hg = _gs_hier(p)
    _, it_j, _ = solve.pcg(H, p.b[0], rtol=1e-8)
    _, it_g, _ = solve.pcg(Hg, p.b[0], rtol=1e-8)
    assert it_g < it_j


def test_robust_criteria_keep_gauss_seidel_two_grid_conditioned_across_jumps():
    """Sec. 5's coefficient-jump experiment with the Gauss-Seidel smoother,
    as the paper runs it (kappa about 2.84 with mu_p, mu_g against about 270
    with mu_s alone on its mesh): here the 4 x 4 checkerboard of E = 10^4 and
    E = 1 boxes on a 17 x 17 mesh, one coarsening step, the symmetric hybrid
    Gauss-Seidel two-grid preconditioner, kappa from a dense eigen-solve."""
    def checker(c, nb=4):
        i = np.floor(c[:, 0] * nb).clip(0, nb - 1)
        j = np.floor(c[:, 1] * nb).clip(0, nb - 1)
        return np.where((i + j) % 2 == 1, 1e4, 1.0)

    p = make_problem((17, 17), seed=1, nu=0.25, E_fn=checker)
    kappas = []
    for scalar_only in (False, True):
        H = hierarchy.setup(p, hierarchy.SetupParams(max_levels=2, coarse_max=1,
                                                     scalar_only=scalar_only))
        Hg = solve.prepare(H.A[0], H.P, "hybrid_gs")
        n = Hg.A[0].n_rows * Hg.A[0].br
        V = np.column_stack([solve.vcycle(Hg, e) for e in np.eye(n)])
        A = Hg.A[0].scipy().toarray()
        ev = np.linalg.eigvals(V @ A).real
        assert ev.min() > 0
        kappas.append(ev.max() / ev.min())
    robust, scalar = kappas
    assert robust < 10.0
    assert scalar > 50.0 * robust
