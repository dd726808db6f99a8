"""The C solve phase of the oracle (oracle/csolve.c) against oracle/solve.py
(itself pinned against the paper by tests/test_oracle_solve.py and
tests/test_oracle_gs.py) and against facts of its own: the Galerkin product
equals the dense P^T A P, the V-cycle (block-l1 Jacobi and hybrid
Gauss-Seidel) is symmetric positive definite, PCG recovers a manufactured
solution, and the results do not depend on the number of threads."""
import numpy as np
import pytest

from oracle import csolve, hierarchy, solve
from workloads import configs, make_problem

CASES = {
    "square32": lambda: (configs.square32(), hierarchy.SetupParams()),
    "cube10": lambda: (make_problem((10, 10, 10), seed=2), hierarchy.SetupParams(coarse_max=8)),
    "box_jump": lambda: (make_problem((9, 7, 8), seed=3, jump_boxes=6, nu_range=(0.25, 0.45)),
                         hierarchy.SetupParams(coarse_max=6)),
}
_H = {}


def _case(name):
    if name not in _H:
        p, prm = CASES[name]()
        H = hierarchy.setup(p, prm)
        _H[name] = (p, H, csolve.Hierarchy(H.A[0], H.P))
    return _H[name]


def maxrel(a, b):
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))


@pytest.mark.parametrize("name", sorted(CASES))
def test_galerkin_matches_numpy_oracle(name):
    """Same structural pattern (bit-exact) and values to 1e-13 on every level."""
    p, H, Hc = _case(name)
    assert Hc.n_levels == H.n_levels
    for l in range(1, H.n_levels):
        np.testing.assert_array_equal(Hc.A[l].rowptr, H.A[l].rowptr)
        np.testing.assert_array_equal(Hc.A[l].colidx, H.A[l].colidx)
        assert maxrel(Hc.A[l].vals, H.A[l].vals) <= 1e-13, l


def test_galerkin_equals_dense_triple_product():
    """A_c = P^T A P against the dense product on a tiny mesh, and every
    structurally reached block is stored."""
    p = make_problem((6, 5), seed=4)
    H = hierarchy.setup(p, hierarchy.SetupParams(coarse_max=2))
    A, P = H.A[0], H.P[0]
    Ac = csolve.galerkin(P, A)
    dense = P.scipy().toarray().T @ A.scipy().toarray() @ P.scipy().toarray()
    assert np.abs(Ac.scipy().toarray() - dense).max() <= 1e-13 * np.abs(dense).max()
    k = P.bc
    pat = (np.abs(P.scipy().toarray()).T > 0).astype(int) @ (np.abs(A.scipy().toarray()) > 0) @ \
        (np.abs(P.scipy().toarray()) > 0)
    blocks = pat.reshape(P.n_cols, k, P.n_cols, k).sum(axis=(1, 3)) > 0
    stored = np.zeros_like(blocks)
    for i in range(Ac.n_rows):
        stored[i, Ac.colidx[Ac.rowptr[i]:Ac.rowptr[i + 1]]] = True
    assert np.array_equal(stored, blocks)


@pytest.mark.parametrize("name", sorted(CASES))
def test_spmv_and_vcycle_match_numpy_oracle(name):
    p, H, Hc = _case(name)
    rng = np.random.default_rng(5)
    n = H.A[0].n_rows * H.A[0].br
    x = rng.normal(size=n)
    assert maxrel(csolve.spmv(H.A[0], x), H.A[0].scipy() @ x) <= 1e-14
    for r in (p.b[0], x):
        assert maxrel(Hc.vcycle(r), solve.vcycle(H, r)) <= 1e-11


def test_vcycle_symmetric_positive():
    p, H, Hc = _case("cube10")
    rng = np.random.default_rng(6)
    n = H.A[0].n_rows * H.A[0].br
    x, y = rng.normal(size=(2, n))
    bx, by = Hc.vcycle(x), Hc.vcycle(y)
    assert abs(y @ bx - x @ by) <= 1e-12 * abs(x @ bx)
    assert x @ bx > 0 and y @ by > 0


@pytest.mark.parametrize("name", sorted(CASES))
def test_pcg_matches_numpy_oracle(name):
    p, H, Hc = _case(name)
    f = p.b[0]
    u, it, hist = Hc.pcg(f, rtol=1e-8)
    u_np, it_np, hist_np = solve.pcg(H, f, rtol=1e-8)
    assert abs(it - it_np) <= 1 and hist[-1] <= 1e-8
    u_k = u_np if it == it_np else solve.pcg(H, f, rtol=0.0, maxit=it)[0]
    assert maxrel(u, u_k) <= 1e-10


def test_pcg_recovers_manufactured_solution():
    p, H, Hc = _case("box_jump")
    A = H.A[0]
    u_star = np.random.default_rng(7).normal(size=A.n_rows * A.br)
    f = A.scipy() @ u_star
    u, it, _ = Hc.pcg(f, rtol=1e-12, maxit=1000)
    e = u - u_star
    assert np.sqrt(e @ (A.scipy() @ e) / (u_star @ (A.scipy() @ u_star))) <= 1e-9


def test_results_do_not_depend_on_threads():
    p, H, Hc = _case("cube10")
    f = p.b[0]
    outs = []
    try:
        for t in (1, 4):
            csolve.set_threads(t)
            Ac = csolve.galerkin(H.P[0], H.A[0])
            u, it, _ = Hc.pcg(f, rtol=1e-8)
            outs.append((Ac, u, it))
    finally:
        csolve.set_threads(csolve.max_threads())
    (A1, u1, i1), (A4, u4, i4) = outs
    assert np.array_equal(A1.vals, A4.vals) and np.array_equal(A1.colidx, A4.colidx)
    assert i1 == i4 and maxrel(u4, u1) <= 1e-12


def test_pcg_zero_rhs_stops_at_once():
    p, H, Hc = _case("square32")
    u, it, hist = Hc.pcg(np.zeros_like(p.b[0]), rtol=1e-8)
    assert it == 0 and not u.any() and hist == [0.0]


_GS = {}


def _gs_case(name):
    """The same hierarchy with the block-l1 hybrid Gauss-Seidel smoother, in
    oracle/solve.py and in the C solve phase."""
    if name not in _GS:
        p, H, _ = _case(name)
        _GS[name] = (p, solve.prepare(H.A[0], H.P, smoother="hybrid_gs"),
                     csolve.Hierarchy(H.A[0], H.P, smoother="hybrid_gs"))
    return _GS[name]


@pytest.mark.parametrize("name", sorted(CASES))
def test_gs_vcycle_matches_numpy_oracle(name):
    p, Hg, Hc = _gs_case(name)
    for l, c in enumerate(Hg.colour):
        np.testing.assert_array_equal(Hc.colour[l], c)
    n = Hg.A[0].n_rows * Hg.A[0].br
    for r in (p.b[0], np.random.default_rng(8).normal(size=n)):
        assert maxrel(Hc.vcycle(r), solve.vcycle(Hg, r)) <= 1e-11


def test_gs_vcycle_differs_from_jacobi_and_is_symmetric_positive():
    """The forward / backward sweeps make a symmetric V-cycle (the backward
    sweep is the adjoint of the forward one); it is not the Jacobi V-cycle."""
    p, Hg, Hc = _gs_case("cube10")
    _, _, Hj = _case("cube10")
    rng = np.random.default_rng(9)
    n = Hg.A[0].n_rows * Hg.A[0].br
    x, y = rng.normal(size=(2, n))
    bx, by = Hc.vcycle(x), Hc.vcycle(y)
    assert abs(y @ bx - x @ by) <= 1e-12 * abs(x @ bx)
    assert x @ bx > 0 and y @ by > 0
    assert maxrel(bx, Hj.vcycle(x)) > 1e-3


@pytest.mark.parametrize("name", sorted(CASES))
def test_gs_pcg_matches_numpy_oracle(name):
    p, Hg, Hc = _gs_case(name)
    f = p.b[0]
    u, it, hist = Hc.pcg(f, rtol=1e-8)
    u_np, it_np, _ = solve.pcg(Hg, f, rtol=1e-8)
    assert abs(it - it_np) <= 1 and hist[-1] <= 1e-8
    u_k = u_np if it == it_np else solve.pcg(Hg, f, rtol=0.0, maxit=it)[0]
    assert maxrel(u, u_k) <= 1e-10


def test_gs_results_do_not_depend_on_threads():
    p, Hg, Hc = _gs_case("box_jump")
    f = p.b[0]
    outs = []
    try:
        for t in (1, 4):
            csolve.set_threads(t)
            outs.append(Hc.pcg(f, rtol=1e-8)[:2])
    finally:
        csolve.set_threads(csolve.max_threads())
    (u1, i1), (u4, i4) = outs
    assert i1 == i4 and maxrel(u4, u1) <= 1e-12


def test_unknown_smoother_rejected():
    p, H, _ = _case("square32")
    with pytest.raises(ValueError):
        csolve.Hierarchy(H.A[0], H.P, smoother="gs")
