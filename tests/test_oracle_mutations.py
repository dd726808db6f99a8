"""Planted mistakes in the oracle (on the CPU) must each fail a pin.

Each case monkeypatches one oracle function with a plausible error (a sign,
a dropped term, a transposed operand, a wrong frame) and checks that the
pin written for that part of the paper catches it."""
import numpy as np
import pytest

import oracle.coarsening as CO
import oracle.criteria as C
import oracle.prolongation as PR
import oracle.solve as S
import oracle.topology as T
from tests import test_oracle_criteria as tc
from tests import test_oracle_prolongation as tp
from tests import test_oracle_solve as ts
from tests import test_oracle_topology as tt


def _fails(fn, *a, **kw):
    with pytest.raises((AssertionError, np.linalg.LinAlgError)):
        fn(*a, **kw)


def test_wrong_sign_in_half_transfer(monkeypatch):
    monkeypatch.setattr(T, "Q_half", lambda xi, xj: T.Q(-0.5 * (np.asarray(xj) - np.asarray(xi))))
    _fails(tt.test_aux_matrix_annihilates_rigid_modes, (5, 5))


def test_transposed_skew(monkeypatch):
    orig = T.skew
    monkeypatch.setattr(T, "skew", lambda t: orig(t).T if len(t) == 3 else orig(t))
    _fails(tt.test_skew_is_cross_product, 3)


def test_dirichlet_edges_not_folded(monkeypatch):
    orig = T.coarse_topology
    monkeypatch.setattr(T, "coarse_topology",
                        lambda topo, agg, n_c, xc, use_dirichlet=True: orig(topo, agg, n_c, xc, False))
    monkeypatch.setattr(CO, "coarse_topology", T.coarse_topology)
    _fails(tt.test_galerkin_of_aux_matrix_is_coarse_aux_matrix, (7, 6), True)


def test_missing_l1_term(monkeypatch):
    def no_l1(A):
        n, k = A.n_rows, A.br
        rows = np.repeat(np.arange(n), np.diff(A.rowptr))
        diag = A.colidx == rows
        Mv = np.zeros((n, k, k))
        Mv[rows[diag]] = A.vals[diag]
        return S.batched_pinv(Mv, S.KERNEL_RTOL)
    monkeypatch.setattr(S, "block_l1_inverse", no_l1)
    p = tt.make_problem((11, 10), seed=21)
    H = ts.hierarchy.setup(p, ts.hierarchy.SetupParams(coarse_max=6, passes_first=2, passes_later=2))
    _fails(_l1_check, H)


def _l1_check(H):
    class Req:
        def getfixturevalue(self, name):
            return (None, H)
    ts.test_block_l1_smoother_dominates_A("h", Req())


def test_transposed_galerkin_operand(monkeypatch):
    orig = S.galerkin

    def bad(P, A):
        # P A P^T-style slip: each coarse block transposed
        C = orig(P, A)
        C.vals = np.ascontiguousarray(np.transpose(C.vals, (0, 2, 1)))
        return C
    p = tt.make_problem((11, 10), seed=21)
    H = ts.hierarchy.setup(p, ts.hierarchy.SetupParams(coarse_max=6, passes_first=2, passes_later=2))
    H.A = [H.A[0]] + [bad(P, A) for P, A in zip(H.P, H.A[:-1])]

    class Req:
        def getfixturevalue(self, name):
            return (p, H)
    _fails(ts.test_galerkin_pattern_and_values_brute_force, "h", Req())


def test_skipped_post_smoother(monkeypatch):
    def vc(H, b, level=0):
        if level == H.n_levels - 1:
            return S.coarse_solve(H, b)
        x = S.smooth(H.A[level], H.Minv[level], b)
        r = b - S.spmv(H.A[level], x)
        ec = vc(H, S.spmv(H.R[level], r), level + 1)
        return x + S.spmv(H.P[level], ec)
    monkeypatch.setattr(S, "vcycle", vc)
    p = tt.make_problem((11, 10), seed=21)
    H = ts.hierarchy.setup(p, ts.hierarchy.SetupParams(coarse_max=6, passes_first=2, passes_later=2))

    class Req:
        def getfixturevalue(self, name):
            return (p, H)
    _fails(ts.test_vcycle_is_spd, "h", Req())


def test_auxiliary_row_in_wrong_frame(monkeypatch):
    orig_half = T.Q_half

    def smoothed_wrong(A_rows, P_rows, topo, agg, D, rowmap, bad, first_level, pp=PR.ProlongParams()):
        # diagonal of an auxiliary row transported with Q^{li} instead of Q^{il}
        monkeypatch.setattr(PR, "Q_half", lambda xi, xj: orig_half(xj, xi))
        try:
            return orig_smoothed(A_rows, P_rows, topo, agg, D, rowmap, bad, first_level, pp)
        finally:
            monkeypatch.setattr(PR, "Q_half", orig_half)
    orig_smoothed = PR.smoothed
    monkeypatch.setattr(PR, "smoothed", smoothed_wrong)
    _fails(tp.test_prolongations_reproduce_rigid_modes, (10, 9), False)


def test_dropped_delta_term(monkeypatch):
    orig = C.mu_p
    monkeypatch.setattr(C, "mu_p", lambda topo, Dhat, nbrs, i, j, delta=1: orig(topo, Dhat, nbrs, i, j, 0))
    _fails(tc.test_mu_p_equals_mu_g_on_coarse_neumann_level)


def test_pair_measures_that_never_object(monkeypatch):
    """mu_p and mu_g that accept every pair (e.g. a dropped harmonic-mean
    term making the left side vanish) leave only mu_s: the two-grid
    robustness pin across coefficient jumps must fail."""
    monkeypatch.setattr(CO, "mu_p", lambda *a, **k: 0.0)
    monkeypatch.setattr(CO, "mu_g", lambda *a, **k: 0.0)
    _fails(tc.test_robust_criteria_keep_two_grid_conditioned_across_jumps)


@pytest.mark.parametrize("omega", [1.0, 4.0 / 3.0])
def test_wrong_smoothing_damping(monkeypatch, omega):
    """A damping other than the smoothed-aggregation one (undamped Jacobi,
    or 4/3 from a spectral-radius estimate of 1) fails the energy pin."""
    import dataclasses
    orig = PR.smoothed

    def wrong(A_rows, P_t, topo, agg, D, rowmap, bad, first, pp):
        return orig(A_rows, P_t, topo, agg, D, rowmap, bad, first, dataclasses.replace(pp, omega=omega))
    monkeypatch.setattr(PR, "smoothed", wrong)
    _fails(tp.test_smoothing_lowers_prolongation_energy, (7, 7, 7))


def test_candidate_of_maximal_mu_s(monkeypatch):
    """The text of Sec. 5.2 says 'maximizes'; the listing's minimal mu_s is
    the reading taken.  Ordering candidates by 1/mu_s tries the maximal one
    first and must fail the hand-derived pin."""
    orig = C.mu_s
    monkeypatch.setattr(CO, "mu_s", lambda tmax, tr, i, j: 1.0 / orig(tmax, tr, i, j))
    _fails(tc.test_algorithm1_tries_the_candidate_of_minimal_mu_s_first)


def test_later_pass_in_insertion_order(monkeypatch):
    monkeypatch.setattr(CO, "later_pass_order", lambda m: list(range(m)))
    _fails(tc.test_algorithm1_later_pass_visits_in_reverse_insertion_order)


def test_c_oracle_with_transposed_blocks(monkeypatch):
    """The C solve phase handed every square block transposed (a plausible
    row/column-major mix-up) must fail the dense Galerkin pin."""
    import oracle.csolve as CS
    from tests import test_oracle_csolve as tcs
    orig = CS._bsr

    def transposed(M):
        rp, ci, v = orig(M)
        if v.ndim == 3 and v.shape[1] == v.shape[2]:
            v = np.ascontiguousarray(np.transpose(v, (0, 2, 1)))
        return rp, ci, v
    monkeypatch.setattr(CS, "_bsr", transposed)
    _fails(tcs.test_galerkin_equals_dense_triple_product)


def test_gauss_seidel_post_sweep_not_reversed(monkeypatch):
    """Both sweeps forward: the V-cycle is no longer symmetric."""
    from tests import test_oracle_gs as tg
    orig = S.gs_sweep
    monkeypatch.setattr(S, "gs_sweep", lambda A, M, c, b, x=None, forward=True: orig(A, M, c, b, x, True))
    _fails(tg.test_gs_vcycle_symmetric_positive_and_two_grid_contracts)


def test_gauss_seidel_with_stale_values(monkeypatch):
    """A sweep that reads the values from before the sweep (block Jacobi
    with the Gauss-Seidel blocks) fails the splitting pin."""
    from tests import test_oracle_gs as tg

    def jacobi_like(A, Minv, colour, b, x=None, forward=True):
        n, k = A.n_rows, A.br
        x0 = np.zeros(n * k) if x is None else x.copy()
        r = (b - A.scipy() @ x0).reshape(n, k)
        return x0 + np.einsum("nij,nj->ni", Minv, r).ravel()
    monkeypatch.setattr(S, "gs_sweep", jacobi_like)
    _fails(tg.test_sweep_equals_block_triangular_splitting)


def test_colouring_in_index_order(monkeypatch):
    """Rows coloured in index order instead of smallest-last order fail the
    hand-derived colouring pin."""
    from tests import test_oracle_gs as tg
    monkeypatch.setattr(S, "smallest_last_order", lambda A: list(range(A.n_rows)))
    _fails(tg.test_colouring_follows_smallest_last_order_by_hand)


def test_smallest_last_without_tie_break_by_index(monkeypatch):
    """Ties of least degree broken by the largest index fail the pin too."""
    from tests import test_oracle_gs as tg
    import heapq

    def largest_index_first(A):
        n = A.n_rows
        deg = [int(np.sum(A.colidx[A.rowptr[i]:A.rowptr[i + 1]] != i)) for i in range(n)]
        heap = [(deg[i], -i) for i in range(n)]
        heapq.heapify(heap)
        removed, out = [False] * n, []
        while heap:
            d, mi = heapq.heappop(heap)
            i = -mi
            if removed[i] or d != deg[i]:
                continue
            removed[i] = True
            out.append(i)
            for j in A.colidx[A.rowptr[i]:A.rowptr[i + 1]].tolist():
                if j != i and not removed[j]:
                    deg[j] -= 1
                    heapq.heappush(heap, (deg[j], -j))
        return out[::-1]
    monkeypatch.setattr(S, "smallest_last_order", largest_index_first)
    _fails(tg.test_colouring_follows_smallest_last_order_by_hand)


def test_scalar_edge_weights_with_sign(monkeypatch):
    """E^{ij} = A_ij instead of |A_ij| (negative weights) fails the exact
    M-matrix splitting pin."""
    from tests import test_oracle_scalar as tsc
    orig = T.finest_topology_scalar

    def signed(coords, rp, ci, vals, dirichlet):
        t = orig(coords, rp, ci, vals, dirichlet)
        rows = np.repeat(np.arange(coords.shape[0]), np.diff(rp))
        upper = np.asarray(ci) > rows
        t.E = np.asarray(vals, dtype=np.float64).reshape(-1)[upper].reshape(-1, 1, 1)
        return t
    monkeypatch.setattr(T, "finest_topology_scalar", signed)
    _fails(tsc.test_weights_split_an_m_matrix_exactly)
