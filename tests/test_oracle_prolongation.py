"""Pins of the prolongations and coarse matrices (Sec. 3 Def. pwp/pwp_el,
Lemma eet_is_diag, Sec. 6 Def. aux_sp): kernel preservation, row caps and
the block-local kernel of the coarse matrices."""
import numpy as np
import pytest

from oracle import hierarchy, topology as T
from workloads import make_problem


def _setup(shape, clamp, seed=11, **kw):
    p = make_problem(shape, seed=seed, clamp=clamp)
    params = hierarchy.SetupParams(coarse_max=kw.pop("coarse_max", 4), passes_first=2,
                                   passes_later=2, **kw)
    return p, hierarchy.setup(p, params, factor=clamp)


def _rigid_fine(p):
    return T.rigid_modes(p.coords[p.free], with_rotations=False)


@pytest.mark.parametrize("shape", [(10, 9), (5, 5, 5)])
@pytest.mark.parametrize("clamp", [False, True])
def test_prolongations_reproduce_rigid_modes(shape, clamp):
    """P_l w_c = w on every non-D row, for the tentative and the smoothed P
    (the kernel preservation that Def. pwp and Def. aux_sp are built for)."""
    p, H = _setup(shape, clamp)
    assert H.n_levels >= 3
    for lev, rec in enumerate(H.info["records"]):
        P = H.P[lev].scipy()
        xc = rec["xc"]
        Wc = T.rigid_modes(xc, with_rotations=True)
        if lev == 0:
            Wf = _rigid_fine(p)
        else:
            Wf = T.rigid_modes(H.info["records"][lev - 1]["xc"], with_rotations=True)
        kr = H.P[lev].br
        Dmask = rec["D"][rec["rowmap"]]
        rows_ok = np.repeat(~Dmask, kr)
        res = (P @ Wc - Wf)[rows_ok]
        assert np.abs(res).max() <= 1e-12 * max(1.0, np.abs(Wf).max()), (lev, np.abs(res).max())
        # tentative P: same statement (Def. pwp)
        k = T.kdim(p.dim)
        for r, row in enumerate(rec["tentative"]):
            for J, blk in row.items():
                np.testing.assert_allclose(blk @ Wc[J * k:(J + 1) * k], Wf[r * kr:(r + 1) * kr],
                                           atol=1e-13)


@pytest.mark.parametrize("shape", [(10, 9), (5, 5, 5)])
def test_neumann_coarse_matrices_annihilate_rigid_modes(shape):
    """Without Dirichlet conditions every A_l annihilates the level's rigid
    modes (the coarse spaces contain the kernel, Sec. 3)."""
    p, H = _setup(shape, clamp=False)
    W0 = _rigid_fine(p)
    A0 = H.A[0].scipy()
    assert np.abs(A0 @ W0).max() <= 1e-12 * np.abs(A0).max()
    for lev in range(1, H.n_levels):
        xc = H.info["records"][lev - 1]["xc"]
        W = T.rigid_modes(xc, with_rotations=True)
        Al = H.A[lev].scipy()
        assert np.abs(Al @ W).max() <= 1e-10 * np.abs(Al).max(), lev


@pytest.mark.parametrize("shape", [(10, 9), (5, 5, 5)])
def test_dirichlet_coarse_kernel_is_block_local(shape):
    """Lemma eet_is_diag: ker(A_l) is spanned by vectors living on single
    vertices, i.e. by the kernels of the diagonal blocks."""
    p, H = _setup(shape, clamp=True)
    for lev in range(1, H.n_levels):
        A = H.A[lev]
        Ad = A.scipy().toarray()
        scale = np.abs(Ad).max()
        w = np.linalg.eigvalsh(Ad)
        n_null = int((np.abs(w) <= 1e-10 * scale).sum())
        k = A.br
        local = 0
        for i in range(A.n_rows):
            Aii = A.block(i, i)
            wi, Vi = np.linalg.eigh(Aii)
            K = Vi[:, np.abs(wi) <= 1e-10 * scale]
            local += K.shape[1]
            for c in range(K.shape[1]):
                v = np.zeros(Ad.shape[0])
                v[i * k:(i + 1) * k] = K[:, c]
                assert np.abs(Ad @ v).max() <= 1e-9 * scale
        assert n_null == local
        assert w.min() >= -1e-10 * scale


def test_smoothed_prolongation_row_caps():
    """Row caps of Sec. 7: <= 8 (S, first level) / 6 (S, later) / 4 (A) blocks."""
    p, H = _setup((12, 12), clamp=True)
    for lev, rec in enumerate(H.info["records"]):
        P = H.P[lev]
        cnt = np.diff(P.rowptr)
        kinds = np.array(rec["kinds"])
        capS = 8 if lev == 0 else 6
        assert cnt[kinds == "S"].max(initial=0) <= capS
        assert cnt[kinds == "A"].max(initial=0) <= 4
        assert cnt[kinds == "D"].max(initial=0) == 0


@pytest.mark.parametrize("shape", [(17, 17), (7, 7, 7)])
def test_smoothing_lowers_prolongation_energy(shape):
    """Def. aux_sp smooths the tentative prolongation with one damped Jacobi
    step on the auxiliary matrix; with the smoothed-aggregation damping
    (omega = 2/3 for rho(D^-1 A) <= 2) it must lower the A-energy of every
    coarse basis function, and of the whole prolongation well below half
    (measured: 0.32-0.33 in total, at most 0.54 per column).  A damping of
    1, 4/3 or 2 misses these bounds."""
    from oracle import prolongation, solve
    p = make_problem(shape, seed=2)
    H = hierarchy.setup(p, hierarchy.SetupParams(max_levels=2, coarse_max=1))
    rec = H.info["records"][0]
    rp, ci, v = prolongation.to_bsr(rec["tentative"], H.P[0].n_cols, H.P[0].br, H.P[0].bc)
    Pt = solve.Mat(H.P[0].n_rows, H.P[0].n_cols, rp, ci, v).scipy().toarray()
    Ps = H.P[0].scipy().toarray()
    A = H.A[0].scipy().toarray()
    et = np.einsum("ij,ij->j", Pt, A @ Pt)
    es = np.einsum("ij,ij->j", Ps, A @ Ps)
    live = et > 1e-14 * et.max()
    assert (es[live] / et[live]).max() < 0.6
    assert es.sum() / et.sum() < 0.4
