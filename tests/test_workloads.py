"""Pins of the seeded input generator: P1 elasticity matrices are symmetric,
annihilate the rigid-body modes (Neumann), are SPD after clamping, and the
load vector integrates the body force."""
import numpy as np
import pytest
import scipy.sparse as sp

from workloads import configs, make_problem


def _csr(B):
    return sp.bsr_matrix((B.vals, B.colidx, B.rowptr),
                         shape=(B.n_rows * B.br, B.n_cols * B.bc)).tocsr()


def _rigid(x):
    n, d = x.shape
    if d == 2:
        W = np.zeros((n, 2, 3))
        W[:, 0, 0] = W[:, 1, 1] = 1
        W[:, 0, 2], W[:, 1, 2] = -x[:, 1], x[:, 0]
        return W.reshape(2 * n, 3)
    W = np.zeros((n, 3, 6))
    for a in range(3):
        W[:, a, a] = 1
    for r in range(3):
        e = np.zeros(3)
        e[r] = 1
        W[:, :, 3 + r] = np.cross(e, x)
    return W.reshape(3 * n, 6)


@pytest.mark.parametrize("shape", [(6, 5), (4, 5, 3)])
def test_matrix_symmetric_rigid_spd(shape):
    p = make_problem(shape, seed=3, nu_range=(0.25, 0.45), jump_boxes=3)
    AN = _csr(p.A_full)
    assert abs(AN - AN.T).max() == 0.0
    W = _rigid(p.coords)
    assert np.abs(AN @ W).max() <= 1e-13 * np.abs(AN).max()
    A = _csr(p.A).toarray()
    assert np.linalg.eigvalsh(A).min() > 0
    assert np.all(np.diff(p.A.colidx[p.A.rowptr[0]:p.A.rowptr[1]]) > 0)


def test_structured_sizes():
    p = configs.square32()
    assert (p.n_all, p.n_free, p.ndof) == (1089, 1056, 2112)
    assert np.diff(p.A_full.rowptr).max() == 7
    q = make_problem((6, 6, 6), seed=1)
    assert np.diff(q.A_full.rowptr).max() == 15
    assert q.n_free == 6 * 6 * 5


def test_load_vector_integrates_force():
    p = make_problem((7, 7), seed=4, forces=[[0.0, -1.0]], clamp=False)
    # sum of f |T|/(d+1) over vertices = f * area of the unit square
    assert abs(p.b[0].reshape(-1, 2)[:, 1].sum() + 1.0) < 1e-13


def test_boundary_stays_on_box():
    p = make_problem((5, 6, 4), seed=9)
    idx = np.stack(np.meshgrid(*[np.arange(s) for s in (5, 6, 4)], indexing="ij"), -1)
    idx = idx.reshape(-1, 3, order="F")
    for a, s in enumerate((5, 6, 4)):
        on = idx[:, a] == 0
        assert np.all(p.coords[on, a] == 0.0)
    X = p.coords[p.elements]
    J = np.transpose(X[:, 1:, :] - X[:, :1, :], (0, 2, 1))
    assert np.linalg.det(J).min() > 0


def test_seeded_reproducible():
    a = make_problem((5, 5), seed=12)
    b = make_problem((5, 5), seed=12)
    assert np.array_equal(a.A.vals, b.A.vals) and np.array_equal(a.coords, b.coords)


def test_jump_boxes_and_nu_per_element():
    """Inclusion boxes: every element modulus is the background E or one of
    the drawn 10^U(-3,3) values, inside [1e-3, 1e3], with several distinct
    boxes present; the modulus of an element equals that of the last box
    holding its centroid.  Per-element nu stays in its range.  Coefficient
    jumps leave A symmetric and SPD."""
    p = make_problem((9, 8, 7), seed=3, jump_boxes=40, nu_range=(0.25, 0.45))
    E = p.E_el
    assert np.all((E == 1.0) | ((E >= 1e-3) & (E <= 1e3)))
    assert len(np.unique(E[E != 1.0])) >= 5
    assert np.all((p.nu_el >= 0.25) & (p.nu_el <= 0.45))
    # last box wins: redraw the boxes from the same stream and recheck
    d = 3
    brng = np.random.default_rng([3, 1])
    ext = np.array([(s - 1) * p.h for s in p.shape])
    centres = brng.uniform(0.0, 1.0, size=(40, d)) * ext
    sides = brng.uniform(0.02, 0.2, size=(40, d)) * ext
    moduli = 10.0 ** brng.uniform(-3.0, 3.0, size=40)
    cen = p.coords[p.elements].mean(axis=1)
    for e in np.random.default_rng(0).choice(len(E), 200, replace=False):
        inside = [b for b in range(40) if np.all(np.abs(cen[e] - centres[b]) <= 0.5 * sides[b])]
        assert E[e] == (moduli[inside[-1]] if inside else 1.0)
    A = _csr(p.A).toarray()
    assert np.abs(A - A.T).max() <= 1e-12 * np.abs(A).max()
    assert np.linalg.eigvalsh(A).min() > 0


def test_paper_workloads_beam_and_eleven_boxes():
    """Sec. 7's vector model problem (beam [0,10] x [0,1]^2, clamped at
    x = 0, mu = 1, lambda = 0) and the difficult problem (eleven diagonal
    boxes [(i-1)/11, i/11]^3 with mu = lambda = 10^4, 1 elsewhere)."""
    from workloads import configs
    p = configs.beam(4)
    assert p.shape == (41, 5, 5) and abs(p.coords[:, 0].max() - 10.0) < 1e-12
    assert np.allclose(p.coords[:, 1:].max(axis=0), 1.0)
    assert p.n_free == 41 * 25 - 25 and np.all(p.nu_el == 0.0) and np.all(p.E_el == 1.0)
    q = configs.jump11(23)              # two cells per box side
    cen = q.coords[q.elements].mean(axis=1)
    k = np.floor(cen * 11).clip(0, 10)
    inside = (k[:, 0] == k[:, 1]) & (k[:, 1] == k[:, 2])
    mu = q.E_el / (1.0 + q.nu_el)       # the paper's mu (= 2 mu of the Hooke law)
    lam = q.E_el * q.nu_el / ((1 + q.nu_el) * (1 - 2 * q.nu_el))
    assert np.allclose(mu[inside], 1e4) and np.allclose(mu[~inside], 1.0)
    assert np.allclose(lam, mu)         # mu = lambda in the paper's form
    # every one of the eleven boxes holds elements (48 per box at 2 cells per side)
    assert sorted(np.unique(k[inside, 0]).astype(int).tolist()) == list(range(11))
    assert inside.sum() == 11 * 8 * 6
