"""Pins of the learned-smoother oracle (oracle/learned.py) against what the
mathematics fixes: central finite differences for the backward pass, SPD
outputs, closed forms for zero weights, invariances of the features, the
Schur-complement form and Loewner bound of the patch targets, and a dense
eigen-solve for the Lanczos estimate."""
import copy

import numpy as np
import pytest

from oracle import hierarchy, learned, solve
from workloads import make_problem


def _prob(shape=(5, 4, 4), seed=3, **kw):
    p = make_problem(shape, seed=seed, **kw)
    return p, solve.mat_from(p.A), p.coords[p.free]


def test_param_count():
    assert learned.N_PARAMS == 13 * 64 + 64 + 64 * 64 + 64 + 6 * 64 + 6 == 5446
    th = np.arange(learned.N_PARAMS, dtype=float)
    assert np.array_equal(learned.pack(learned.unpack(th)), th)


def test_backward_matches_central_differences():
    rng = np.random.default_rng(1)
    theta = learned.init_params(2) + 0.05 * rng.normal(size=learned.N_PARAMS)
    X = rng.normal(size=(17, 13))
    M = rng.normal(size=(17, 3, 3))
    T = np.einsum("nab,ncb->nac", M, M) + 0.1 * np.eye(3)
    loss, g = learned.loss_grad(theta, X, T)
    idx = np.concatenate([rng.choice(learned.N_PARAMS, 60, replace=False),
                          np.arange(learned.N_PARAMS - 6, learned.N_PARAMS)])
    h = 1e-6
    for i in idx:
        tp, tm = theta.copy(), theta.copy()
        tp[i] += h
        tm[i] -= h
        fd = (learned.loss_grad(tp, X, T)[0] - learned.loss_grad(tm, X, T)[0]) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 * max(1.0, abs(g[i])) + 1e-8, (i, fd, g[i])


def test_outputs_spd_and_zero_weight_closed_form():
    rng = np.random.default_rng(4)
    theta = learned.init_params(5)
    X = rng.normal(size=(50, 13))
    tr = rng.uniform(0.5, 3.0, size=50)
    B = learned.smoother_blocks(theta, X, tr)
    assert np.allclose(B, np.transpose(B, (0, 2, 1)))
    assert np.linalg.eigvalsh(B).min() > 0
    # zero weights: the output is the bias b3, B = (L(b3) L(b3)^T + eps I) / tr
    p = learned.unpack(np.zeros(learned.N_PARAMS))
    p["b3"] = np.array([2.0, 0.5, 1.0, -0.25, 0.75, 3.0])
    B0 = learned.smoother_blocks(learned.pack(p), X, tr)
    L = np.array([[2.0, 0, 0], [0.5, 1.0, 0], [-0.25, 0.75, 3.0]])
    want = (L @ L.T + 1e-6 * np.eye(3))
    assert np.allclose(B0 * tr[:, None, None], want, rtol=0, atol=1e-14)


def test_features_invariances():
    p, A, x = _prob()
    X, tr = learned.features(A, x)
    assert X.shape == (A.n_rows, 13)
    # scaling the operator or the geometry (rigidly moved, uniformly scaled)
    A2 = solve.Mat(A.n_rows, A.n_cols, A.rowptr, A.colidx, 7.5 * A.vals)
    X2, tr2 = learned.features(A2, x)
    assert np.allclose(X2, X, rtol=1e-14, atol=1e-15) and np.allclose(tr2, 7.5 * tr)
    R = np.linalg.qr(np.random.default_rng(0).normal(size=(3, 3)))[0]
    X3, _ = learned.features(A, 3.0 * x @ R.T + 1.0)
    assert np.allclose(X3[:, 12], X[:, 12])
    # the edge sum rotates with the geometry: its trace is invariant
    assert np.allclose(X3[:, 6:9].sum(1), X[:, 6:9].sum(1), rtol=1e-12)
    # diagonal-block features have unit trace; degree counts off-diagonal blocks
    assert np.allclose(X[:, 0:3].sum(1), 1.0)
    deg = np.diff(A.rowptr) - 1
    assert np.allclose(X[:, 12] * 14, deg)


def test_patch_target_schur_form_and_loewner_bound():
    p, A, x = _prob()
    for v in (0, 7, A.n_rows // 2, A.n_rows - 1):
        T = learned.patch_target(A, v)
        nb, D = learned.patch(A, v)
        # v is last: the vv block of the inverse is the inverse Schur complement
        m = 3 * (len(nb) - 1)
        S = D[m:, m:] - D[m:, :m] @ np.linalg.solve(D[:m, :m], D[:m, m:])
        assert np.allclose(T, np.linalg.inv(S), rtol=1e-10, atol=0)
        # and it dominates the inverse of the diagonal block (Loewner order)
        Dinv = np.linalg.inv(D[m:, m:])
        assert np.linalg.eigvalsh(T - Dinv).min() >= -1e-12 * np.abs(T).max()
    # scale invariance of the normalised target
    A2 = solve.Mat(A.n_rows, A.n_cols, A.rowptr, A.colidx, 3.0 * A.vals)
    assert np.allclose(learned.targets(A2)[:5], learned.targets(A)[:5], rtol=1e-12)


def test_patch_target_decoupled_vertex_is_block_inverse():
    """A vertex whose off-diagonal blocks are zero: T_v = A_vv^{-1}."""
    p, A, x = _prob()
    vals = A.vals.copy()
    v = 5
    for q in range(A.rowptr[v], A.rowptr[v + 1]):
        if A.colidx[q] != v:
            vals[q] = 0.0
    A2 = solve.Mat(A.n_rows, A.n_cols, A.rowptr, A.colidx, vals)
    D = [A.vals[q] for q in range(A.rowptr[v], A.rowptr[v + 1]) if A.colidx[q] == v][0]
    assert np.allclose(learned.patch_target(A2, v), np.linalg.inv(D), rtol=1e-12)


def test_lanczos_exact_on_small_space_and_lower_bound():
    p, A, x = _prob((2, 3, 3), seed=6)          # 9 free vertices, 27 dofs
    rng = np.random.default_rng(2)
    M = rng.normal(size=(A.n_rows, 3, 3))
    B = np.einsum("nab,ncb->nac", M, M) + 0.5 * np.eye(3)
    Ad = np.zeros((27, 27))
    for r in range(A.n_rows):
        for q in range(A.rowptr[r], A.rowptr[r + 1]):
            c = A.colidx[q]
            Ad[3 * r:3 * r + 3, 3 * c:3 * c + 3] = A.vals[q]
    Bd = np.zeros((27, 27))
    for r in range(A.n_rows):
        Bd[3 * r:3 * r + 3, 3 * r:3 * r + 3] = B[r]
    lam = np.linalg.eigvals(Bd @ Ad).real.max()
    assert abs(learned.lanczos_lambda_max(A, B) - lam) <= 1e-8 * lam
    p, A, x = _prob((6, 5, 5), seed=7)
    B = np.tile(np.eye(3), (A.n_rows, 1, 1)) * 0.3
    est = learned.lanczos_lambda_max(A, B, steps=10)
    full = learned.lanczos_lambda_max(A, B, steps=200)
    assert est <= full * (1 + 1e-12)


def test_learned_vcycle_is_spd_and_pcg_converges():
    """With any SPD blocks and the safeguarded omega, the V-cycle stays a
    symmetric positive definite preconditioner and PCG converges."""
    p = make_problem((8, 7, 7), seed=8)
    H = hierarchy.setup(p)
    A0 = H.A[0]
    X, tr = learned.features(A0, p.coords[p.free])
    B = learned.smoother_blocks(learned.init_params(3), X, tr)
    w = learned.omega(learned.lanczos_lambda_max(A0, B))
    H2 = copy.copy(H)
    H2.Minv = list(H.Minv)
    H2.Minv[0] = w * B
    rng = np.random.default_rng(0)
    a, b = rng.normal(size=(2, A0.n_rows * 3))
    va, vb = solve.vcycle(H2, a), solve.vcycle(H2, b)
    assert abs(b @ va - a @ vb) <= 1e-10 * abs(a @ va)
    assert a @ va > 0 and b @ vb > 0
    # V-cycle iteration x <- x + B_V (f - A x) contracts: rho(I - B_V A) < 1
    n = A0.n_rows * 3
    rho = solve.spectral_radius_power(lambda e: e - solve.vcycle(H2, solve.spmv(A0, e)), n,
                                      iters=300)
    assert rho < 1.0
    u, it, hist = solve.pcg(H2, p.b[0], rtol=1e-8, maxit=2000)
    assert hist[-1] <= 1e-8
