"""Learned per-vertex smoother for the finest level (an extension; the paper
has no learned component): FP64 reference of features, training targets,
the MLP with its forward and backward pass, and the damping safeguard.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

* Features of vertex v (13): the diagonal block A_vv (6 unique entries) and
  the sum over the vertex's edges of the finest-level edge matrices'
  displacement part c^{vj} t t^T (t = x_j - x_v, c^{vj} the mean absolute
  entry of the off-diagonal block, Thm. deng_elast with its Remark), both
  divided by tr A_vv, the edge sum also by the mean squared edge length at v
  (so that the features do not depend on the mesh size), and the degree / 14
  (14 = degree of an interior vertex of the Kuhn tetrahedral grid).
* Target: the vv block of the inverse of the patch matrix A_{N(v),N(v)},
  N(v) = v and its neighbours, times tr A_vv.
* MLP 13 -> 64 -> 64 -> 6 with ReLU; the 6 outputs are a lower-triangular
  3x3 factor L and the smoother block is B_v = (L L^T + 1e-6 I) / tr A_vv,
  symmetric positive definite by construction.
* Loss: mean over vertices of ||L L^T + 1e-6 I - T_v tr A_vv||_F^2.
* Safeguard: x += omega B r is a convergent smoother iff omega lambda_max(BA)
  < 2; lambda_max comes from 30 Lanczos steps (times 1.05) and omega =
  4 / (3 lambda_hat), the usual damping of Jacobi-type smoothers.

The smoother replaces the block-l1 Jacobi blocks of level 0 in the V-cycle
(``solve.vcycle`` with ``Minv[0] = omega * B``).
"""
from __future__ import annotations

from typing import Dict, Tuple

import numpy as np

from .solve import Mat, spmv

N_IN, N_HID, N_OUT = 13, 64, 6
SHAPES = [("W1", (N_HID, N_IN)), ("b1", (N_HID,)), ("W2", (N_HID, N_HID)), ("b2", (N_HID,)),
          ("W3", (N_OUT, N_HID)), ("b3", (N_OUT,))]
N_PARAMS = sum(int(np.prod(s)) for _, s in SHAPES)  # 5446
TRIL = [(0, 0), (1, 0), (1, 1), (2, 0), (2, 1), (2, 2)]
EPS = 1e-6
DEGREE_SCALE = 14.0
LANCZOS_STEPS = 30
LANCZOS_SAFETY = 1.05
OMEGA_NUM = 4.0 / 3.0
UNIQUE = [(0, 0), (1, 1), (2, 2), (0, 1), (0, 2), (1, 2)]


def unpack(theta) -> Dict[str, np.ndarray]:
    out, o = {}, 0
    for name, shape in SHAPES:
        m = int(np.prod(shape))
        out[name] = np.asarray(theta[o:o + m], dtype=np.float64).reshape(shape)
        o += m
    return out


def pack(p: Dict[str, np.ndarray]) -> np.ndarray:
    return np.concatenate([np.asarray(p[name], dtype=np.float64).reshape(-1) for name, _ in SHAPES])


def _diag_block(A: Mat, v: int) -> np.ndarray:
    for q in range(A.rowptr[v], A.rowptr[v + 1]):
        if A.colidx[q] == v:
            return A.vals[q]
    raise ValueError(f"row {v} has no diagonal block")


def features(A: Mat, coords) -> Tuple[np.ndarray, np.ndarray]:
    """(X (n, 13), tr A_vv (n,)) for the 3x3-block matrix A on vertices with
    positions coords (n, 3)."""
    if A.br != 3:
        raise ValueError("the learned smoother is defined for 3D elasticity (3x3 blocks)")
    coords = np.asarray(coords, dtype=np.float64)
    n = A.n_rows
    X = np.zeros((n, N_IN))
    tr = np.zeros(n)
    for v in range(n):
        D = _diag_block(A, v)
        tr[v] = np.trace(D)
        S = np.zeros((3, 3))
        l2, deg = 0.0, 0
        for q in range(A.rowptr[v], A.rowptr[v + 1]):
            j = A.colidx[q]
            if j == v:
                continue
            c = np.abs(A.vals[q]).sum() / 9.0
            t = coords[j] - coords[v]
            S += c * np.outer(t, t)
            l2 += t @ t
            deg += 1
        hs = l2 / deg if deg else 1.0
        X[v, 0:6] = [D[a, b] / tr[v] for a, b in UNIQUE]
        X[v, 6:12] = [S[a, b] / (tr[v] * hs) for a, b in UNIQUE]
        X[v, 12] = deg / DEGREE_SCALE
    return X, tr


def patch(A: Mat, v: int):
    """Vertices of N(v) (neighbours in row order, v last) and the dense patch
    matrix A_{N(v),N(v)}."""
    nb = [int(c) for c in A.colidx[A.rowptr[v]:A.rowptr[v + 1]] if c != v] + [v]
    pos = {c: i for i, c in enumerate(nb)}
    m = len(nb)
    D = np.zeros((3 * m, 3 * m))
    for a, r in enumerate(nb):
        for q in range(A.rowptr[r], A.rowptr[r + 1]):
            b = pos.get(int(A.colidx[q]))
            if b is not None:
                D[3 * a:3 * a + 3, 3 * b:3 * b + 3] = A.vals[q]
    return nb, D


def patch_target(A: Mat, v: int) -> np.ndarray:
    """[(A_{N(v),N(v)})^{-1}]_{vv} (3x3)."""
    _, D = patch(A, v)
    return np.linalg.inv(D)[-3:, -3:]


def targets(A: Mat) -> np.ndarray:
    """Normalised targets T_v tr A_vv, (n, 3, 3)."""
    out = np.zeros((A.n_rows, 3, 3))
    for v in range(A.n_rows):
        out[v] = patch_target(A, v) * np.trace(_diag_block(A, v))
    return out


def forward(theta, X):
    """Outputs (n, 6) and the activations the backward pass needs."""
    p = unpack(theta)
    X = np.asarray(X, dtype=np.float64)
    z1 = X @ p["W1"].T + p["b1"]
    h1 = np.maximum(z1, 0.0)
    z2 = h1 @ p["W2"].T + p["b2"]
    h2 = np.maximum(z2, 0.0)
    out = h2 @ p["W3"].T + p["b3"]
    return out, (X, z1, h1, z2, h2)


def factor(out) -> np.ndarray:
    """Lower-triangular L (n, 3, 3) from the 6 outputs (row-major lower order)."""
    L = np.zeros((out.shape[0], 3, 3))
    for o, (a, b) in enumerate(TRIL):
        L[:, a, b] = out[:, o]
    return L


def spd_blocks(out) -> np.ndarray:
    """L L^T + eps I (the normalised smoother block)."""
    L = factor(out)
    return np.einsum("nab,ncb->nac", L, L) + EPS * np.eye(3)


def loss_grad(theta, X, Tn):
    """Mean loss over the n samples and its gradient (flat, N_PARAMS)."""
    p = unpack(theta)
    out, (X, z1, h1, z2, h2) = forward(theta, X)
    n = X.shape[0]
    L = factor(out)
    G = spd_blocks(out) - Tn
    loss = float((G ** 2).sum() / n)
    dS = 2.0 * G / n                                   # d loss / d S
    dL = np.einsum("nac,ncb->nab", dS + np.transpose(dS, (0, 2, 1)), L)
    dout = np.stack([dL[:, a, b] for a, b in TRIL], axis=1)
    g = {"W3": dout.T @ h2, "b3": dout.sum(0)}
    dh2 = (dout @ p["W3"]) * (z2 > 0)
    g["W2"] = dh2.T @ h1
    g["b2"] = dh2.sum(0)
    dh1 = (dh2 @ p["W2"]) * (z1 > 0)
    g["W1"] = dh1.T @ X
    g["b1"] = dh1.sum(0)
    return loss, pack(g)


def smoother_blocks(theta, X, tr) -> np.ndarray:
    """B_v = (L L^T + eps I) / tr A_vv, (n, 3, 3)."""
    out, _ = forward(theta, X)
    return spd_blocks(out) / np.asarray(tr)[:, None, None]


def apply_blocks(B, r):
    n = B.shape[0]
    return np.einsum("vab,vb->va", B, np.asarray(r).reshape(n, 3)).reshape(-1)


def lanczos_lambda_max(A: Mat, B, steps=LANCZOS_STEPS, seed=0) -> float:
    """Largest eigenvalue of the Lanczos tridiagonal matrix of BA in the
    A-inner product (BA is self-adjoint there): a lower estimate of
    lambda_max(BA) that is exact once the Krylov space is invariant."""
    n = A.n_rows * A.br
    v = np.random.default_rng(seed).normal(size=n)
    u = spmv(A, v)
    nrm = np.sqrt(v @ u)
    v, u = v / nrm, u / nrm
    v_old, u_old, beta = np.zeros(n), np.zeros(n), 0.0
    al, be = [], []
    for k in range(min(steps, n)):
        w = apply_blocks(B, u)                        # B A v
        alpha = w @ u                                 # <BAv, v>_A
        w = w - alpha * v - beta * v_old
        z = spmv(A, w)
        beta_new = np.sqrt(max(w @ z, 0.0))
        al.append(alpha)
        if k == steps - 1 or beta_new <= 1e-14 * abs(alpha):
            break
        be.append(beta_new)
        v_old, u_old = v, u
        v, u = w / beta_new, z / beta_new
        beta = beta_new
    Tk = np.diag(al) + np.diag(be[:len(al) - 1], 1) + np.diag(be[:len(al) - 1], -1)
    return float(np.linalg.eigvalsh(Tk)[-1])


def omega(lam_lanczos: float) -> float:
    return OMEGA_NUM / (LANCZOS_SAFETY * lam_lanczos)


def init_params(seed: int) -> np.ndarray:
    """He-normal weights, zero biases (a reference initialisation for tests)."""
    rng = np.random.default_rng(seed)
    p = {}
    for name, shape in SHAPES:
        if name.startswith("W"):
            p[name] = rng.normal(size=shape) * np.sqrt(2.0 / shape[1])
        else:
            p[name] = np.zeros(shape)
    return pack(p)
