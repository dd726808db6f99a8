"""Solve phase: BSR products, Galerkin, block-l1 smoother, coarsest solve,
V-cycle and PCG.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

* Two-grid / V-cycle: Algorithm tg of Sec. 3 (pre-smoothing, coarse-grid
  correction with P and P^T, post-smoothing with M^T = M), applied
  recursively; the coarse system of level l+1 is the Galerkin product
  A_{l+1} = P_l^T A_l P_l (Sec. 3 and Sec. 6).
* Smoother: block version of the l1 smoother (Sec. 7): blocks are the dofs
  of one vertex, M_v = A_vv + diag(sum of |a_rc| over the columns c outside
  the block), applied as block Jacobi; singular M_v are pseudo-inverted
  (Sec. 3 after Lemma eet_is_diag, "pseudo smoother").  The other form of
  the l1 smoothers the paper cites, hybrid Gauss-Seidel, is read for one
  device as block Gauss-Seidel over the colour classes of a distance-1
  colouring (a class plays the part of a processor's block; the l1 term
  covers couplings inside a class, of which a distance-1 colouring has
  none): forward sweep before, backward sweep after the coarse correction.
* Coarsest level: A_L + (I - E_L E_L^T) with E_L spanning the orthogonal
  complement of the kernels of the diagonal blocks (Lemma eet_is_diag and
  the regularisation identity of Sec. 3 after Lemma eet_is_diag), solved by Cholesky.
* PCG with one V-cycle as preconditioner (Sec. 7).
"""
from __future__ import annotations

import dataclasses
from typing import List

import numpy as np
import scipy.linalg as sla
import scipy.sparse as sp

from .criteria import pinv_sym

KERNEL_RTOL = 1e-12


@dataclasses.dataclass
class Mat:
    """BSR matrix in plain arrays."""

    n_rows: int
    n_cols: int
    rowptr: np.ndarray
    colidx: np.ndarray
    vals: np.ndarray            # (nnzb, br, bc)

    @property
    def br(self):
        return int(self.vals.shape[1])

    @property
    def bc(self):
        return int(self.vals.shape[2])

    @property
    def nnzb(self):
        return int(self.colidx.shape[0])

    def scipy(self):
        return sp.bsr_matrix((self.vals, self.colidx, self.rowptr),
                             shape=(self.n_rows * self.br, self.n_cols * self.bc)).tocsr()

    def block(self, i, j):
        s, e = self.rowptr[i], self.rowptr[i + 1]
        hit = np.nonzero(self.colidx[s:e] == j)[0]
        if hit.size == 0:
            return None
        return self.vals[s + hit[0]]


def mat_from(obj) -> Mat:
    return Mat(int(obj.n_rows), int(obj.n_cols), np.asarray(obj.rowptr), np.asarray(obj.colidx),
               np.asarray(obj.vals, dtype=np.float64))


def spmv(A: Mat, x):
    """y_i = sum_j A_ij x_j."""
    return A.scipy() @ x


def transpose(P: Mat) -> Mat:
    """Explicit block transpose R = P^T with sorted columns."""
    rows = np.repeat(np.arange(P.n_rows), np.diff(P.rowptr))
    order = np.lexsort((rows, P.colidx))
    cnt = np.bincount(P.colidx, minlength=P.n_cols)
    rp = np.zeros(P.n_cols + 1, dtype=np.int64)
    np.cumsum(cnt, out=rp[1:])
    return Mat(P.n_cols, P.n_rows, rp, rows[order].astype(np.int64),
               np.ascontiguousarray(np.transpose(P.vals[order], (0, 2, 1))))


def galerkin(P: Mat, A: Mat) -> Mat:
    """A_c = P^T A P with the structural block pattern (no dropping).

    The pattern is the product of the 0/1 block patterns (all block pairs
    that meet, numerically zero or not); values come from the sparse product.
    """
    nf, nc = P.n_rows, P.n_cols
    Pp = sp.csr_matrix((np.ones(P.nnzb), P.colidx, P.rowptr), shape=(nf, nc))
    Ap = sp.csr_matrix((np.ones(A.nnzb), A.colidx, A.rowptr), shape=(nf, nf))
    S = (Pp.T @ Ap @ Pp).tocsr()
    S.sort_indices()
    Ps = P.scipy()
    C = (Ps.T @ A.scipy() @ Ps).tocsr()
    k = P.bc
    rows = np.repeat(np.arange(nc), np.diff(S.indptr))
    cols = S.indices.astype(np.int64)
    Cd = C.tocoo()
    # scatter the scalar entries into the structural blocks (sorted block keys)
    key_blocks = rows * nc + cols
    vals = np.zeros((cols.shape[0], k, k))
    crow = Cd.row.astype(np.int64) // k   # 64-bit keys: nc^2 exceeds 2^31 beyond 46,340 rows
    ccol = Cd.col.astype(np.int64) // k
    pos = np.searchsorted(key_blocks, crow * nc + ccol)
    vals[pos, Cd.row % k, Cd.col % k] = Cd.data
    return Mat(nc, nc, S.indptr.astype(np.int64), cols, vals)


def block_l1_inverse(A: Mat):
    """(M_v)^+ for every block row: M_v = A_vv + diag_r(sum_{c outside v} |a_rc|)."""
    n, k = A.n_rows, A.br
    rows = np.repeat(np.arange(n), np.diff(A.rowptr))
    diag = A.colidx == rows
    Mv = np.zeros((n, k, k))
    Mv[rows[diag]] = A.vals[diag]
    l1 = np.zeros((n, k))
    np.add.at(l1, rows[~diag], np.abs(A.vals[~diag]).sum(axis=2))
    Mv[:, np.arange(k), np.arange(k)] += l1
    return batched_pinv(Mv, KERNEL_RTOL)


def smallest_last_order(A: Mat):
    """Smallest-last order of the block graph of A (Matula and Beck):
    repeatedly remove a remaining block row of least degree among the
    remaining rows (ties: the smallest index); the order is the reverse of
    the removals."""
    import heapq
    n = A.n_rows
    deg = [int(np.sum(A.colidx[A.rowptr[i]:A.rowptr[i + 1]] != i)) for i in range(n)]
    heap = [(deg[i], i) for i in range(n)]
    heapq.heapify(heap)
    removed = [False] * n
    out = []
    while heap:
        d, i = heapq.heappop(heap)
        if removed[i] or d != deg[i]:
            continue
        removed[i] = True
        out.append(i)
        for j in A.colidx[A.rowptr[i]:A.rowptr[i + 1]].tolist():
            if j != i and not removed[j]:
                deg[j] -= 1
                heapq.heappush(heap, (deg[j], j))
    return out[::-1]


def greedy_colouring(A: Mat):
    """Distance-1 colouring of the block graph of A: block rows in
    smallest-last order, each takes the smallest colour that none of its
    already coloured neighbours holds.  Rows of one colour never couple."""
    n = A.n_rows
    col = -np.ones(n, dtype=np.int64)
    for i in smallest_last_order(A):
        nb = A.colidx[A.rowptr[i]:A.rowptr[i + 1]]
        used = set(col[nb].tolist())
        c = 0
        while c in used:
            c += 1
        col[i] = c
    return col


def hybrid_gs_inverse(A: Mat, colour):
    """(M_v)^+ of the block-l1 hybrid Gauss-Seidel smoother: M_v = A_vv +
    diag_r(sum of |a_rc| over the columns c of the other rows of v's own
    colour), the couplings a colour-parallel sweep treats Jacobi-wise; with a
    distance-1 colouring there are none and M_v = A_vv."""
    n, k = A.n_rows, A.br
    rows = np.repeat(np.arange(n), np.diff(A.rowptr))
    diag = A.colidx == rows
    Mv = np.zeros((n, k, k))
    Mv[rows[diag]] = A.vals[diag]
    same = (~diag) & (colour[A.colidx] == colour[rows])
    l1 = np.zeros((n, k))
    np.add.at(l1, rows[same], np.abs(A.vals[same]).sum(axis=2))
    Mv[:, np.arange(k), np.arange(k)] += l1
    return batched_pinv(Mv, KERNEL_RTOL)


def batched_pinv(B, rtol):
    """Symmetric pseudo-inverse of every block (eigenvalues <= rtol * max|w| dropped)."""
    w, V = np.linalg.eigh(0.5 * (B + np.transpose(B, (0, 2, 1))))
    wmax = np.abs(w).max(axis=1, keepdims=True)
    keep = w > rtol * wmax
    winv = np.where(keep, 1.0 / np.where(keep, w, 1.0), 0.0)
    return np.einsum("nik,nk,njk->nij", V, winv, V)


def block_apply(B, x):
    n, k, _ = B.shape
    return np.einsum("nij,nj->ni", B, x.reshape(n, k)).ravel()


def diag_kernels(A: Mat):
    """Orthonormal bases of ker(A_vv) per block (eigenvalues <= 1e-12 lambda_max)."""
    out = []
    for i in range(A.n_rows):
        Aii = A.block(i, i)
        w, V = np.linalg.eigh(0.5 * (Aii + Aii.T))
        wmax = np.max(np.abs(w))
        keep = w <= KERNEL_RTOL * wmax if wmax > 0 else np.ones_like(w, dtype=bool)
        out.append(V[:, keep])
    return out


def coarsest_matrix(A: Mat):
    """Dense A_L + (I - E_L E_L^T) (Sec. 3 after Lemma eet_is_diag)."""
    k = A.br
    Ad = A.scipy().toarray()
    for i, K in enumerate(diag_kernels(A)):
        Ad[i * k:(i + 1) * k, i * k:(i + 1) * k] += K @ K.T
    return Ad


@dataclasses.dataclass
class Hierarchy:
    A: List[Mat]
    P: List[Mat]
    R: List[Mat] = dataclasses.field(default_factory=list)
    Minv: list = dataclasses.field(default_factory=list)
    coarse_chol: object = None
    info: dict = dataclasses.field(default_factory=dict)
    smoother: str = "l1_jacobi"           # or "hybrid_gs"
    colour: list = dataclasses.field(default_factory=list)

    @property
    def n_levels(self):
        return len(self.A)


def prepare(A0: Mat, P: List[Mat], smoother: str = "l1_jacobi") -> Hierarchy:
    """Galerkin coarse matrices, explicit R = P^T, smoothers, coarsest factor.
    smoother: "l1_jacobi" (block-l1 Jacobi) or "hybrid_gs" (block-l1 hybrid
    Gauss-Seidel over the colour classes of greedy_colouring)."""
    A = [A0]
    for Pl in P:
        A.append(galerkin(Pl, A[-1]))
    H = Hierarchy(A=A, P=list(P), smoother=smoother)
    H.R = [transpose(Pl) for Pl in P]
    if smoother == "hybrid_gs":
        H.colour = [greedy_colouring(Al) for Al in A[:-1]]
        H.Minv = [hybrid_gs_inverse(Al, c) for Al, c in zip(A[:-1], H.colour)]
    elif smoother == "l1_jacobi":
        H.Minv = [block_l1_inverse(Al) for Al in A[:-1]]
    else:
        raise ValueError(f"unknown smoother {smoother}")
    H.coarse_chol = sla.cho_factor(coarsest_matrix(A[-1]), lower=True)
    return H


def smooth(A: Mat, Minv, b, x=None):
    """One block-l1 Jacobi sweep x <- x + M^+ (b - A x); from x = 0 it is M^+ b."""
    if x is None:
        return block_apply(Minv, b)
    return x + block_apply(Minv, b - spmv(A, x))


def gs_sweep(A: Mat, Minv, colour, b, x=None, forward=True):
    """One block-l1 hybrid Gauss-Seidel sweep: the colour classes in
    increasing (forward) or decreasing (backward) order; the rows of a class
    take x_v <- x_v + M_v^+ (b - A x)_v with x as updated by the classes
    before (Jacobi-wise inside a class).  x = None starts from x = 0."""
    n, k = A.n_rows, A.br
    x = np.zeros(n * k) if x is None else x.copy()
    As = A.scipy()
    ncol = int(colour.max()) + 1 if n else 0
    order = range(ncol) if forward else range(ncol - 1, -1, -1)
    for c in order:
        rows = np.nonzero(colour == c)[0]
        dofs = (rows[:, None] * k + np.arange(k)).ravel()
        r = (b[dofs] - As[dofs] @ x).reshape(-1, k)
        x[dofs] += np.einsum("nij,nj->ni", Minv[rows], r).ravel()
    return x


def coarse_solve(H: Hierarchy, b):
    return sla.cho_solve(H.coarse_chol, b)


def vcycle(H: Hierarchy, b, level=0):
    """One V-cycle: Algorithm tg applied recursively, one pre/post sweep."""
    if level == H.n_levels - 1:
        return coarse_solve(H, b)
    A, Minv = H.A[level], H.Minv[level]
    if H.smoother == "hybrid_gs":
        # forward sweep before, backward sweep after: the post-smoother is the
        # adjoint of the pre-smoother, so the V-cycle stays symmetric
        col = H.colour[level]
        x = gs_sweep(A, Minv, col, b, None, forward=True)
        bc = spmv(H.R[level], b - spmv(A, x))
        x = x + spmv(H.P[level], vcycle(H, bc, level + 1))
        return gs_sweep(A, Minv, col, b, x, forward=False)
    x = smooth(A, Minv, b)
    r = b - spmv(A, x)
    bc = spmv(H.R[level], r)
    ec = vcycle(H, bc, level + 1)
    x = x + spmv(H.P[level], ec)
    return smooth(A, Minv, b, x)


def pcg(H: Hierarchy, f, rtol=1e-8, maxit=500, x0=None, precond=None):
    """CG preconditioned by one V-cycle; stops when ||r||_2 <= rtol ||f||_2
    (recurrence residual).  Returns (x, iterations, relres history)."""
    A = H.A[0]
    B = precond if precond is not None else (lambda r: vcycle(H, r))
    x = np.zeros_like(f) if x0 is None else x0.copy()
    r = f - spmv(A, x)
    nf = np.linalg.norm(f)

    # relative residual; for f = 0 the stopping rule ||r|| <= rtol ||f||
    # asks for r = 0, and ||r|| itself is recorded
    def rel(r):
        return np.linalg.norm(r) / nf if nf > 0 else np.linalg.norm(r)

    def converged(h):
        return h <= rtol if nf > 0 else h <= 0.0

    hist = [rel(r)]
    if converged(hist[-1]):
        return x, 0, hist
    p = None
    rho_old = None
    it = 0
    while it < maxit:
        z = B(r)
        rho = float(r @ z)
        p = z.copy() if p is None else z + (rho / rho_old) * p
        q = spmv(A, p)
        alpha = rho / float(p @ q)
        x = x + alpha * p
        r = r - alpha * q
        rho_old = rho
        it += 1
        hist.append(rel(r))
        if converged(hist[-1]):
            break
    return x, it, hist


def two_grid_matrix(A: np.ndarray, Minv: np.ndarray, P: np.ndarray):
    """E_TG = (I - M^{-T} A)(I - P (P^T A P)^+ P^T A)(I - M^{-1} A) (Sec. 3)."""
    n = A.shape[0]
    I = np.eye(n)
    Ac = P.T @ A @ P
    CG = I - P @ pinv_sym(Ac) @ P.T @ A
    return (I - Minv.T @ A) @ CG @ (I - Minv @ A)


def block_diag_dense(B):
    n, k, _ = B.shape
    out = np.zeros((n * k, n * k))
    for i in range(n):
        out[i * k:(i + 1) * k, i * k:(i + 1) * k] = B[i]
    return out


def two_grid_apply(A, Minv, P, Ac_pinv, x):
    """Error propagation of one step of Algorithm tg (b = 0) on a vector."""
    x = x - Minv @ (A @ x)
    x = x - P @ (Ac_pinv @ (P.T @ (A @ x)))
    return x - Minv.T @ (A @ x)


def spectral_radius_power(apply, n, iters=400, seed=0):
    """Power iteration for rho of a linear map (dominant real eigenvalue)."""
    rng = np.random.default_rng(seed)
    x = rng.normal(size=n)
    x /= np.linalg.norm(x)
    lam = 0.0
    for _ in range(iters):
        y = apply(x)
        lam = np.linalg.norm(y)
        if lam == 0.0:
            return 0.0
        x = y / lam
    return float(lam)
