"""Auxiliary topology: kernel transfer matrices, edge/vertex matrices, A-hat.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

Follows Sec. 3 (rigid-body modes, eq. (qij_epseps)), Sec. 4 Def. deng
(eq. (auxa)), Thm. deng_elast with the Remark on c^{ij}, and Thm. cemats.
Notation: d = spatial dimension, k = d + d(d-1)/2 dofs per vertex of the
auxiliary topology (3 in 2D, 6 in 3D).
"""
from __future__ import annotations

import dataclasses

import numpy as np


def kdim(d: int) -> int:
    """Number of rigid-body modes in dimension d (Sec. 3, k = d + d(d-1)/2)."""
    return d + d * (d - 1) // 2


def skew(t) -> np.ndarray:
    """Skew(t) of Sec. 3: the d x (k-d) matrix with u(x) = d + Skew(x) r.

    2D: (-t_1, t_0)^T.  3D: the cross-product matrix, Skew(t) r = t x r
    (the paper's 1-based t_1..t_3 are read as t_0..t_2).
    """
    t = np.asarray(t, dtype=np.float64)
    if t.shape[0] == 1:
        # the scalar problem (k = kdim(1) = 1): no rotations, Q = 1
        return np.zeros((1, 0))
    if t.shape[0] == 2:
        return np.array([[-t[1]], [t[0]]])
    return np.array([[0.0, -t[2], t[1]],
                     [t[2], 0.0, -t[0]],
                     [-t[1], t[0], 0.0]])


def Q(t) -> np.ndarray:
    """[[I, Skew(t)], [0, I]]: change of rigid-mode coordinates by a shift t.

    Q^{v_i -> v_j} = Q(x_j - x_i) (eq. (qij_epseps)); Q^{ij} = Q(t^{ij}/2)
    (Remark after Def. deng).
    """
    t = np.asarray(t, dtype=np.float64)
    d = t.shape[0]
    k = kdim(d)
    q = np.eye(k)
    q[:d, d:] = skew(t)
    return q


def Q_transfer(xi, xj) -> np.ndarray:
    """Q^{v_i -> v_j}: coordinates of a rigid mode at x_i -> at x_j."""
    return Q(np.asarray(xj) - np.asarray(xi))


def Q_half(xi, xj) -> np.ndarray:
    """Q^{ij} = sqrt(Q^{v_i -> v_j}): coordinates at x_i -> at the edge midpoint."""
    return Q(0.5 * (np.asarray(xj) - np.asarray(xi)))


@dataclasses.dataclass
class Topology:
    """Vertices, edges and the edge/vertex weight matrices of Def. deng."""

    pos: np.ndarray           # (n, d)
    edges: np.ndarray         # (m, 2) int, i < j
    E: np.ndarray             # (m, k, k) symmetric PSD edge weights
    M: np.ndarray             # (n, k, k) symmetric PSD vertex weights
    dirichlet: np.ndarray     # (n,) bool: Dirichlet vertices V_D

    @property
    def n(self) -> int:
        return int(self.pos.shape[0])

    @property
    def d(self) -> int:
        return int(self.pos.shape[1])

    @property
    def k(self) -> int:
        return kdim(self.d)

    def adjacency(self):
        """Neighbour lists {j: edge id} per vertex."""
        nb = [dict() for _ in range(self.n)]
        for e, (i, j) in enumerate(self.edges):
            nb[int(i)][int(j)] = e
            nb[int(j)][int(i)] = e
        return nb


def finest_topology(coords, A_rowptr, A_colidx, A_vals, dirichlet) -> Topology:
    """Finest-level edge matrices for elasticity (Thm. deng_elast + Remark).

    E^{ij} = c^{ij} [[t t^T, 0], [0, 0]] with t = x_j - x_i and
    c^{ij} = (1/d^2) sum_{l,m} |(A_ij)_{lm}| over the d x d block of the full
    (Neumann) matrix; M^i = 0 (beta = 0).  Every off-diagonal block of the
    full matrix is an edge, including edges to Dirichlet vertices.
    """
    coords = np.asarray(coords, dtype=np.float64)
    n, d = coords.shape
    k = kdim(d)
    rows = np.repeat(np.arange(n), np.diff(A_rowptr))
    upper = A_colidx > rows
    ei = rows[upper]
    ej = np.asarray(A_colidx)[upper]
    blocks = np.asarray(A_vals)[upper]
    c = np.abs(blocks).sum(axis=(1, 2)) / d ** 2
    t = coords[ej] - coords[ei]
    E = np.zeros((ei.shape[0], k, k))
    E[:, :d, :d] = c[:, None, None] * np.einsum("ma,mb->mab", t, t)
    M = np.zeros((n, k, k))
    return Topology(pos=coords, edges=np.stack([ei, ej], axis=1).astype(np.int64), E=E, M=M,
                    dirichlet=np.asarray(dirichlet, dtype=bool).copy())


def finest_topology_scalar(coords, A_rowptr, A_colidx, A_vals, dirichlet) -> Topology:
    """Finest-level edge and vertex weights of the scalar problem (Sec. 4,
    after Def. deng: E^{ij} = |A_ij|, M^i = max{0, A_ii - sum_{j != i} |A_ij|}
    over the full (Neumann) matrix, which split an M-matrix exactly).  The
    kernel transfers of the scalar problem are the identity (k = 1); the
    topology expresses this with one coordinate per vertex (kdim(1) = 1), the
    first one of the mesh."""
    coords = np.asarray(coords, dtype=np.float64)
    n = coords.shape[0]
    rows = np.repeat(np.arange(n), np.diff(A_rowptr))
    vals = np.asarray(A_vals, dtype=np.float64).reshape(-1)
    cols = np.asarray(A_colidx)
    upper = cols > rows
    off = cols != rows
    E = np.abs(vals[upper]).reshape(-1, 1, 1)
    diag = np.zeros(n)
    np.add.at(diag, rows[~off], vals[~off])
    absoff = np.zeros(n)
    np.add.at(absoff, rows[off], np.abs(vals[off]))
    M = np.maximum(0.0, diag - absoff).reshape(n, 1, 1)
    return Topology(pos=coords[:, :1].copy(), edges=np.stack([rows[upper], cols[upper]], axis=1).astype(np.int64),
                    E=E, M=M, dirichlet=np.asarray(dirichlet, dtype=bool).copy())


def edge_form(xi, xj, Eij):
    """The 2k x 2k matrix of ||Q^{ij} u_i - Q^{ji} u_j||^2_{E^{ij}} (eq. (deng))."""
    qij = Q_half(xi, xj)
    qji = Q_half(xj, xi)
    k = Eij.shape[0]
    F = np.zeros((2 * k, 2 * k))
    F[:k, :k] = qij.T @ Eij @ qij
    F[:k, k:] = -qij.T @ Eij @ qji
    F[k:, :k] = -qji.T @ Eij @ qij
    F[k:, k:] = qji.T @ Eij @ qji
    return F


def aux_diagonal(topo: Topology) -> np.ndarray:
    """Diagonal blocks D-hat_ii = M^i + sum_j Q^{ij,T} E^{ij} Q^{ij} of A-hat (eq. (auxa))."""
    D = topo.M.copy()
    for e, (i, j) in enumerate(topo.edges):
        qij = Q_half(topo.pos[i], topo.pos[j])
        qji = Q_half(topo.pos[j], topo.pos[i])
        D[i] += qij.T @ topo.E[e] @ qij
        D[j] += qji.T @ topo.E[e] @ qji
    return D


def aux_matrix_dense(topo: Topology) -> np.ndarray:
    """Dense A-hat of eq. (auxa) (small topologies only)."""
    n, k = topo.n, topo.k
    A = np.zeros((n * k, n * k))
    for i in range(n):
        A[i * k:(i + 1) * k, i * k:(i + 1) * k] += topo.M[i]
    for e, (i, j) in enumerate(topo.edges):
        qij = Q_half(topo.pos[i], topo.pos[j])
        qji = Q_half(topo.pos[j], topo.pos[i])
        Ee = topo.E[e]
        A[i * k:(i + 1) * k, i * k:(i + 1) * k] += qij.T @ Ee @ qij
        A[j * k:(j + 1) * k, j * k:(j + 1) * k] += qji.T @ Ee @ qji
        A[i * k:(i + 1) * k, j * k:(j + 1) * k] -= qij.T @ Ee @ qji
        A[j * k:(j + 1) * k, i * k:(i + 1) * k] -= qji.T @ Ee @ qij
    return A


def coarse_topology(topo: Topology, agg: np.ndarray, n_c: int, xc: np.ndarray,
                    use_dirichlet: bool = True) -> Topology:
    """Coarse edge and vertex matrices of Thm. cemats.

    ``agg[i]`` is the coarse vertex I of fine vertex i, or -1 for i in D.
    E^{IJ} = sum_{i in C_I, j in C_J} Q^{IJ->ij,T} E^{ij} Q^{IJ->ij} with
    Q^{IJ->ij} = Q^{ij} Q^{v_I->v_i} Q^{JI};
    M^I = sum_{i in C_I} Q^{v_I->v_i,T} (M^i + sum_{j in D} Q^{ij,T} E^{ij} Q^{ij}) Q^{v_I->v_i}.
    Edges inside one agglomerate drop out; edges between two D vertices too.
    ``use_dirichlet=False`` ignores edges to D (later passes of Algorithm 1
    have no D vertices left).
    """
    k = topo.k
    M = np.zeros((n_c, k, k))
    for i in range(topo.n):
        I = agg[i]
        if I >= 0:
            q = Q_transfer(xc[I], topo.pos[i])
            M[I] += q.T @ topo.M[i] @ q
    coarse = {}
    for e, (i, j) in enumerate(topo.edges):
        I, J = int(agg[i]), int(agg[j])
        Ee = topo.E[e]
        if I >= 0 and J >= 0:
            if I == J:
                continue
            a, b, ia, jb = (I, J, i, j) if I < J else (J, I, j, i)
            qhalf = Q_half(topo.pos[ia], topo.pos[jb])              # Q^{ij}
            q_Ii = Q_transfer(xc[a], topo.pos[ia])                   # Q^{v_I -> v_i}
            q_JI = Q_half(xc[b], xc[a])                              # Q^{JI}
            qt = qhalf @ q_Ii @ q_JI                                 # Q^{IJ -> ij}
            contrib = qt.T @ Ee @ qt
            if (a, b) in coarse:
                coarse[(a, b)] += contrib
            else:
                coarse[(a, b)] = contrib.copy()
        elif use_dirichlet and (I >= 0) != (J >= 0):
            ia, jd, I0 = (i, j, I) if I >= 0 else (j, i, J)
            qh = Q_half(topo.pos[ia], topo.pos[jd])                  # Q^{ij}, j in D
            q_Ii = Q_transfer(xc[I0], topo.pos[ia])
            M[I0] += q_Ii.T @ (qh.T @ Ee @ qh) @ q_Ii
    keys = sorted(coarse.keys())
    edges = np.array(keys, dtype=np.int64).reshape(-1, 2)
    E = np.array([coarse[key] for key in keys]).reshape(-1, k, k)
    return Topology(pos=np.asarray(xc, dtype=np.float64), edges=edges, E=E, M=M,
                    dirichlet=np.zeros(n_c, dtype=bool))


def rigid_modes(pos: np.ndarray, with_rotations: bool) -> np.ndarray:
    """Rigid-body modes u(x) = d + Skew(x) r sampled at the vertices.

    Returns (n*k_v, k) with k_v = k (displacement + rotation coordinates per
    vertex, the nodal representation of eq. (qij_epseps)) or k_v = d.
    """
    pos = np.asarray(pos, dtype=np.float64)
    n, d = pos.shape
    k = kdim(d)
    kv = k if with_rotations else d
    W = np.zeros((n, kv, k))
    for i in range(n):
        W[i, :d, :d] = np.eye(d)
        W[i, :d, d:] = skew(pos[i])
        if with_rotations:
            W[i, d:, d:] = np.eye(k - d)
    return W.reshape(n * kv, k)
