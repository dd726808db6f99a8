"""Agglomerate quality measures of Sec. 5.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

* ``mu_D``  eq. (mu_d): sup_v v^T D-hat_vv v / v^T M^v v.
* ``mu_g``  Thm. mu1 / eq. (mu_a) with delta in {0, 1}.
* ``mu_p``  Lemma mu2 / eq. (mub_ineq) with harmonic means H(A,B) = A(A+B)^+ B.
* ``mu_s``  Def. muc (trace-based scalar measure).

Generalised eigenvalue problems with a singular right-hand side are solved on
the range of the right-hand side (the smallest constant mu with
x^T L x <= mu x^T R x for all x); mu = +inf if L has energy on ker(R).
"""
from __future__ import annotations

import numpy as np

from .topology import Q, Q_half, Q_transfer, Topology

# relative thresholds: eigenvalues of R below RTOL_RANGE * lambda_max(R) form
# ker(R); energy of L on ker(R) above RTOL_LEAK * lambda_max(L) means mu = inf.
RTOL_PINV = 1e-12
RTOL_RANGE = 1e-10
RTOL_LEAK = 1e-8


def sym(A):
    return 0.5 * (A + A.T)


def pinv_sym(A, rtol=RTOL_PINV):
    """Pseudo-inverse of a symmetric PSD matrix by its eigen-decomposition."""
    w, V = np.linalg.eigh(sym(A))
    wmax = np.max(np.abs(w)) if w.size else 0.0
    if wmax <= 0.0:
        return np.zeros_like(A)
    keep = w > rtol * wmax
    return (V[:, keep] / w[keep]) @ V[:, keep].T


def harmonic(A, B):
    """H(A, B) = A (A + B)^+ B (Lemma mu2)."""
    return sym(A @ pinv_sym(A + B) @ B)


def gen_lambda_max(L, R):
    """Largest mu with L v = mu R v, i.e. the smallest mu with L <= mu R."""
    L = sym(L)
    R = sym(R)
    wl = np.linalg.eigvalsh(L)
    lmax = wl.max() if wl.size else 0.0
    if lmax <= 0.0:
        return 0.0
    wr, Vr = np.linalg.eigh(R)
    rmax = wr.max() if wr.size else 0.0
    if rmax <= 0.0:
        return np.inf
    rng = wr > RTOL_RANGE * rmax
    Vk = Vr[:, ~rng]
    if Vk.shape[1] > 0:
        leak = np.linalg.eigvalsh(Vk.T @ L @ Vk).max()
        if leak > RTOL_LEAK * lmax:
            return np.inf
    S = Vr[:, rng] / np.sqrt(wr[rng])
    return float(np.linalg.eigvalsh(S.T @ L @ S).max())


def mu_D(Dhat_v, M_v):
    """eq. (mu_d): Dirichlet-like measure of one vertex."""
    return gen_lambda_max(Dhat_v, M_v)


def trace_max(topo: Topology, nbrs):
    """max{tr M^i, max_{l != i} tr E^{il}} for every vertex (Def. muc)."""
    m = np.array([np.trace(topo.M[i]) for i in range(topo.n)])
    for i in range(topo.n):
        for l, e in nbrs[i].items():
            m[i] = max(m[i], np.trace(topo.E[e]))
    return m


def mu_s(tmax, trE_ij, i, j):
    """Def. muc: sqrt(max_i * max_j) / tr E^{ij}."""
    if trE_ij <= 0.0:
        return np.inf
    return float(np.sqrt(tmax[i] * tmax[j]) / trE_ij)


def mu_p(topo: Topology, Dhat, nbrs, i, j, delta=1):
    """Lemma mu2: pair measure mu_p^delta(v_i, v_j) as a k x k eigenproblem.

    Left: H(Q^{ji,T} D_ii Q^{ji}, Q^{ij,T} D_jj Q^{ij}).
    Right: E^{ij} + delta/2 sum_{l in N} Q^{ji,T} Q^{v_i->v_l,T}
           H(Q^{li,T} E^{il} Q^{li}, Q^{lj,T} E^{jl} Q^{lj}) Q^{v_i->v_l} Q^{ji},
    with N the neighbours common to v_i and v_j.
    """
    xi, xj = topo.pos[i], topo.pos[j]
    qji = Q_half(xj, xi)
    qij = Q_half(xi, xj)
    left = harmonic(qji.T @ Dhat[i] @ qji, qij.T @ Dhat[j] @ qij)
    right = topo.E[nbrs[i][j]].copy()
    if delta:
        common = set(nbrs[i].keys()) & set(nbrs[j].keys())
        for l in sorted(common):
            xl = topo.pos[l]
            qli = Q_half(xl, xi)
            qlj = Q_half(xl, xj)
            eil = qli.T @ topo.E[nbrs[i][l]] @ qli
            ejl = qlj.T @ topo.E[nbrs[j][l]] @ qlj
            T = Q_transfer(xi, xl) @ qji
            right += 0.5 * delta * (T.T @ harmonic(eil, ejl) @ T)
    return gen_lambda_max(left, right)


def mu_g_matrices(topo: Topology, Dhat, nbrs, C, delta=1):
    """Left and right matrices of eq. (mu_a) for one agglomerate C.

    Left: inf_w ||v_C - P_C w||^2_{D_C}
          = D_C - D_C P_C (P_C^T D_C P_C)^+ P_C^T D_C,
          P_C stacking Q^{v_H -> v_i} with v_H at the centroid.
    Right: sum_{i in C} M^i + the edges inside C (each edge once, as in
           eq. (auxa)) + delta/2 sum_{j not in C} of the Schur complement that
           eliminates w from sum_{i in C} ||Q^{ij} v_i - Q^{ji} w||^2_{E^{ij}}.
    """
    C = sorted(int(c) for c in C)
    k = topo.k
    loc = {v: a for a, v in enumerate(C)}
    nC = len(C)
    xH = topo.pos[C].mean(axis=0)
    PC = np.vstack([Q_transfer(xH, topo.pos[v]) for v in C])
    DC = np.zeros((nC * k, nC * k))
    for a, v in enumerate(C):
        DC[a * k:(a + 1) * k, a * k:(a + 1) * k] = Dhat[v]
    S = PC.T @ DC @ PC
    left = DC - DC @ PC @ pinv_sym(S) @ PC.T @ DC
    right = np.zeros((nC * k, nC * k))
    outside = {}
    for a, v in enumerate(C):
        right[a * k:(a + 1) * k, a * k:(a + 1) * k] += topo.M[v]
        for l, e in nbrs[v].items():
            if l in loc:
                if l > v:
                    b = loc[l]
                    qvl = Q_half(topo.pos[v], topo.pos[l])
                    qlv = Q_half(topo.pos[l], topo.pos[v])
                    Ee = topo.E[e]
                    right[a * k:(a + 1) * k, a * k:(a + 1) * k] += qvl.T @ Ee @ qvl
                    right[b * k:(b + 1) * k, b * k:(b + 1) * k] += qlv.T @ Ee @ qlv
                    right[a * k:(a + 1) * k, b * k:(b + 1) * k] -= qvl.T @ Ee @ qlv
                    right[b * k:(b + 1) * k, a * k:(a + 1) * k] -= qlv.T @ Ee @ qvl
            else:
                outside.setdefault(l, []).append((a, v, e))
    if delta:
        for l, lst in sorted(outside.items()):
            KCC = np.zeros((nC * k, nC * k))
            KCl = np.zeros((nC * k, k))
            Kll = np.zeros((k, k))
            for a, v, e in lst:
                qvl = Q_half(topo.pos[v], topo.pos[l])
                qlv = Q_half(topo.pos[l], topo.pos[v])
                Ee = topo.E[e]
                KCC[a * k:(a + 1) * k, a * k:(a + 1) * k] += qvl.T @ Ee @ qvl
                KCl[a * k:(a + 1) * k, :] -= qvl.T @ Ee @ qlv
                Kll += qlv.T @ Ee @ qlv
            right += 0.5 * delta * (KCC - KCl @ pinv_sym(Kll) @ KCl.T)
    return sym(left), sym(right)


def mu_g(topo: Topology, Dhat, nbrs, C, delta=1):
    """Thm. mu1: the smallest mu_g^delta(C) satisfying eq. (mu_a)."""
    left, right = mu_g_matrices(topo, Dhat, nbrs, C, delta)
    return gen_lambda_max(left, right)
