"""Tentative and auxiliary smoothed prolongations (Sec. 3 Def. pwp / pwp_el,
Sec. 6 Def. aux_sp).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

Matrices here are lists of dicts ``rows[r] = {col: block}``; ``to_bsr``
turns them into sorted BSR arrays.

Readings of Def. aux_sp (shared with the CUDA library's host setup):
* omega = 2/3; (D-hat^0)^+ (pseudo-inverse) instead of the inverse;
* the filtered off-diagonal "M^{ij}" is read as E^{ij}, and the diagonal of an
  auxiliary row as sum_{l in F^i} Q^{il,T} E^{il} Q^{il} (the row-i form of
  eq. (auxa)); on the finest elasticity level the d x d form of Thm.
  deng_elast is used (Q = I, E = c t t^T);
* a vertex is "standard" (S, real matrix row) when its row of A touches at
  most cap_S distinct agglomerates (8 on the first level, 6 later), it does
  not couple to D, and its row is kernel-exact (it annihilates the rigid
  modes: on the first level, no clamped neighbour; on coarse levels, no
  inexact fine row in the support of its prolongation column);  otherwise it
  is "auxiliary" (A);
* F^i = the non-D edge neighbours whose agglomerates rank in the top
  cap_A = 4 by sum of tr E^{il}, the vertex's own agglomerate always kept.
"""
from __future__ import annotations

import dataclasses

import numpy as np

from .criteria import pinv_sym
from .topology import Q_half, Q_transfer, Topology, kdim


@dataclasses.dataclass
class ProlongParams:
    omega: float = 2.0 / 3.0
    cap_S_first: int = 8
    cap_S_later: int = 6
    cap_A: int = 4


def to_bsr(rows, n_cols, br, bc):
    rowptr = np.zeros(len(rows) + 1, dtype=np.int64)
    cols, vals = [], []
    for r, row in enumerate(rows):
        keys = sorted(row.keys())
        rowptr[r + 1] = rowptr[r] + len(keys)
        cols.extend(keys)
        vals.extend(row[c] for c in keys)
    vals = np.array(vals, dtype=np.float64).reshape(-1, br, bc)
    return rowptr, np.array(cols, dtype=np.int64), vals


def tentative(topo: Topology, agg, xc, rowmap, first_level: bool):
    """Def. pwp: P_{iJ} = Q^{v_J -> v_i} for i in C_J; on the finest elasticity
    level only the displacement rows (Def. pwp_el, P^f = R P)."""
    d = topo.d
    kr = d if first_level else kdim(d)
    rows = []
    for v in rowmap:
        J = int(agg[v])
        if J < 0:
            rows.append({})
        else:
            rows.append({J: Q_transfer(xc[J], topo.pos[v])[:kr, :].copy()})
    return rows


def smoothed(A_rows, P_rows, topo: Topology, agg, D, rowmap, bad, first_level: bool,
             pp: ProlongParams = ProlongParams()):
    """Def. aux_sp: P_s = (I - omega (D-hat^0)^+ A-hat^0) P.

    ``A_rows`` are the rows of the level matrix (dicts over row indices),
    ``rowmap[r]`` the topology vertex of row r, ``bad[r]`` marks rows that
    are not kernel-exact or couple to D.  Returns P_s rows and the per-row
    kind ('S', 'A' or 'D').
    """
    d = topo.d
    k = kdim(d)
    kr = d if first_level else k
    cap_S = pp.cap_S_first if first_level else pp.cap_S_later
    row_of = {int(v): r for r, v in enumerate(rowmap)}
    nbrs = topo.adjacency()
    out, kinds = [], []
    for r, v in enumerate(rowmap):
        v = int(v)
        if D[v]:
            out.append({})
            kinds.append("D")
            continue
        touched = {int(agg[rowmap[c]]) for c in A_rows[r] if not D[rowmap[c]]}
        if len(touched) <= cap_S and not bad[r]:
            kinds.append("S")
            Dinv = pinv_sym(A_rows[r][r])
            acc = {}
            for c, Ab in A_rows[r].items():
                for J, Pb in P_rows[c].items():
                    acc[J] = acc.get(J, 0.0) + Ab @ Pb
        else:
            kinds.append("A")
            weight = {}
            for l, e in nbrs[v].items():
                if D[l]:
                    continue
                J = int(agg[l])
                weight[J] = weight.get(J, 0.0) + np.trace(topo.E[e])
            own = int(agg[v])
            others = sorted((J for J in weight if J != own), key=lambda J: (-weight[J], J))
            keep = {own} | set(others[:pp.cap_A - 1])
            F = [l for l in sorted(nbrs[v]) if not D[l] and int(agg[l]) in keep]
            Ahat_ii = np.zeros((kr, kr))
            offd = []
            for l in F:
                Ee = topo.E[nbrs[v][l]]
                if first_level:
                    Ahat_ii += Ee[:d, :d]
                    offd.append((l, -Ee[:d, :d]))
                else:
                    qil = Q_half(topo.pos[v], topo.pos[l])
                    qli = Q_half(topo.pos[l], topo.pos[v])
                    Ahat_ii += qil.T @ Ee @ qil
                    offd.append((l, -qil.T @ Ee @ qli))
            Dinv = pinv_sym(Ahat_ii)
            acc = {}
            for J, Pb in P_rows[r].items():
                acc[J] = acc.get(J, 0.0) + Ahat_ii @ Pb
            for l, Ab in offd:
                for J, Pb in P_rows[row_of[l]].items():
                    acc[J] = acc.get(J, 0.0) + Ab @ Pb
        row = {J: (P_rows[r][J].copy() if J in P_rows[r] else np.zeros((kr, k)))
               for J in acc}
        for J in acc:
            row[J] = row[J] - pp.omega * (Dinv @ acc[J])
        out.append(row)
    return out, kinds
