"""Algorithm 1 (successive matching) of Sec. 5.2.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

Readings of gaps in the printed algorithm (the same readings the CUDA
library's host setup implements):
* the initial agglomerates are the singletons of V \\ D (the listing's
  "C \\ D" is read as V \\ D) and the first-pass branch tests k == 1;
* candidates are unmatched neighbours (tr E^{IJ} > 0) with mu_s < sigma;
  the one with minimal mu_s is tried first (R = 1), ties broken by the
  iteration order; it is accepted if mu_p < sigma and, when the union holds
  more than two vertices of the level, mu_g^delta(union) < sigma (mu_g is
  evaluated with the level's own edge/vertex matrices);
* pass 1 visits vertices in Cuthill-McKee order (start: non-D vertex of
  minimal degree, lowest id; neighbours by increasing degree, then id);
  later passes visit the previous pass's agglomerates in reverse insertion
  order (pairs in the order they were formed, then singletons);
* coarse vertices sit at the centroid of their agglomerate (Remark after
  Def. pwp); coarse E/M of every pass follow Thm. cemats (pass 1 folds edges
  to D into M).
"""
from __future__ import annotations

import dataclasses

import numpy as np

from .criteria import mu_D, mu_g, mu_p, mu_s, trace_max
from .topology import Topology, aux_diagonal, coarse_topology


@dataclasses.dataclass
class CoarsenParams:
    sigma: float = 30.0
    delta: int = 1
    passes: int = 5
    # True: the comparison variant of Sec. 5's coefficient-jump figures, in
    # which only the scalar measure mu_s is used (mu_p and mu_g are not
    # computed; the first candidate is taken)
    scalar_only: bool = False


def cuthill_mckee(topo: Topology, active: np.ndarray):
    """Cuthill-McKee order of the active vertices of the edge graph."""
    nbrs = [[] for _ in range(topo.n)]
    for i, j in topo.edges:
        if active[i] and active[j]:
            nbrs[i].append(int(j))
            nbrs[j].append(int(i))
    deg = np.array([len(a) for a in nbrs])
    seen = ~np.asarray(active, dtype=bool).copy()
    order = []
    while True:
        cand = np.nonzero(~seen)[0]
        if cand.size == 0:
            break
        start = int(cand[np.lexsort((cand, deg[cand]))[0]])
        seen[start] = True
        queue = [start]
        head = 0
        while head < len(queue):
            v = queue[head]
            head += 1
            order.append(v)
            for w in sorted(nbrs[v], key=lambda u: (deg[u], u)):
                if not seen[w]:
                    seen[w] = True
                    queue.append(w)
    return order


def later_pass_order(m):
    """Visiting order of passes 2, 3, ...: the previous pass's m agglomerates
    (numbered pairs first, in the order they were formed, then singletons)
    in reverse insertion order."""
    return list(range(m - 1, -1, -1))


def _match(Tc: Topology, order, sizes, members, level_topo, level_Dhat, level_nbrs, p):
    """One round of matching (procedure match_vertices)."""
    nbrs = Tc.adjacency()
    Dhat = aux_diagonal(Tc)
    tmax = trace_max(Tc, nbrs)
    rank = {v: r for r, v in enumerate(order)}
    inT = np.zeros(Tc.n, dtype=bool)
    inT[list(order)] = True
    pairs, singles = [], []
    for ci in order:
        if not inT[ci]:
            continue
        inT[ci] = False
        Ns = []
        for cj, e in nbrs[ci].items():
            if inT[cj]:
                m = mu_s(tmax, np.trace(Tc.E[e]), ci, cj)
                if m < p.sigma:
                    Ns.append((m, rank[cj], cj))
        matched = False
        if p.scalar_only and Ns:
            Ns.sort()
            pairs.append((ci, Ns[0][2]))
            inT[Ns[0][2]] = False
            continue
        while Ns:
            Ns.sort()
            _, _, cj = Ns.pop(0)
            mu = mu_p(Tc, Dhat, nbrs, ci, cj, p.delta)
            if mu < p.sigma:
                if sizes[ci] + sizes[cj] == 2:
                    ok = True
                else:
                    union = members[ci] + members[cj]
                    ok = mu_g(level_topo, level_Dhat, level_nbrs, union, p.delta) < p.sigma
                if ok:
                    pairs.append((ci, cj))
                    inT[cj] = False
                    matched = True
                    break
        if not matched:
            singles.append((ci,))
    return pairs + singles


def successive_matching(topo: Topology, p: CoarsenParams = CoarsenParams()):
    """Algorithm 1: agglomerates of the vertices of one level.

    Returns ``agg`` ((n,) coarse id or -1 for D), ``n_c``, the coarse
    positions (centroids) and the coarse topology (Thm. cemats).
    """
    n = topo.n
    nbrs0 = topo.adjacency()
    Dhat0 = aux_diagonal(topo)
    D = topo.dirichlet.copy()
    for v in range(n):
        if not D[v] and mu_D(Dhat0[v], topo.M[v]) < p.sigma:
            D[v] = True
    active = ~D
    order = cuthill_mckee(topo, active)
    # pass 1 works on the level's own graph (D vertices present, not matchable)
    Tc = topo
    members = {v: [v] for v in range(n)}
    sizes = {v: 1 for v in range(n)}
    for k in range(1, p.passes + 1):
        groups = _match(Tc, order, sizes, members, topo, Dhat0, nbrs0, p)
        new_members = [sum((members[c] for c in g), []) for g in groups]
        m = len(groups)
        cagg = -np.ones(Tc.n, dtype=np.int64)
        for gi, g in enumerate(groups):
            for c in g:
                cagg[c] = gi
        xc = np.array([topo.pos[mem].mean(axis=0) for mem in new_members]).reshape(m, topo.d)
        Tc = coarse_topology(Tc, cagg, m, xc, use_dirichlet=(k == 1))
        members = {gi: mem for gi, mem in enumerate(new_members)}
        sizes = {gi: len(mem) for gi, mem in enumerate(new_members)}
        order = later_pass_order(m)
    agg = -np.ones(n, dtype=np.int64)
    for gi, mem in members.items():
        agg[mem] = gi
    return agg, len(members), Tc.pos.copy(), Tc, D
