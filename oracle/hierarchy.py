"""Multi-level setup: auxiliary topology -> Algorithm 1 -> P_s -> Galerkin.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

Level loop (Sec. 5-6): finest edge matrices from the full matrix (Thm.
deng_elast), coarsen with Algorithm 1 (passes: 5 on the first level, 4
later, as for the paper's vector model problem), tentative P (Def. pwp /
pwp_el), auxiliary smoothed P_s (Def. aux_sp), A_{l+1} = P_s^T A_l P_s, coarse
edge/vertex matrices (Thm. cemats) for the next level.  Coarsening stops when
a level has at most ``coarse_max`` vertices (reading of the paper's "minimum
of 1000 and n/10^4": min(1000, max(64, ceil(n_0/10^4)))), when a level
shrinks by less than ``min_ratio`` or at ``max_levels``.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

from . import coarsening, prolongation, solve, topology


@dataclasses.dataclass
class SetupParams:
    sigma: float = 30.0
    delta: int = 1
    passes_first: int = 5
    passes_later: int = 4
    omega: float = 2.0 / 3.0
    cap_S_first: int = 8
    cap_S_later: int = 6
    cap_A: int = 4
    coarse_max: int = 0          # 0: min(1000, max(64, ceil(n0/1e4)))
    min_ratio: float = 1.5
    max_levels: int = 16
    scalar_only: bool = False    # Algorithm 1 with mu_s alone (Sec. 5 comparison)


def rows_as_dicts(M: solve.Mat):
    out = []
    for i in range(M.n_rows):
        s, e = M.rowptr[i], M.rowptr[i + 1]
        out.append({int(M.colidx[p]): M.vals[p] for p in range(s, e)})
    return out


def setup(problem, params: SetupParams = SetupParams(), factor: bool = True):
    """Build the hierarchy {A_l, P_l} of one ``workloads.Problem``.

    Returns a ``solve.Hierarchy`` with the per-level setup records in
    ``info``; ``factor=False`` skips smoothers and the coarsest Cholesky
    factor (for singular Neumann problems).
    """
    Af = problem.A_full
    if getattr(problem, "k", problem.dim) == 1:
        topo = topology.finest_topology_scalar(problem.coords, Af.rowptr, Af.colidx, Af.vals,
                                               problem.dirichlet)
    else:
        topo = topology.finest_topology(problem.coords, Af.rowptr, Af.colidx, Af.vals,
                                        problem.dirichlet)
    A = solve.mat_from(problem.A)
    rowmap = np.asarray(problem.free, dtype=np.int64)
    n0 = A.n_rows
    cmax = params.coarse_max or min(1000, max(64, math.ceil(n0 / 1e4)))
    # rows that are not kernel-exact on the finest level: clamped neighbours
    bad_exact = np.zeros(A.n_rows, dtype=bool)
    Ps, As, records = [], [A], []
    level = 0
    while A.n_rows > cmax and level + 1 < params.max_levels:
        first = level == 0
        cp = coarsening.CoarsenParams(sigma=params.sigma, delta=params.delta,
                                      passes=params.passes_first if first else params.passes_later,
                                      scalar_only=params.scalar_only)
        agg, n_c, xc, topo_c, D = coarsening.successive_matching(topo, cp)
        if n_c == 0 or A.n_rows < params.min_ratio * n_c:
            break
        # rows coupling to D (through the full graph on the first level)
        if first:
            adj_full = Af
            couples = np.zeros(A.n_rows, dtype=bool)
            for r, v in enumerate(rowmap):
                cols = adj_full.colidx[adj_full.rowptr[v]:adj_full.rowptr[v + 1]]
                couples[r] = bool(D[cols].any())
        else:
            couples = np.array([bool(D[rowmap[A.colidx[A.rowptr[r]:A.rowptr[r + 1]]]].any())
                                for r in range(A.n_rows)])
        bad = bad_exact | couples
        A_rows = rows_as_dicts(A)
        P_t = prolongation.tentative(topo, agg, xc, rowmap, first)
        pp = prolongation.ProlongParams(omega=params.omega, cap_S_first=params.cap_S_first,
                                        cap_S_later=params.cap_S_later, cap_A=params.cap_A)
        P_rows, kinds = prolongation.smoothed(A_rows, P_t, topo, agg, D, rowmap, bad, first, pp)
        br = topo.d if first else topo.k
        rp, ci, vals = prolongation.to_bsr(P_rows, n_c, br, topo.k)
        P = solve.Mat(A.n_rows, n_c, rp, ci, vals)
        # kernel-exactness of the next level's rows
        nxt_bad = np.zeros(n_c, dtype=bool)
        rows = np.repeat(np.arange(P.n_rows), np.diff(P.rowptr))
        np.logical_or.at(nxt_bad, P.colidx, bad[rows])
        A_next = solve.galerkin(P, A)
        records.append(dict(level=level, n=A.n_rows, n_c=n_c, agg=agg, D=D, kinds=kinds,
                            xc=xc, topo=topo, rowmap=rowmap, tentative=P_t))
        Ps.append(P)
        As.append(A_next)
        A = A_next
        topo = topo_c
        rowmap = np.arange(n_c, dtype=np.int64)
        bad_exact = nxt_bad
        level += 1
    if factor:
        H = solve.prepare(As[0], Ps)
    else:
        H = solve.Hierarchy(A=As, P=Ps, R=[solve.transpose(P) for P in Ps])
    H.info = dict(coarse_max=cmax, records=records)
    return H
