"""Seeded scalar Poisson problems (the paper's scalar model problem, Sec. 2
Problem "gg" with beta = 0, and Sec. 7): -div(alpha grad u) = f on a box,
u = 0 on the whole boundary, P1 elements on the same structured, perturbed
meshes as the elasticity workloads (``workloads/elasticity``).

This is input generation only (no multigrid arithmetic).  For a simplex with
barycentric gradients g_a the element matrix is |T| alpha g_a . g_b; a
constant source f adds f |T| / (d + 1) per vertex.  The full matrix over all
vertices (1 x 1 blocks) and its restriction to the interior vertices are
returned, as for elasticity.
"""
from __future__ import annotations

from typing import Optional, Sequence

import numpy as np

from .elasticity import (BSR, Problem, _cells, _elements, _grid_coords, _lin, _pattern, _perturb,
                         _restrict)


def make_poisson(shape: Sequence[int], seed: int, h: Optional[float] = None, alpha: float = 1.0,
                 f: float = 1.0, name: str = "", amp: float = 0.2) -> Problem:
    """``amp``: amplitude of the coordinate perturbation in units of h (0:
    the plain grid)."""
    shape = tuple(int(s) for s in shape)
    d = len(shape)
    if h is None:
        h = 1.0 / (shape[0] - 1)
    rng = np.random.default_rng(seed)
    idx, coords = _grid_coords(shape, h)
    n_all = coords.shape[0]
    elements, temps, cells = _elements(shape)
    if amp > 0.0:
        coords = _perturb(idx, shape, h, coords, elements, rng, amp=amp)
    rowptr, colidx, offs, posmap = _pattern(shape, temps, n_all)
    off_index = {o: k for k, o in enumerate(offs)}
    acc = np.zeros(colidx.shape[0])
    rhs = np.zeros(n_all)
    n_cells = cells.shape[0]
    nv = d + 1
    for t in temps:
        vid = _lin(shape, cells[:, None, :] + t[None, :, :])        # (n_cells, nv)
        X = coords[vid]
        J = np.transpose(X[:, 1:, :] - X[:, :1, :], (0, 2, 1))
        vol = np.abs(np.linalg.det(J)) / (2.0 if d == 2 else 6.0)
        Jinv = np.linalg.inv(J)
        g = np.empty((n_cells, nv, d))
        g[:, 1:, :] = Jinv
        g[:, 0, :] = -Jinv.sum(axis=1)
        K = (alpha * vol)[:, None, None] * np.einsum("mad,mbd->mab", g, g)
        for a in range(nv):
            for b in range(nv):
                pos = posmap[vid[:, a], off_index[tuple(t[b] - t[a])]]
                acc += np.bincount(pos, weights=K[:, a, b], minlength=acc.shape[0])
        rhs += np.bincount(vid.ravel(), weights=np.repeat(f * vol / nv, nv), minlength=n_all)
    del posmap
    boundary = np.zeros(n_all, dtype=bool)
    for a in range(d):
        boundary |= (idx[:, a] == 0) | (idx[:, a] == shape[a] - 1)
    keep = ~boundary
    free = np.nonzero(keep)[0].astype(np.int64)
    vals = acc.reshape(-1, 1, 1)
    rp0, ci0, v0 = _restrict(rowptr, colidx, vals, keep)
    A_full = BSR(n_all, n_all, rowptr, colidx, vals)
    A = BSR(free.shape[0], free.shape[0], rp0, ci0, np.ascontiguousarray(v0))
    n_el = elements.shape[0]
    return Problem(dim=d, shape=shape, h=h, coords=coords, dirichlet=boundary, A_full=A_full,
                   free=free, A=A, b=rhs[free][None, :].copy(), elements=elements,
                   E_el=np.full(n_el, alpha), nu_el=np.zeros(n_el), name=name, dofs=1)
