"""Seeded synthetic P1 linear-elasticity problems on structured, perturbed meshes.

This module is the shared input generator.  It produces the linear system
A u = b of the paper's elasticity problem (Sec. 2, Problem "epseps",
eq. (lineq)/(auf)) on structured meshes that stand in for the paper's
unstructured Netgen meshes; it holds none of the multigrid method's arithmetic
(no edge matrices, coarsening, prolongation or solver).  Both the CPU oracle
and the GPU library consume what it returns.

Mesh recipe
-----------
* 2D: an ``nx x ny`` vertex grid on ``[0, (nx-1)h] x [0, (ny-1)h]``; each
  square is split by its SW->NE diagonal into two triangles.
* 3D: an ``nx x ny x nz`` vertex grid; each cube is split into the six
  Kuhn (Freudenthal) tetrahedra along its main diagonal.
* Every coordinate is perturbed by an independent uniform draw in
  ``[-0.2h, 0.2h]``; the normal component is not perturbed for vertices on a
  boundary face (the domain stays a box).  Elements whose Jacobian would be
  non-positive get the perturbation of their vertices halved until every
  element is positively oriented (deterministic).
* Vertex numbering: ``v = i + nx*(j + ny*k)``.  The face ``x = 0`` is
  clamped (Dirichlet), which removes all dofs of its vertices.

Assembly
--------
The bilinear form is the standard Hooke law
``a(u,v) = int 2 mu eps(u):eps(v) + lam div u div v`` with
``mu = E/(2(1+nu))`` and ``lam = E nu/((1+nu)(1-2nu))`` per element (the
paper writes ``mu eps:eps``; the factor 2 only rescales ``mu``).  For a simplex
with barycentric gradients ``g_a`` the ``d x d`` block coupling vertex ``a``
(test) and ``b`` (trial) is ``|T| (mu (g_a.g_b) I + mu g_b g_a^T + lam g_a g_b^T)``.
The right-hand side of a constant body force ``f`` is ``f |T|/(d+1)`` per
vertex and element.

The full (Neumann) matrix over all vertices is returned together with the
matrix restricted to free vertices (the Dirichlet elimination of Sec. 2,
eq. (auf)).
"""
from __future__ import annotations

import dataclasses
import itertools
from typing import Optional, Sequence

import numpy as np


@dataclasses.dataclass
class BSR:
    """Block-sparse-row matrix: ``rowptr`` (n+1), sorted ``colidx`` (nnzb),
    row-major blocks ``vals`` (nnzb, br, bc)."""

    n_rows: int
    n_cols: int
    rowptr: np.ndarray
    colidx: np.ndarray
    vals: np.ndarray

    @property
    def nnzb(self) -> int:
        return int(self.colidx.shape[0])

    @property
    def br(self) -> int:
        return int(self.vals.shape[1])

    @property
    def bc(self) -> int:
        return int(self.vals.shape[2])


@dataclasses.dataclass
class Problem:
    """One elasticity system ``A u = b`` on the free vertices of a mesh."""

    dim: int
    shape: tuple
    h: float
    coords: np.ndarray          # (n_all, dim) vertex positions
    dirichlet: np.ndarray       # (n_all,) bool, clamped vertices
    A_full: BSR                 # Neumann matrix over all vertices (dim x dim blocks)
    free: np.ndarray            # (n_free,) ids of the free vertices, ascending
    A: BSR                      # matrix on the free vertices (Dirichlet eliminated)
    b: np.ndarray               # (nrhs, n_free*dim) right-hand sides
    elements: np.ndarray        # (n_el, dim+1) vertex ids
    E_el: np.ndarray            # (n_el,) Young's modulus per element
    nu_el: np.ndarray           # (n_el,) Poisson ratio per element
    name: str = ""
    dofs: int = 0               # dofs per vertex: 0 means dim (elasticity), 1 scalar

    @property
    def k(self) -> int:
        """Dofs per vertex (block size of A)."""
        return self.dofs or self.dim

    @property
    def n_all(self) -> int:
        return int(self.coords.shape[0])

    @property
    def n_free(self) -> int:
        return int(self.free.shape[0])

    @property
    def ndof(self) -> int:
        return self.n_free * self.k


# --------------------------------------------------------------------------
# structured grids
# --------------------------------------------------------------------------

def _lin(shape, idx):
    """Linear vertex id of integer grid coordinates ``idx`` (..., dim)."""
    if len(shape) == 2:
        return idx[..., 0] + shape[0] * idx[..., 1]
    return idx[..., 0] + shape[0] * (idx[..., 1] + shape[1] * idx[..., 2])


def _simplex_templates(dim):
    """Corner offsets (in {0,1}^dim) of the simplices that split one cell.

    Every simplex is listed with positive orientation in the unperturbed grid.
    """
    if dim == 2:
        return [np.array([[0, 0], [1, 0], [1, 1]]), np.array([[0, 0], [1, 1], [0, 1]])]
    temps = []
    for perm in itertools.permutations(range(3)):
        path = [np.zeros(3, dtype=np.int64)]
        for ax in perm:
            nxt = path[-1].copy()
            nxt[ax] += 1
            path.append(nxt)
        t = np.array(path)
        J = (t[1:] - t[0]).T
        if np.linalg.det(J) < 0:
            t = t[[0, 1, 3, 2]]
        temps.append(t)
    return temps


def _cells(shape):
    """Integer corner (lower-left) coordinates of all cells, (n_cells, dim)."""
    rng = [np.arange(s - 1) for s in shape]
    grids = np.meshgrid(*rng, indexing="ij")
    # order cells like vertices: x fastest
    return np.stack([g.ravel(order="F") for g in grids], axis=1)


def _grid_coords(shape, h):
    rng = [np.arange(s) for s in shape]
    grids = np.meshgrid(*rng, indexing="ij")
    idx = np.stack([g.ravel(order="F") for g in grids], axis=1)
    return idx, idx.astype(np.float64) * h


def _elements(shape):
    cells = _cells(shape)
    temps = _simplex_templates(len(shape))
    els = [_lin(shape, cells[:, None, :] + t[None, :, :]) for t in temps]
    # element order: template-major
    return np.concatenate(els, axis=0).astype(np.int64), temps, cells


def _jacobians(coords, elements):
    X = coords[elements]                      # (n_el, d+1, d)
    J = np.transpose(X[:, 1:, :] - X[:, :1, :], (0, 2, 1))
    return J, np.linalg.det(J)


def _perturb(idx, shape, h, coords, elements, rng, amp=0.2):
    d = len(shape)
    delta = rng.uniform(-amp * h, amp * h, size=coords.shape)
    for a in range(d):
        on_face = (idx[:, a] == 0) | (idx[:, a] == shape[a] - 1)
        delta[on_face, a] = 0.0
    ref_vol = h ** d
    for _ in range(60):
        _, det = _jacobians(coords + delta, elements)
        bad = det <= 1e-3 * ref_vol
        if not bad.any():
            break
        verts = np.unique(elements[bad].ravel())
        delta[verts] *= 0.5
    else:  # pragma: no cover - 60 halvings always resolve it
        raise RuntimeError("mesh perturbation did not converge")
    return coords + delta


# --------------------------------------------------------------------------
# block pattern and assembly
# --------------------------------------------------------------------------

def _pattern(shape, temps, n_all):
    """BSR pattern of all vertex pairs that share a simplex.

    Columns come out sorted because the neighbour offsets are enumerated in
    increasing linear order.
    """
    d = len(shape)
    offs = set()
    for t in temps:
        for a in range(len(t)):
            for b in range(len(t)):
                offs.add(tuple(t[b] - t[a]))
    offs = sorted(offs, key=lambda o: _lin(shape, np.array(o)))
    lin_off = np.array([_lin(shape, np.array(o)) for o in offs], dtype=np.int64)
    idx, _ = _grid_coords(shape, 1.0)
    mask = np.zeros((len(offs), n_all), dtype=bool)
    cells = _cells(shape)
    for t in temps:
        for a in range(len(t)):
            for b in range(len(t)):
                o = tuple(t[b] - t[a])
                k = offs.index(o)
                mask[k, _lin(shape, cells + t[a])] = True
    mask_t = np.ascontiguousarray(mask.T)                     # (n_all, n_off)
    counts = mask_t.sum(axis=1)
    rowptr = np.zeros(n_all + 1, dtype=np.int64)
    np.cumsum(counts, out=rowptr[1:])
    u, k = np.nonzero(mask_t)
    colidx = (u + lin_off[k]).astype(np.int64)
    posmap = np.cumsum(mask_t, axis=1, dtype=np.int64) - 1 + rowptr[:-1, None]
    return rowptr, colidx, offs, posmap


def _lame(E, nu):
    mu = E / (2.0 * (1.0 + nu))
    lam = E * nu / ((1.0 + nu) * (1.0 - 2.0 * nu))
    return mu, lam


def _element_chunk(shape, coords, temps, cells, posmap, off_index, E_el, nu_el, c0, c1):
    """Element matrices of the cells c0..c1 (all templates): the BSR slot of
    every block contribution, the contributions, and the vertex ids and
    volumes for the right-hand side."""
    d = len(shape)
    n_cells = cells.shape[0]
    nv = d + 1
    eye = np.eye(d)
    cc = cells[c0:c1]
    all_pos, all_K, all_vid, all_fv = [], [], [], []
    for ti, t in enumerate(temps):
        vid = _lin(shape, cc[:, None, :] + t[None, :, :])          # (m, nv)
        el = ti * n_cells + np.arange(c0, c1)
        X = coords[vid]
        J = np.transpose(X[:, 1:, :] - X[:, :1, :], (0, 2, 1))
        det = np.linalg.det(J)
        Jinv = np.linalg.inv(J)
        g = np.empty((c1 - c0, nv, d))
        g[:, 1:, :] = Jinv
        g[:, 0, :] = -Jinv.sum(axis=1)
        vol = np.abs(det) / (2.0 if d == 2 else 6.0)
        mu, lam = _lame(E_el[el], nu_el[el])
        G = np.einsum("mad,mbd->mab", g, g)                           # g_a . g_b
        # K[m,a,b,i,j] = vol (mu G_ab d_ij + mu g_b,i g_a,j + lam g_a,i g_b,j)
        K = (mu * vol)[:, None, None, None, None] * (
            G[:, :, :, None, None] * eye[None, None, None]
            + np.einsum("mbi,maj->mabij", g, g))
        K += (lam * vol)[:, None, None, None, None] * np.einsum("mai,mbj->mabij", g, g)
        for a in range(nv):
            for b in range(nv):
                k = off_index[tuple(t[b] - t[a])]
                all_pos.append(posmap[vid[:, a], k])
                all_K.append(K[:, a, b].reshape(-1, d * d))
        all_vid.append(vid)
        all_fv.append(vol)
    return (np.concatenate(all_pos), np.concatenate(all_K, axis=0),
            np.concatenate(all_vid).ravel(), np.repeat(np.concatenate(all_fv) / (d + 1), nv))


def _assemble(shape, coords, temps, cells, rowptr, colidx, offs, posmap,
              E_el, nu_el, forces, chunk=60_000):
    """Assembled matrix values and right-hand sides.  Element matrices of
    several chunks are computed by a thread pool; their sums go into the
    matrix one chunk after another in cell order, so the result does not
    depend on the number of threads."""
    from concurrent.futures import ThreadPoolExecutor
    import os
    d = len(shape)
    nnzb = colidx.shape[0]
    n_all = coords.shape[0]
    acc = np.zeros((d * d, nnzb))
    nrhs = forces.shape[0]
    rhs = np.zeros((nrhs, d, n_all))
    n_cells = cells.shape[0]
    off_index = {o: k for k, o in enumerate(offs)}
    bounds = [(c0, min(n_cells, c0 + chunk)) for c0 in range(0, n_cells, chunk)]
    workers = max(1, min(8, os.cpu_count() or 1))
    with ThreadPoolExecutor(max_workers=workers) as ex:
        futs = []
        for b in bounds[:workers]:
            futs.append(ex.submit(_element_chunk, shape, coords, temps, cells, posmap, off_index,
                                  E_el, nu_el, *b))
        nxt = workers
        for i in range(len(bounds)):
            pos, Kc, vids, w = futs[i].result()
            futs[i] = None
            if nxt < len(bounds):
                futs.append(ex.submit(_element_chunk, shape, coords, temps, cells, posmap,
                                      off_index, E_el, nu_el, *bounds[nxt]))
                nxt += 1
            p0 = int(pos.min())
            span = int(pos.max()) - p0 + 1
            for e in range(d * d):
                acc[e, p0:p0 + span] += np.bincount(pos - p0, weights=Kc[:, e], minlength=span)
            for r in range(nrhs):
                for i_ in range(d):
                    if forces[r][i_] != 0.0:
                        rhs[r, i_] += forces[r][i_] * np.bincount(vids, weights=w, minlength=n_all)
    vals = np.ascontiguousarray(acc.T).reshape(nnzb, d, d)
    return vals, np.ascontiguousarray(np.transpose(rhs, (0, 2, 1)))


def _restrict(rowptr, colidx, vals, keep):
    """Rows/columns of the vertices flagged in ``keep`` (Dirichlet elimination)."""
    n_all = rowptr.shape[0] - 1
    newid = -np.ones(n_all, dtype=np.int64)
    newid[keep] = np.arange(int(keep.sum()))
    rows = np.repeat(np.arange(n_all), np.diff(rowptr))
    m = keep[rows] & keep[colidx]
    nr = newid[rows[m]]
    counts = np.bincount(nr, minlength=int(keep.sum()))
    rp = np.zeros(counts.shape[0] + 1, dtype=np.int64)
    np.cumsum(counts, out=rp[1:])
    return rp, newid[colidx[m]], vals[m]


# --------------------------------------------------------------------------
# public generator
# --------------------------------------------------------------------------

def make_problem(shape: Sequence[int], seed: int, h: Optional[float] = None,
                 E: float = 1.0, nu: float = 0.3, forces=None,
                 jump_boxes: int = 0, nu_range=None, name: str = "",
                 clamp: bool = True, E_fn=None) -> Problem:
    """Build one seeded elasticity problem.

    ``shape`` is the number of vertices per axis (2 or 3 entries).  ``h``
    defaults to ``1/(shape[0]-1)`` (unit square / cube).  ``forces`` is a
    list of constant body-force vectors (one right-hand side each).
    ``jump_boxes > 0`` draws that many axis-aligned inclusion boxes (centres
    uniform in the domain, side lengths uniform in [0.02, 0.2] of the domain,
    ``E = 10**U(-3, 3)``); the last box that contains an element's centroid
    sets its modulus, ``E`` elsewhere.  ``nu_range=(lo, hi)`` draws the
    Poisson ratio per element.  ``clamp=False`` keeps the pure Neumann
    problem (no Dirichlet vertices; A is then singular with the rigid-body
    modes as its kernel).  ``E_fn`` (optional) maps the element centroids
    (n_el x d) to the element moduli, replacing ``E`` and the boxes.
    """
    shape = tuple(int(s) for s in shape)
    d = len(shape)
    if h is None:
        h = 1.0 / (shape[0] - 1)
    rng = np.random.default_rng(seed)
    idx, coords = _grid_coords(shape, h)
    n_all = coords.shape[0]
    elements, temps, cells = _elements(shape)
    coords = _perturb(idx, shape, h, coords, elements, rng)
    n_el = elements.shape[0]
    E_el = np.full(n_el, float(E))
    nu_el = np.full(n_el, float(nu))
    if jump_boxes:
        brng = np.random.default_rng([seed, 1])
        ext = np.array([(s - 1) * h for s in shape])
        centres = brng.uniform(0.0, 1.0, size=(jump_boxes, d)) * ext
        sides = brng.uniform(0.02, 0.2, size=(jump_boxes, d)) * ext
        moduli = 10.0 ** brng.uniform(-3.0, 3.0, size=jump_boxes)
        cen = coords[elements].mean(axis=1)
        n_cells = cells.shape[0]
        cdims = [s - 1 for s in shape]
        for bi in range(jump_boxes):
            # an element's centroid lies within 0.2h of its cell, so only the
            # elements of cells overlapping the box (with a margin) can be
            # inside; the test itself is the same on those
            ranges = []
            for a in range(d):
                lo = int(np.floor((centres[bi][a] - 0.5 * sides[bi][a]) / h)) - 2
                hi = int(np.floor((centres[bi][a] + 0.5 * sides[bi][a]) / h)) + 2
                ranges.append(np.arange(max(lo, 0), min(hi, cdims[a] - 1) + 1))
            if any(r.size == 0 for r in ranges):
                continue
            g = np.meshgrid(*ranges, indexing="ij")
            cid = g[0].ravel()
            stride = 1
            for a in range(1, d):
                stride *= cdims[a - 1]
                cid = cid + stride * g[a].ravel()
            cand = (np.arange(len(temps))[:, None] * n_cells + cid[None, :]).ravel()
            inside = np.all(np.abs(cen[cand] - centres[bi]) <= 0.5 * sides[bi], axis=1)
            E_el[cand[inside]] = moduli[bi]
    if E_fn is not None:
        E_el = np.asarray(E_fn(coords[elements].mean(axis=1)), dtype=np.float64).reshape(n_el)
    if nu_range is not None:
        nrng = np.random.default_rng([seed, 2])
        nu_el = nrng.uniform(nu_range[0], nu_range[1], size=n_el)
    if forces is None:
        f = np.zeros(d)
        f[-1] = -1.0
        forces = [f]
    forces = np.asarray(forces, dtype=np.float64).reshape(-1, d)
    rowptr, colidx, offs, posmap = _pattern(shape, temps, n_all)
    vals, rhs = _assemble(shape, coords, temps, cells, rowptr, colidx, offs, posmap,
                          E_el, nu_el, forces)
    del posmap
    dirichlet = (idx[:, 0] == 0) if clamp else np.zeros(n_all, dtype=bool)
    keep = ~dirichlet
    free = np.nonzero(keep)[0].astype(np.int64)
    rp0, ci0, v0 = _restrict(rowptr, colidx, vals, keep)
    b = rhs[:, free, :].reshape(forces.shape[0], -1)
    A_full = BSR(n_all, n_all, rowptr, colidx, vals)
    A = BSR(free.shape[0], free.shape[0], rp0, ci0, np.ascontiguousarray(v0))
    return Problem(dim=d, shape=shape, h=h, coords=coords, dirichlet=dirichlet,
                   A_full=A_full, free=free, A=A, b=b, elements=elements,
                   E_el=E_el, nu_el=nu_el, name=name)
