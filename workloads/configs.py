"""The five seeded synthetic workloads (elasticity on structured perturbed meshes).

They stand in for the paper's Netgen meshes (Sec. 7, "Numerical Results"),
which are not available: same operator (P1 linear elasticity, Problem
"epseps"), clamped face, constant or jumping coefficients.

* ``square32``  2D unit square, 33x33 vertices (32x32 cells), E=1, nu=0.3,
  body force (0,-1), seed 1 -> 1,056 free vertices, 2,112 dofs.
* ``cube64``    3D unit cube, 64^3 vertices, E=1, nu=0.3, body force (0,0,-1),
  seed 2 -> 258,048 free vertices, 774,144 dofs.
* ``cube128jump`` 3D unit cube, 128^3 vertices, 200 inclusion boxes with
  E = 10**U(-3,3), nu per element U[0.25,0.45], seed 3 -> 6.24M dofs.
* ``batch64``   64 independent boxes, vertices per axis U{16..48}, h = 1/32,
  E ~ U[0.1,10], nu ~ U[0.2,0.4] per system, 6 load cases (+-x,+-y,+-z unit
  body forces), seed 4.
* ``cube96nu``  3D unit cube, 96^3 vertices, E=1, nu per element U[0.3,0.45],
  seed 5; the learned smoother trains on ten 32^3 meshes (seeds 100..109).

The paper's own three workloads (Sec. 7), on structured perturbed meshes:

* ``beam``      the vector model problem: the beam [0,10] x [0,1]^2 clamped
  at x = 0 with mu = 1, lambda = 0 (E = 1, nu = 0 in the Hooke law
  2 mu eps:eps + lambda div div, whose 2 mu is the paper's mu); default
  h = 1/32 -> 321 x 33 x 33 vertices, 348,480 free, 1.05M dofs; seed 6.
* ``jump11``    the difficult vector problem: the unit cube clamped at x = 0,
  mu = lambda = 10^4 in the eleven diagonal boxes [(i-1)/11, i/11]^3 and
  mu = lambda = 1 elsewhere (nu = 1/3, E = 4/3 mu); default 67^3 vertices
  (six cells per box side), 296,274 free, 888,822 dofs; seed 7.
Body forces are not given in the paper; both use (0, 0, -1).
* ``poisson``   the scalar model problem: -Laplace u = 1 on the unit cube,
  u = 0 on the boundary; default 128^3 vertices (126^3 = 2,000,376
  unknowns); seed 8.
"""
from __future__ import annotations

import numpy as np

from .elasticity import make_problem

SIX_LOADS = np.array([[1, 0, 0], [-1, 0, 0], [0, 1, 0], [0, -1, 0], [0, 0, 1], [0, 0, -1]],
                     dtype=np.float64)


def square32(n: int = 33, seed: int = 1):
    return make_problem((n, n), seed=seed, E=1.0, nu=0.3, forces=[[0.0, -1.0]], name=f"square{n-1}")


def cube(n: int = 64, seed: int = 2):
    return make_problem((n, n, n), seed=seed, E=1.0, nu=0.3, forces=[[0.0, 0.0, -1.0]],
                        name=f"cube{n}")


def cube64():
    return cube(64, 2)


def cube128jump(n: int = 128, seed: int = 3):
    return make_problem((n, n, n), seed=seed, forces=[[0.0, 0.0, -1.0]], jump_boxes=200,
                        nu_range=(0.25, 0.45), name=f"cube{n}jump")


def batch_specs(n_systems: int = 64, seed: int = 4, lo: int = 16, hi: int = 48):
    """Per-system (shape, E, nu, seed) of the batched workload."""
    rng = np.random.default_rng(seed)
    shapes = rng.integers(lo, hi + 1, size=(n_systems, 3))
    Es = rng.uniform(0.1, 10.0, size=n_systems)
    nus = rng.uniform(0.2, 0.4, size=n_systems)
    return [(tuple(int(v) for v in shapes[i]), float(Es[i]), float(nus[i]), 1000 * seed + i)
            for i in range(n_systems)]


def batch_problem(spec):
    shape, E, nu, s = spec
    return make_problem(shape, seed=s, h=1.0 / 32, E=E, nu=nu, forces=SIX_LOADS,
                        name=f"box{shape[0]}x{shape[1]}x{shape[2]}")


def cube96nu(n: int = 96, seed: int = 5):
    return make_problem((n, n, n), seed=seed, E=1.0, forces=[[0.0, 0.0, -1.0]],
                        nu_range=(0.3, 0.45), name=f"cube{n}nu")


def training_meshes(n: int = 32, seeds=range(100, 110)):
    return [make_problem((n, n, n), seed=s, E=1.0, forces=[[0.0, 0.0, -1.0]],
                         nu_range=(0.3, 0.45), name=f"train{n}_{s}") for s in seeds]


BEAM_LENGTH = 10


def beam(m: int = 32, seed: int = 6):
    """The beam [0,10] x [0,1]^2 with h = 1/m (10m+1 x m+1 x m+1 vertices)."""
    return make_problem((BEAM_LENGTH * m + 1, m + 1, m + 1), seed=seed, h=1.0 / m, E=1.0, nu=0.0,
                        forces=[[0.0, 0.0, -1.0]], name=f"beam{m}")


def jump11_modulus(c, mu_in=1e4, mu_out=1.0, nu=1.0 / 3.0, boxes=11):
    """E per element centroid c: mu_in inside the union of the boxes
    [(i-1)/boxes, i/boxes]^3, mu_out elsewhere, as E = mu (1 + nu)."""
    idx = np.floor(np.asarray(c) * boxes).clip(0, boxes - 1)
    inside = (idx[:, 0] == idx[:, 1]) & (idx[:, 1] == idx[:, 2])
    return np.where(inside, mu_in, mu_out) * (1.0 + nu)


def jump11(n: int = 67, seed: int = 7):
    """The difficult vector problem on n^3 vertices of the unit cube."""
    return make_problem((n, n, n), seed=seed, nu=1.0 / 3.0, forces=[[0.0, 0.0, -1.0]],
                        E_fn=jump11_modulus, name=f"jump11_{n}")


def poisson(n: int = 128, seed: int = 8):
    """The scalar model problem: -Laplace u = 1 on the unit cube with n^3
    vertices, u = 0 on the whole boundary ((n - 2)^3 unknowns)."""
    from .poisson import make_poisson
    return make_poisson((n, n, n), seed=seed, name=f"poisson{n}")


# Setup parameters the paper states per workload (Sec. 7); the rest are the
# defaults (5 passes on the first level and 4 later, caps 8 / 6 / 4).  The
# scalar problem: mu_s alone, 4 passes first and 3 later, every real-matrix
# row of P capped at 4 entries (the paper: 4 on the first three levels); its
# coarse size min(1600, n / 1250) is set where the problem size is known.
SETUP = {"jump11": {"passes_first": 4, "passes_later": 3},
         "poisson": {"scalar_only": True, "passes_first": 4, "passes_later": 3, "cap_S_first": 4,
                     "cap_S_later": 4}}


def coarse_size(name, n0):
    """The coarse size a workload's setup stops at (0: the library default)."""
    if name == "poisson":
        import math
        return min(1600, math.ceil(n0 / 1250))
    return 0
