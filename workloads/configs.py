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
