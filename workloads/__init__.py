"""Seeded synthetic elasticity workloads shared by the oracle and the GPU path."""
from .elasticity import BSR, Problem, make_problem  # noqa: F401
from . import configs  # noqa: F401
