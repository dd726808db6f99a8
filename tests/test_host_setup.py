"""The library's host setup code (csrc/setup_host.cpp: edge matrices,
Algorithm 1, coarse edge/vertex matrices, tentative and auxiliary smoothed
prolongation) against the oracle's setup, on the CPU: the C++ is compiled
with g++ into a small driver (tests/host_setup_harness.cpp) that supplies the
coarse matrices from a plain host Galerkin product instead of the device
one.  Same levels, same prolongation patterns, values to 1e-10, and the
oracle's PCG with the library's prolongations converges in the oracle's
iteration count (+-1).  Run with 1 and 4 OpenMP threads: the setup's result
must not depend on the thread count."""
import os
import shutil
import subprocess

import numpy as np
import pytest

from oracle import hierarchy, solve
from workloads import configs, make_problem

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "..", "paper_2011_13325_gb300", "csrc")


def _checker(c, nb=4):
    """4 x 4 checkerboard of E = 10^4 and E = 1 boxes on the unit square."""
    i = np.floor(c[:, 0] * nb).clip(0, nb - 1)
    j = np.floor(c[:, 1] * nb).clip(0, nb - 1)
    return np.where((i + j) % 2 == 1, 1e4, 1.0)


CASES = {
    "square32": (lambda: configs.square32(), {}),
    "cube10": (lambda: make_problem((10, 10, 10), seed=2), {"coarse_max": 8}),
    "box_jump": (lambda: make_problem((9, 7, 8), seed=3, jump_boxes=6, nu_range=(0.25, 0.45)),
                 {"coarse_max": 6}),
    "rect2d_nu": (lambda: make_problem((41, 23), seed=9, nu_range=(0.3, 0.45)), {"coarse_max": 10}),
    "checker2d": (lambda: make_problem((17, 17), seed=1, nu=0.25, E_fn=_checker), {"coarse_max": 4}),
    "beam": (lambda: configs.beam(4), {"coarse_max": 8}),
    "jump11": (lambda: configs.jump11(12), {"coarse_max": 8, "passes_first": 4, "passes_later": 3}),
    # the scalar model problem with the paper's scalar parameters (mu_s alone,
    # 4 / 3 passes, real-row cap 4) and with the full criteria
    "poisson3d": (lambda: configs.poisson(14), dict(configs.SETUP["poisson"], coarse_max=12)),
    "poisson3d_full": (lambda: configs.poisson(12), {"coarse_max": 10}),
    "poisson2d": (lambda: __import__("workloads.poisson", fromlist=["x"]).make_poisson((23, 19), seed=5),
                  {"coarse_max": 6}),
}


@pytest.fixture(scope="module")
def harness(tmp_path_factory):
    gxx = shutil.which("g++")
    if gxx is None:
        pytest.skip("g++ not available")
    out = str(tmp_path_factory.mktemp("harness") / "host_setup_harness")
    cmd = [gxx, "-O2", "-std=c++17", "-fopenmp", "-I", CSRC, os.path.join(CSRC, "setup_host.cpp"),
           os.path.join(HERE, "host_setup_harness.cpp"), "-o", out]
    r = subprocess.run(cmd, capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    return out


def _write_problem(p, d):
    Af = p.A_full
    with open(os.path.join(d, "problem.bin"), "wb") as f:
        np.array([p.dim, p.coords.shape[0], Af.colidx.shape[0], getattr(p, "k", p.dim)],
                 dtype=np.int32).tofile(f)
        np.ascontiguousarray(p.coords, dtype=np.float64).tofile(f)
        np.ascontiguousarray(p.dirichlet, dtype=np.uint8).tofile(f)
        np.ascontiguousarray(Af.rowptr, dtype=np.int32).tofile(f)
        np.ascontiguousarray(Af.colidx, dtype=np.int32).tofile(f)
        np.ascontiguousarray(Af.vals, dtype=np.float64).tofile(f)


def _read_prolongations(d):
    raw = open(os.path.join(d, "P.bin"), "rb").read()
    pos = 0

    def take(dtype, n):
        nonlocal pos
        a = np.frombuffer(raw, dtype=dtype, count=n, offset=pos)
        pos += a.nbytes
        return a

    out = []
    for _ in range(int(take(np.int32, 1)[0])):
        nr, nc, br, bc, nnzb = (int(v) for v in take(np.int32, 5))
        rp = take(np.int32, nr + 1).astype(np.int64)
        ci = take(np.int32, nnzb).astype(np.int64)
        v = take(np.float64, nnzb * br * bc).reshape(nnzb, br, bc)
        out.append(solve.Mat(nr, nc, rp, ci, v.copy()))
    assert pos == len(raw)
    return out


_ORACLE = {}


def _oracle(name):
    if name not in _ORACLE:
        make, kw = CASES[name]
        p = make()
        _ORACLE[name] = (p, kw, hierarchy.setup(p, hierarchy.SetupParams(**kw)))
    return _ORACLE[name]


@pytest.mark.parametrize("threads", [1, 4])
@pytest.mark.parametrize("name", sorted(CASES))
def test_host_setup_matches_oracle_setup(harness, tmp_path, name, threads):
    p, kw, H = _oracle(name)
    _write_problem(p, str(tmp_path))
    env = dict(os.environ, OMP_NUM_THREADS=str(threads))
    r = subprocess.run([harness, str(tmp_path), str(kw.get("coarse_max", 0)),
                        str(kw.get("passes_first", 5)), str(kw.get("passes_later", 4)),
                        str(int(kw.get("scalar_only", False))), str(kw.get("cap_S_first", 8)),
                        str(kw.get("cap_S_later", 6))],
                       capture_output=True,
                       text=True, env=env, timeout=300)
    assert r.returncode == 0, r.stderr
    Ps = _read_prolongations(str(tmp_path))
    assert len(Ps) + 1 == H.n_levels
    for l, (P, Po) in enumerate(zip(Ps, H.P)):
        assert (P.n_rows, P.n_cols, P.vals.shape[1:]) == (Po.n_rows, Po.n_cols, Po.vals.shape[1:]), l
        np.testing.assert_array_equal(P.rowptr, Po.rowptr)
        np.testing.assert_array_equal(P.colidx, Po.colidx)
        assert np.abs(P.vals - Po.vals).max() <= 1e-10 * np.abs(Po.vals).max(), l
    # the oracle's solver on the library's prolongations
    Hl = solve.prepare(solve.mat_from(p.A), Ps)
    f = p.b[0]
    _, it_lib, _ = solve.pcg(Hl, f, rtol=1e-8)
    _, it_or, _ = solve.pcg(H, f, rtol=1e-8)
    assert abs(it_lib - it_or) <= 1


def _colour_with_library(harness, d, A):
    with open(os.path.join(d, "pattern.bin"), "wb") as f:
        np.array([A.n_rows, A.colidx.shape[0]], dtype=np.int32).tofile(f)
        np.ascontiguousarray(A.rowptr, dtype=np.int32).tofile(f)
        np.ascontiguousarray(A.colidx, dtype=np.int32).tofile(f)
    r = subprocess.run([harness, "--colour", d], capture_output=True, text=True, timeout=120)
    assert r.returncode == 0, r.stderr
    raw = np.fromfile(os.path.join(d, "colour.bin"), dtype=np.int32)
    assert raw.shape[0] == A.n_rows + 1
    return int(raw[0]), raw[1:].astype(np.int64)


@pytest.mark.parametrize("name", ["cube10", "box_jump", "checker2d", "jump11", "poisson3d"])
def test_gs_colouring_matches_oracle_colouring(harness, tmp_path, name):
    """The hybrid Gauss-Seidel smoother's colouring in the library
    (smallest-last greedy order, ties by the smallest index) equals the
    oracle's on every level of the oracle's hierarchy, colour by colour, and
    is a distance-1 colouring: no two rows of one colour couple."""
    _, _, H = _oracle(name)
    for l, A in enumerate(H.A):
        n_col, col = _colour_with_library(harness, str(tmp_path), A)
        np.testing.assert_array_equal(col, solve.greedy_colouring(A), err_msg=f"level {l}")
        assert n_col == int(col.max()) + 1
        rows = np.repeat(np.arange(A.n_rows), np.diff(A.rowptr))
        off = A.colidx != rows
        assert not np.any(col[rows[off]] == col[A.colidx[off]]), l
