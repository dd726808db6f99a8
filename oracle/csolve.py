"""The oracle's solve phase on many host cores: ``oracle/csolve.c`` (plain C,
FP64, OpenMP over rows) through ctypes.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

It computes what ``oracle/solve.py`` computes -- Galerkin products A_{l+1} =
P_l^T A_l P_l with the structural block pattern (Sec. 3, Sec. 6), the V-cycle
of Algorithm tg with the block-l1 Jacobi or the block-l1 hybrid Gauss-Seidel
smoother of Sec. 7 and the regularised coarsest solve of Sec. 3 after Lemma
eet_is_diag, and the PCG of Sec. 7 -- with the products written out as C
loops, so that the CPU baseline can use every host core.  The smoother
blocks, the colour classes, the explicit transposes and the coarsest
Cholesky factor come from ``oracle/solve.py`` itself.  Pinned
against ``oracle/solve.py`` (which is pinned against the paper) and by its
own closed-form checks in ``tests/test_oracle_csolve.py``.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

from . import solve

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "csolve.c")
LIB = os.path.join(HERE, "_build", "libcsolve.so")

_lib = None


def build() -> str:
    """Compile csolve.c with gcc (-O2 -fopenmp) if the library is missing or
    older than the source."""
    if os.path.exists(LIB) and os.path.getmtime(LIB) >= os.path.getmtime(SRC):
        return LIB
    os.makedirs(os.path.dirname(LIB), exist_ok=True)
    tmp = LIB + f".{os.getpid()}.tmp"
    cmd = ["gcc", "-O2", "-std=c99", "-fopenmp", "-fPIC", "-shared", SRC, "-o", tmp, "-lm"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"building the C oracle failed: {' '.join(cmd)}\n{r.stderr}")
    os.replace(tmp, LIB)
    return LIB


def lib():
    global _lib
    if _lib is None:
        _lib = C.CDLL(build())
        _lib.oc_max_threads.restype = C.c_int
        _lib.oc_galerkin_rows.restype = C.c_int
        _lib.oc_galerkin_fill.restype = C.c_int
        _lib.oc_pcg.restype = C.c_int
        _lib.oc_vcycle.restype = C.c_int
    return _lib


def set_threads(n: int):
    lib().oc_set_threads(int(n))


def max_threads() -> int:
    return int(lib().oc_max_threads())


def _p(a):
    return a.ctypes.data_as(C.c_void_p)


def _bsr(M: solve.Mat):
    return (np.ascontiguousarray(M.rowptr, dtype=np.int64), np.ascontiguousarray(M.colidx, dtype=np.int32),
            np.ascontiguousarray(M.vals, dtype=np.float64))


def galerkin(P: solve.Mat, A: solve.Mat, R: solve.Mat = None) -> solve.Mat:
    """A_c = P^T A P (R = P^T, built by solve.transpose when not given)."""
    if R is None:
        R = solve.transpose(P)
    Rrp, Rci, Rv = _bsr(R)
    Arp, Aci, Av = _bsr(A)
    Prp, Pci, Pv = _bsr(P)
    nc = P.n_cols
    crp = np.zeros(nc + 1, dtype=np.int64)
    L = lib()
    if L.oc_galerkin_rows(nc, nc, _p(Rrp), _p(Rci), A.n_rows, _p(Arp), _p(Aci), _p(Prp), _p(Pci),
                          _p(crp)) != 0:
        raise MemoryError("C oracle Galerkin: scratch allocation failed")
    np.cumsum(crp, out=crp)
    nnzb = int(crp[-1])
    kf, kc = P.br, P.bc
    cci = np.zeros(max(nnzb, 1), dtype=np.int32)
    cv = np.zeros((max(nnzb, 1), kc, kc))
    if L.oc_galerkin_fill(nc, nc, kf, kc, _p(Rrp), _p(Rci), _p(Rv), A.n_rows, _p(Arp), _p(Aci), _p(Av),
                          _p(Prp), _p(Pci), _p(Pv), _p(crp), _p(cci), _p(cv)) != 0:
        raise MemoryError("C oracle Galerkin: scratch allocation failed")
    return solve.Mat(nc, nc, crp, cci[:nnzb].astype(np.int64), cv[:nnzb])


class Hierarchy:
    """The solve-phase data of one hierarchy {A_0, P_l}: coarse matrices by
    the C Galerkin product, R_l = P_l^T, the smoother's blocks (and for
    smoother="hybrid_gs" its colour classes, solve.greedy_colouring) and the
    coarsest factor by oracle/solve.py.  smoother: "l1_jacobi" or
    "hybrid_gs", as solve.prepare."""

    def __init__(self, A0: solve.Mat, P, smoother: str = "l1_jacobi"):
        if smoother not in ("l1_jacobi", "hybrid_gs"):
            raise ValueError(f"unknown smoother {smoother!r}")
        self.smoother = smoother
        self.P = list(P)
        self.R = [solve.transpose(Pl) for Pl in self.P]
        self.A = [A0]
        for Pl, Rl in zip(self.P, self.R):
            self.A.append(galerkin(Pl, self.A[-1], Rl))
        if smoother == "hybrid_gs":
            self.colour = [solve.greedy_colouring(Al) for Al in self.A[:-1]]
            self.Minv = [np.ascontiguousarray(solve.hybrid_gs_inverse(Al, c))
                         for Al, c in zip(self.A[:-1], self.colour)]
        else:
            self.colour = []
            self.Minv = [np.ascontiguousarray(solve.block_l1_inverse(Al)) for Al in self.A[:-1]]
        self.Lc = np.ascontiguousarray(np.linalg.cholesky(solve.coarsest_matrix(self.A[-1])))
        self._pack()

    @property
    def n_levels(self):
        return len(self.A)

    def _pack(self):
        L = self.n_levels
        self._keep = []

        def arr(ctype, items):
            a = (ctype * max(L, 1))(*items)
            self._keep.append(a)
            return a

        Ab = [_bsr(A) for A in self.A]
        Pb = [_bsr(P) for P in self.P] + [(np.zeros(1, np.int64), np.zeros(1, np.int32), np.zeros(1))]
        Rb = [_bsr(R) for R in self.R] + [(np.zeros(1, np.int64), np.zeros(1, np.int32), np.zeros(1))]
        Mb = self.Minv + [np.zeros(1)]
        self._keep += [Ab, Pb, Rb, Mb]
        VP = C.c_void_p
        if self.colour:
            # class c of a level: its rows in ascending order (the order
            # inside a class does not matter: Jacobi-wise there)
            cls = []
            for col in self.colour:
                nc = int(col.max()) + 1 if col.size else 0
                ptr = np.zeros(nc + 1, dtype=np.int32)
                np.cumsum(np.bincount(col, minlength=nc), out=ptr[1:])
                cls.append((nc, ptr, np.ascontiguousarray(np.argsort(col, kind="stable"), dtype=np.int32)))
            cls.append((0, np.zeros(1, np.int32), np.zeros(1, np.int32)))
            self._keep.append(cls)
            gs = (arr(C.c_int, [c[0] for c in cls]), arr(VP, [_p(c[1]) for c in cls]),
                  arr(VP, [_p(c[2]) for c in cls]))
        else:
            gs = (None, None, None)
        self._args = (
            L, arr(C.c_int, [A.n_rows for A in self.A]), arr(C.c_int, [A.br for A in self.A]),
            arr(VP, [_p(a[0]) for a in Ab]), arr(VP, [_p(a[1]) for a in Ab]), arr(VP, [_p(a[2]) for a in Ab]),
            arr(VP, [_p(a[0]) for a in Pb]), arr(VP, [_p(a[1]) for a in Pb]), arr(VP, [_p(a[2]) for a in Pb]),
            arr(VP, [_p(a[0]) for a in Rb]), arr(VP, [_p(a[1]) for a in Rb]), arr(VP, [_p(a[2]) for a in Rb]),
            arr(VP, [_p(m) for m in Mb]), *gs, _p(self.Lc))

    def vcycle(self, r):
        r = np.ascontiguousarray(r, dtype=np.float64)
        z = np.zeros_like(r)
        if lib().oc_vcycle(*self._args, _p(r), _p(z)) != 0:
            raise MemoryError("C oracle V-cycle: allocation failed")
        return z

    def pcg(self, f, rtol=1e-8, maxit=500, x0=None):
        """CG preconditioned by one V-cycle, the stopping rule of
        solve.pcg; returns (x, iterations, relres history)."""
        f = np.ascontiguousarray(f, dtype=np.float64)
        x = np.zeros_like(f) if x0 is None else np.array(x0, dtype=np.float64)
        hist = np.zeros(int(maxit) + 1)
        it = lib().oc_pcg(*self._args, _p(f), _p(x), C.c_double(rtol), int(maxit), _p(hist))
        if it < 0:
            raise MemoryError("C oracle PCG: allocation failed")
        return x, int(it), hist[:it + 1].tolist()


def spmv(M: solve.Mat, x):
    rp, ci, v = _bsr(M)
    x = np.ascontiguousarray(x, dtype=np.float64)
    y = np.zeros(M.n_rows * M.br)
    lib().oc_spmv(M.n_rows, M.n_cols, M.br, M.bc, _p(rp), _p(ci), _p(v), _p(x), _p(y))
    return y
