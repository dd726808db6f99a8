"""Thin ctypes binding of libamg (include/amg.h): the same entry points, with
argument marshalling only.  Device vectors are torch CUDA tensors (FP64);
host matrices are numpy arrays.  Every step of the solve runs in libamg's
CUDA kernels; there is no fallback: if libamg.so is missing or no GPU is
present, the calls raise.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIBPATH = os.path.join(HERE, "libamg.so")

AMG_OK = 0
AMG_ERR_ARG = -1
AMG_ERR_CUDA = -2
AMG_ERR_NOT_SPD = -3
AMG_ERR_NO_CONVERGENCE = -4
AMG_ERR_TIMEOUT = -5
AMG_ERR_STATE = -6
ERRORS = {AMG_ERR_ARG: "AMG_ERR_ARG", AMG_ERR_CUDA: "AMG_ERR_CUDA", AMG_ERR_NOT_SPD: "AMG_ERR_NOT_SPD",
          AMG_ERR_NO_CONVERGENCE: "AMG_ERR_NO_CONVERGENCE", AMG_ERR_TIMEOUT: "AMG_ERR_TIMEOUT",
          AMG_ERR_STATE: "AMG_ERR_STATE"}

AMG_PREC_FP64 = 0
AMG_PREC_FP32_VCYCLE = 1
AMG_PREC_BF16_STORAGE = 2
AMG_PREC_BF16_COARSE = 3
AMG_LAYOUT_AUTO = 0
AMG_LAYOUT_SELL_SHORT_ROWS = 1
AMG_LAYOUT_WARP_ROWS = 2
AMG_LAYOUT_ROW_LANES = 3
AMG_LAYOUT_BLOCK_LANES = 4
AMG_LAYOUT_SELL_SPLIT = 5
AMG_SMOOTHER_L1_JACOBI = 0
AMG_SMOOTHER_LEARNED = 1
AMG_SMOOTHER_HYBRID_GS = 2
AMG_CG_FP64 = 0
AMG_CG_DOUBLE_FLOAT = 1
AMG_CG_AUTO = 2


class amg_bsr(C.Structure):
    _fields_ = [("n_rows", C.c_int32), ("n_cols", C.c_int32), ("br", C.c_int32), ("bc", C.c_int32),
                ("nnzb", C.c_int64), ("rowptr", C.POINTER(C.c_int32)),
                ("colidx", C.POINTER(C.c_int32)), ("vals", C.POINTER(C.c_double))]


class amg_bsr_out(C.Structure):
    _fields_ = amg_bsr._fields_


class amg_hierarchy(C.Structure):
    _fields_ = [("A0", amg_bsr), ("n_levels", C.c_int32), ("P", C.POINTER(amg_bsr))]


class amg_problem(C.Structure):
    _fields_ = [("dim", C.c_int32), ("n_vertices", C.c_int32), ("coords", C.POINTER(C.c_double)),
                ("dirichlet", C.POINTER(C.c_uint8)), ("A_full", amg_bsr), ("block", C.c_int32)]


class amg_setup_params(C.Structure):
    _fields_ = [("sigma", C.c_double), ("delta", C.c_int32), ("passes_first", C.c_int32),
                ("passes_later", C.c_int32), ("omega", C.c_double), ("cap_S_first", C.c_int32),
                ("cap_S_later", C.c_int32), ("cap_A", C.c_int32), ("coarse_max", C.c_int32),
                ("min_ratio", C.c_double), ("max_levels", C.c_int32),
                ("host_threads", C.c_int32), ("device_setup", C.c_int32),
                ("keep_topology", C.c_int32), ("scalar_only", C.c_int32),
                ("device_pair_measure", C.c_int32)]


class AmgError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{ERRORS.get(code, code)}: {msg}")
        self.code = code


_lib = None

_P = C.c_void_p
_I = C.c_int
_D = C.c_double
_SIGS = {
    "amg_create": (_I, [C.POINTER(_P), _I, _P]),
    "amg_destroy": (None, [_P]),
    "amg_last_error": (C.c_char_p, [_P]),
    "amg_upload_hierarchy": (_I, [_P, C.POINTER(amg_hierarchy), _I, _I]),
    "amg_galerkin": (_I, [_P, _I, C.POINTER(amg_bsr_out)]),
    "amg_level_info": (_I, [_P, _I, C.POINTER(C.c_int32), C.POINTER(C.c_int32),
                            C.POINTER(C.c_int64), C.POINTER(C.c_int64), C.POINTER(C.c_int32)]),
    "amg_download_matrix": (_I, [_P, _I, _P, _P, _P]),
    "amg_download_smoother": (_I, [_P, _I, _P]),
    "amg_download_coarse_inverse": (_I, [_P, _P]),
    "amg_spmv": (_I, [_P, _I, _P, _P]),
    "amg_residual": (_I, [_P, _I, _P, _P, _P]),
    "amg_smooth": (_I, [_P, _I, _P, _P, _P]),
    "amg_restrict": (_I, [_P, _I, _P, _P]),
    "amg_prolong_add": (_I, [_P, _I, _P, _P]),
    "amg_coarse_solve": (_I, [_P, _P, _P]),
    "amg_vcycle": (_I, [_P, _P, _P, _I]),
    "amg_vcycle_static": (_I, [_P, _P, _P]),
    "amg_pcg_solve": (_I, [_P, _P, _P, _I, _D, _I, C.POINTER(_I), C.POINTER(_D)]),
    "amg_pcg_solve_host": (_I, [_P, _P, _P, _I, _D, _I, C.POINTER(_I), C.POINTER(_D)]),
    "amg_last_solve_ms": (_I, [_P, C.POINTER(C.c_float)]),
    "amg_set_pcg_graph": (_I, [_P, _I]),
    "amg_set_layout_policy": (_I, [_P, _I]),
    "amg_probe_fma_rate": (_I, [_P, C.POINTER(C.c_double), C.POINTER(C.c_double)]),
    "amg_setup_times": (_I, [_P, C.POINTER(C.c_double)]),
    "amg_setup_device_split": (_I, [_P, C.POINTER(C.c_double), C.POINTER(C.c_double),
                                    C.POINTER(C.c_double)]),
    "amg_download_topology": (_I, [_P, _I, C.POINTER(C.c_int32), C.POINTER(C.c_int64),
                                   C.POINTER(C.c_int32), _P, _P, _P, _P, _P]),
    "amg_default_setup_params": (None, [C.POINTER(amg_setup_params)]),
    "amg_setup": (_I, [_P, C.POINTER(amg_problem), C.POINTER(amg_setup_params), _I, _I]),
    "amg_prolongation_info": (_I, [_P, _I, C.POINTER(C.c_int32), C.POINTER(C.c_int32),
                                   C.POINTER(C.c_int32), C.POINTER(C.c_int32), C.POINTER(C.c_int64)]),
    "amg_download_prolongation": (_I, [_P, _I, _P, _P, _P]),
    "amg_describe": (C.c_char_p, [_P]),
    "amg_set_launch_overlap": (_I, [_P, _I]),
    "amg_pcg_launches": (_I, [_P, C.POINTER(C.c_int32), C.POINTER(C.c_int32)]),
    "amg_profile_vcycle": (_I, [_P, _I, _P, _P, _P, _P, _I, C.POINTER(C.c_int32)]),
    "amg_profile_pcg": (_I, [_P, _I, _P, _P, _P, _I, C.POINTER(C.c_int32)]),
    "amg_set_cg_operator": (_I, [_P, _I]),
    "amg_smoother_colouring": (_I, [_P, _I, _P, C.POINTER(C.c_int32)]),
    "amg_cg_operator": (_I, [_P, _P, _P]),
    "amg_mlp_create": (_I, [C.POINTER(_P), _I, C.c_uint64]),
    "amg_mlp_destroy": (None, [_P]),
    "amg_mlp_last_error": (C.c_char_p, [_P]),
    "amg_mlp_n_params": (_I, []),
    "amg_mlp_get_params": (_I, [_P, _P, _I]),
    "amg_mlp_set_params": (_I, [_P, _P]),
    "amg_learned_features": (_I, [_P, _P, _P, _P]),
    "amg_learned_targets": (_I, [_P, _P, _P]),
    "amg_mlp_loss_grad": (_I, [_P, _P, _P, C.c_int64, C.POINTER(_D), _P]),
    "amg_mlp_train": (_I, [_P, _P, _P, C.c_int64, _I, _I, C.c_float, C.c_uint64, _P]),
    "amg_mlp_infer": (_I, [_P, _P, C.c_int64, _P]),
    "amg_set_learned_smoother": (_I, [_P, _P, _P, C.POINTER(_D), C.POINTER(_D)]),
    "amg_reset_smoother": (_I, [_P]),
    "amg_batch_create": (_I, [C.POINTER(_P), C.POINTER(_P), _I, _I]),
    "amg_batch_destroy": (None, [_P]),
    "amg_batch_last_error": (C.c_char_p, [_P]),
    "amg_batch_describe": (C.c_char_p, [_P]),
    "amg_batch_launches": (_I, [_P, C.POINTER(C.c_int32), C.POINTER(C.c_int32)]),
    "amg_batch_layout": (_I, [_P, _I, C.POINTER(C.c_int64), C.POINTER(C.c_int64),
                              C.POINTER(C.c_int64)]),
    "amg_batch_pcg_solve": (_I, [_P, _P, _P, _D, _I, C.POINTER(_I), C.POINTER(_D),
                                 C.POINTER(C.c_float)]),
    "amg_batch_pcg_solve_host": (_I, [_P, _P, _P, _D, _I, C.POINTER(_I), C.POINTER(_D),
                                      C.POINTER(C.c_float)]),
}


def lib():
    """Load libamg.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIBPATH):
            raise RuntimeError(f"{LIBPATH} is missing: build it with "
                               "`python paper_2011_13325_gb300/build.py` (needs nvcc)")
        L = C.CDLL(LIBPATH)
        for name, (res, args) in _SIGS.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def exported_symbols():
    return list(_SIGS.keys())


def _ptr(a, where="argument", host=False, dtype="float64", n=None, device=None):
    """Pointer of a flat array argument of a libamg call, after the checks
    the C side cannot make: a device argument is a CUDA tensor (on `device`
    when given), a host argument a numpy array or CPU tensor; the element
    type is `dtype`, the storage C-contiguous, and at least `n` elements
    long where the caller knows the length.  None passes through as NULL.
    Raises TypeError / ValueError rather than hand the library a pointer it
    would read or write past."""
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        if not host:
            raise TypeError(f"{where}: needs a CUDA tensor, got a numpy array")
        if a.dtype != np.dtype(dtype):
            raise TypeError(f"{where}: needs {dtype} elements, got {a.dtype}")
        if not a.flags.c_contiguous:
            raise ValueError(f"{where}: the array must be C-contiguous")
        size, ptr = a.size, a.ctypes.data
    else:
        if not hasattr(a, "data_ptr"):
            raise TypeError(f"{where}: needs a torch tensor or numpy array, got {type(a).__name__}")
        if bool(a.is_cuda) == bool(host):
            raise TypeError(f"{where}: needs a {'CPU' if host else 'CUDA'} tensor, got one on {a.device}")
        if not host and device is not None and a.device.index != int(device):
            raise ValueError(f"{where}: tensor on {a.device}, the context is on cuda:{int(device)}")
        if str(a.dtype) != f"torch.{dtype}":
            raise TypeError(f"{where}: needs {dtype} elements, got {a.dtype}")
        if not a.is_contiguous():
            raise ValueError(f"{where}: the tensor must be contiguous")
        size, ptr = a.numel(), a.data_ptr()
    if n is not None and size < n:
        raise ValueError(f"{where}: needs at least {n} elements, got {size}")
    return ptr


def bsr_struct(n_rows, n_cols, rowptr, colidx, vals, keep):
    rowptr = np.ascontiguousarray(rowptr, dtype=np.int32)
    colidx = np.ascontiguousarray(colidx, dtype=np.int32)
    vals = np.ascontiguousarray(vals, dtype=np.float64)
    keep.extend([rowptr, colidx, vals])
    return amg_bsr(int(n_rows), int(n_cols), int(vals.shape[1]), int(vals.shape[2]),
                   int(colidx.shape[0]), rowptr.ctypes.data_as(C.POINTER(C.c_int32)),
                   colidx.ctypes.data_as(C.POINTER(C.c_int32)),
                   vals.ctypes.data_as(C.POINTER(C.c_double)))


class Context:
    """One libamg context (amg_create ... amg_destroy)."""

    def __init__(self, device: int = 0, stream=None):
        self.h = _P()
        self.device = int(device)
        s = lib().amg_create(C.byref(self.h), int(device), stream)
        if s != AMG_OK:
            raise AmgError(s, "amg_create failed")

    def close(self):
        if self.h:
            lib().amg_destroy(self.h)
            self.h = _P()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, s):
        if s != AMG_OK:
            raise AmgError(s, lib().amg_last_error(self.h).decode())
        return s

    def _dofs(self, level):
        """Scalar rows of a level, or None without a hierarchy or for a level
        it does not have (the library then reports that error itself)."""
        n, k = C.c_int32(), C.c_int32()
        if lib().amg_level_info(self.h, int(level), C.byref(n), C.byref(k), None, None, None) != AMG_OK:
            return None
        return n.value * k.value

    def _vec(self, a, where, level=0, count=1):
        """Device pointer of an FP64 vector of `count` copies of a level's
        unknowns (length checked when the hierarchy is there)."""
        n = self._dofs(level)
        return _ptr(a, where, n=None if n is None else n * int(count), device=self.device)

    # -- hierarchy ---------------------------------------------------------
    def upload_hierarchy(self, A0, P_list, precision=AMG_PREC_FP64, smoother=AMG_SMOOTHER_L1_JACOBI):
        """A0 / P_list: objects with n_rows, n_cols, rowptr, colidx, vals."""
        keep = []
        a0 = bsr_struct(A0.n_rows, A0.n_cols, A0.rowptr, A0.colidx, A0.vals, keep)
        Ps = (amg_bsr * max(1, len(P_list)))()
        for i, P in enumerate(P_list):
            Ps[i] = bsr_struct(P.n_rows, P.n_cols, P.rowptr, P.colidx, P.vals, keep)
        h = amg_hierarchy(a0, len(P_list) + 1, Ps)
        return self._check(lib().amg_upload_hierarchy(self.h, C.byref(h), int(precision), int(smoother)))

    def setup(self, problem, precision=AMG_PREC_FP64, smoother=AMG_SMOOTHER_L1_JACOBI, **params):
        """amg_setup on a ``workloads.Problem`` (full matrix, coordinates,
        Dirichlet flags); keyword arguments override amg_setup_params."""
        keep = []
        prm = amg_setup_params()
        lib().amg_default_setup_params(C.byref(prm))
        for k, v in params.items():
            setattr(prm, k, v)
        coords = np.ascontiguousarray(problem.coords, dtype=np.float64)
        dmask = np.ascontiguousarray(problem.dirichlet, dtype=np.uint8)
        keep.extend([coords, dmask])
        Af = problem.A_full
        pr = amg_problem(int(problem.dim), int(coords.shape[0]),
                         coords.ctypes.data_as(C.POINTER(C.c_double)),
                         dmask.ctypes.data_as(C.POINTER(C.c_uint8)),
                         bsr_struct(Af.n_rows, Af.n_cols, Af.rowptr, Af.colidx, Af.vals, keep),
                         int(getattr(problem, "k", problem.dim)))
        return self._check(lib().amg_setup(self.h, C.byref(pr), C.byref(prm), int(precision),
                                           int(smoother)))

    def download_prolongation(self, level):
        n, m, br, bc, nnzb = C.c_int32(), C.c_int32(), C.c_int32(), C.c_int32(), C.c_int64()
        self._check(lib().amg_prolongation_info(self.h, int(level), C.byref(n), C.byref(m),
                                                C.byref(br), C.byref(bc), C.byref(nnzb)))
        rp = np.zeros(n.value + 1, dtype=np.int32)
        ci = np.zeros(max(nnzb.value, 1), dtype=np.int32)
        v = np.zeros((max(nnzb.value, 1), br.value, bc.value))
        self._check(lib().amg_download_prolongation(self.h, int(level), rp.ctypes.data,
                                                    ci.ctypes.data, v.ctypes.data))
        return n.value, m.value, rp, ci[:nnzb.value], v[:nnzb.value]

    def level_info(self, level):
        n, k, na, npb, nl = C.c_int32(), C.c_int32(), C.c_int64(), C.c_int64(), C.c_int32()
        self._check(lib().amg_level_info(self.h, int(level), C.byref(n), C.byref(k), C.byref(na),
                                         C.byref(npb), C.byref(nl)))
        return dict(n_rows=n.value, block=k.value, nnzb=na.value, nnzb_P=npb.value, n_levels=nl.value)

    @property
    def n_levels(self):
        nl = C.c_int32()
        lib().amg_level_info(self.h, 0, None, None, None, None, C.byref(nl))
        return nl.value

    def download_matrix(self, level):
        info = self.level_info(level)
        n, k, nnzb = info["n_rows"], info["block"], info["nnzb"]
        rp = np.zeros(n + 1, dtype=np.int32)
        ci = np.zeros(max(nnzb, 1), dtype=np.int32)
        v = np.zeros((max(nnzb, 1), k, k))
        self._check(lib().amg_download_matrix(self.h, int(level), rp.ctypes.data, ci.ctypes.data,
                                              v.ctypes.data))
        return rp, ci[:nnzb], v[:nnzb]

    def galerkin(self, level, download=True):
        if not download:
            return self._check(lib().amg_galerkin(self.h, int(level), None))
        out = amg_bsr_out()
        # sizes are only known after the product: run it, then download
        self._check(lib().amg_galerkin(self.h, int(level), None))
        return self.download_matrix(level + 1)

    def download_smoother(self, level):
        info = self.level_info(level)
        m = np.zeros((info["n_rows"], info["block"], info["block"]))
        self._check(lib().amg_download_smoother(self.h, int(level), m.ctypes.data))
        return m

    def download_coarse_inverse(self):
        info = self.level_info(self.n_levels - 1)
        n = info["n_rows"] * info["block"]
        m = np.zeros((n, n))
        self._check(lib().amg_download_coarse_inverse(self.h, m.ctypes.data))
        return m

    # -- single steps ------------------------------------------------------
    def spmv(self, level, x, y):
        return self._check(lib().amg_spmv(self.h, int(level), self._vec(x, "x", level),
                                          self._vec(y, "y", level)))

    def residual(self, level, b, x, r):
        return self._check(lib().amg_residual(self.h, int(level), self._vec(b, "b", level),
                                              self._vec(x, "x", level), self._vec(r, "r", level)))

    def smooth(self, level, b, x_in, x_out):
        return self._check(lib().amg_smooth(self.h, int(level), self._vec(b, "b", level),
                                            self._vec(x_in, "x_in", level),
                                            self._vec(x_out, "x_out", level)))

    def restrict(self, level, r, bc):
        return self._check(lib().amg_restrict(self.h, int(level), self._vec(r, "r", level),
                                              self._vec(bc, "bc", level + 1)))

    def prolong_add(self, level, ec, x):
        return self._check(lib().amg_prolong_add(self.h, int(level), self._vec(ec, "ec", level + 1),
                                                 self._vec(x, "x", level)))

    def coarse_solve(self, b, x):
        last = self.n_levels - 1
        return self._check(lib().amg_coarse_solve(self.h, self._vec(b, "b", last),
                                                  self._vec(x, "x", last)))

    def vcycle(self, r, z, nrhs=1):
        return self._check(lib().amg_vcycle(self.h, self._vec(r, "r", 0, nrhs),
                                            self._vec(z, "z", 0, nrhs), int(nrhs)))

    def vcycle_static(self, r, z):
        """amg_vcycle_static: one V-cycle without allocating (work vectors in
        the library's fixed device array)."""
        return self._check(lib().amg_vcycle_static(self.h, self._vec(r, "r"), self._vec(z, "z")))

    def pcg_solve(self, f, u, nrhs=1, rtol=1e-8, maxit=500, check=True):
        it = (C.c_int * nrhs)()
        rr = (C.c_double * nrhs)()
        s = lib().amg_pcg_solve(self.h, self._vec(f, "f", 0, nrhs), self._vec(u, "u", 0, nrhs),
                                int(nrhs), float(rtol), int(maxit), it, rr)
        if check:
            self._check(s)
        return s, list(it), list(rr)

    def pcg_solve_host(self, f, u, nrhs=1, rtol=1e-8, maxit=500, check=True):
        it = (C.c_int * nrhs)()
        rr = (C.c_double * nrhs)()
        n = self._dofs(0)
        n = None if n is None else n * int(nrhs)
        s = lib().amg_pcg_solve_host(self.h, _ptr(f, "f", host=True, n=n), _ptr(u, "u", host=True, n=n),
                                     int(nrhs), float(rtol), int(maxit), it, rr)
        if check:
            self._check(s)
        return s, list(it), list(rr)

    def setup_times(self):
        t = (C.c_double * 4)()
        self._check(lib().amg_setup_times(self.h, t))
        g, tp, pm = C.c_double(), C.c_double(), C.c_double()
        self._check(lib().amg_setup_device_split(self.h, C.byref(g), C.byref(tp), C.byref(pm)))
        return dict(host_s=t[0], device_s=t[1], finalize_s=t[2], total_s=t[3],
                    device_galerkin_s=g.value, device_topology_prolongation_s=tp.value,
                    device_pair_measure_s=pm.value)

    def download_topology(self, level):
        """(pos, edges (m x 2), E (m x k x k), M (n x k x k)) of the coarse
        topology of `level` kept by amg_setup(keep_topology=1)."""
        n, m, k = C.c_int32(), C.c_int64(), C.c_int32()
        self._check(lib().amg_download_topology(self.h, int(level), C.byref(n), C.byref(m), C.byref(k),
                                                None, None, None, None, None))
        n, m, k = n.value, m.value, k.value
        d = 2 if k == 3 else 3
        ei = np.zeros(max(m, 1), dtype=np.int32)
        ej = np.zeros(max(m, 1), dtype=np.int32)
        E = np.zeros((max(m, 1), k, k))
        M = np.zeros((max(n, 1), k, k))
        pos = np.zeros((max(n, 1), d))
        self._check(lib().amg_download_topology(self.h, int(level), None, None, None, ei.ctypes.data,
                                                ej.ctypes.data, E.ctypes.data, M.ctypes.data,
                                                pos.ctypes.data))
        return pos[:n], np.stack([ei[:m], ej[:m]], axis=1), E[:m], M[:n]

    def probe_fma_rate(self):
        a, b = C.c_double(), C.c_double()
        self._check(lib().amg_probe_fma_rate(self.h, C.byref(a), C.byref(b)))
        return a.value, b.value

    def learned_features(self, coords, X, tr=None):
        """Features (n_0 x 13 FP32 device tensor X) of the level-0 vertices at
        host positions coords (n_0 x 3)."""
        c = np.ascontiguousarray(coords, dtype=np.float64)
        n = self._n0()
        if n is not None and c.size < 3 * n:
            raise ValueError(f"coords: needs {n} x 3 positions, got {c.size} values")
        return self._check(lib().amg_learned_features(
            self.h, c.ctypes.data,
            _ptr(X, "X", dtype="float32", n=None if n is None else 13 * n, device=self.device),
            _ptr(tr, "tr", n=n, device=self.device)))

    def learned_targets(self, T32=None, T64=None):
        """Patch-inverse targets (n_0 x 9) into device tensors."""
        n = self._n0()
        m = None if n is None else 9 * n
        return self._check(lib().amg_learned_targets(
            self.h, _ptr(T32, "T32", dtype="float32", n=m, device=self.device),
            _ptr(T64, "T64", n=m, device=self.device)))

    def _n0(self):
        """Level-0 vertices (block rows), or None without a hierarchy."""
        n = C.c_int32()
        if lib().amg_level_info(self.h, 0, C.byref(n), None, None, None, None) != AMG_OK:
            return None
        return n.value

    def set_learned_smoother(self, mlp, coords):
        """Install the damped learned blocks at level 0; returns (lambda, omega)."""
        c = np.ascontiguousarray(coords, dtype=np.float64)
        n = self._n0()
        if n is not None and c.size < 3 * n:
            raise ValueError(f"coords: needs {n} x 3 positions, got {c.size} values")
        lam, w = C.c_double(), C.c_double()
        self._check(lib().amg_set_learned_smoother(self.h, mlp.h, c.ctypes.data, C.byref(lam),
                                                   C.byref(w)))
        return lam.value, w.value

    def reset_smoother(self):
        return self._check(lib().amg_reset_smoother(self.h))

    def describe(self):
        return lib().amg_describe(self.h).decode()

    PROFILE_KINDS = ("pre-smooth x = M^+ b", "residual t = b - A x", "restriction R t",
                     "prolongation x += P y", "post-smooth", "coarsest solve")

    def profile_vcycle(self, reps=20):
        """[(level, step, us per launch, algorithmic bytes)] of one V-cycle."""
        m = 8 * 64
        lv = np.zeros(m, dtype=np.int32)
        kd = np.zeros(m, dtype=np.int32)
        us = np.zeros(m)
        by = np.zeros(m)
        n = C.c_int32()
        self._check(lib().amg_profile_vcycle(self.h, int(reps), lv.ctypes.data, kd.ctypes.data,
                                             us.ctypes.data, by.ctypes.data, m, C.byref(n)))
        return [(int(lv[i]), self.PROFILE_KINDS[kd[i]], float(us[i]), float(by[i]))
                for i in range(min(n.value, m))]

    PCG_KINDS = ("rho = r.z", "p = z + beta p", "q = A_0 p, p.q partials", "alpha = rho / p.q",
                 "x += alpha p, r -= alpha q, r.r partials", "loop decision")

    def profile_pcg(self, reps=20):
        """[(step, us per launch, algorithmic bytes)] of the CG kernels of one
        PCG iteration (the V-cycle excluded); overwrites the CG vectors."""
        kd = np.zeros(8, dtype=np.int32)
        us = np.zeros(8)
        by = np.zeros(8)
        n = C.c_int32()
        self._check(lib().amg_profile_pcg(self.h, int(reps), kd.ctypes.data, us.ctypes.data,
                                          by.ctypes.data, 8, C.byref(n)))
        return [(self.PCG_KINDS[kd[i]], float(us[i]), float(by[i])) for i in range(min(n.value, 8))]

    def smoother_colouring(self, level):
        """(colour of every block row of `level`, number of colours) under
        the hybrid Gauss-Seidel smoother."""
        info = self.level_info(level)
        col = np.zeros(max(info["n_rows"], 1), dtype=np.int32)
        nc = C.c_int32()
        self._check(lib().amg_smoother_colouring(self.h, int(level), col.ctypes.data, C.byref(nc)))
        return col[:info["n_rows"]], nc.value

    def set_cg_operator(self, mode: int):
        """AMG_CG_FP64, AMG_CG_DOUBLE_FLOAT or AMG_CG_AUTO (default: double-float with the
        FP32 / BF16 V-cycles): arithmetic of q = A_0 p in the PCG."""
        return self._check(lib().amg_set_cg_operator(self.h, int(mode)))

    def cg_operator(self, p, q):
        """q = A_0 p with the PCG's CG operator (its selected arithmetic)."""
        return self._check(lib().amg_cg_operator(self.h, self._vec(p, "p", 0), self._vec(q, "q", 0)))

    def set_layout_policy(self, policy: int):
        return self._check(lib().amg_set_layout_policy(self.h, int(policy)))

    def pcg_launches(self):
        """(kernels per PCG iteration, fixed kernels per solve)."""
        a, b = C.c_int32(), C.c_int32()
        self._check(lib().amg_pcg_launches(self.h, C.byref(a), C.byref(b)))
        return a.value, b.value

    def set_launch_overlap(self, enable: bool):
        return self._check(lib().amg_set_launch_overlap(self.h, int(bool(enable))))

    def set_pcg_graph(self, enable: bool):
        return self._check(lib().amg_set_pcg_graph(self.h, int(bool(enable))))

    def last_solve_ms(self):
        ms = C.c_float()
        self._check(lib().amg_last_solve_ms(self.h, C.byref(ms)))
        return ms.value


class Batch:
    """amg_batch: independent systems (Contexts with uploaded hierarchies),
    nrhs load cases each, solved by one graph launch."""

    def __init__(self, contexts, nrhs=6):
        self.contexts = list(contexts)          # keep them alive
        self.nrhs = int(nrhs)
        arr = (_P * len(self.contexts))(*[c.h for c in self.contexts])
        self.h = _P()
        s = lib().amg_batch_create(C.byref(self.h), arr, len(self.contexts), self.nrhs)
        if s != AMG_OK:
            raise AmgError(s, "amg_batch_create failed")

    def close(self):
        if self.h:
            lib().amg_batch_destroy(self.h)
            self.h = _P()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def describe(self):
        return lib().amg_batch_describe(self.h).decode()

    def launches(self):
        """(kernels per iteration, fixed kernels per solve)."""
        a, b = C.c_int32(), C.c_int32()
        lib().amg_batch_launches(self.h, C.byref(a), C.byref(b))
        return a.value, b.value

    def layout(self, s):
        o, n, t = C.c_int64(), C.c_int64(), C.c_int64()
        st = lib().amg_batch_layout(self.h, int(s), C.byref(o), C.byref(n), C.byref(t))
        if st != AMG_OK:
            raise AmgError(st, "amg_batch_layout")
        return o.value, n.value, t.value

    def pcg_solve(self, f, u, rtol=1e-8, maxit=500, check=True):
        """Stacked device vectors (torch tensors)."""
        return self._solve(lib().amg_batch_pcg_solve, f, u, rtol, maxit, check, host=False)

    def pcg_solve_host(self, f, u, rtol=1e-8, maxit=500, check=True):
        """Stacked host vectors (numpy arrays or CPU tensors, pinned for speed)."""
        return self._solve(lib().amg_batch_pcg_solve_host, f, u, rtol, maxit, check, host=True)

    def _solve(self, fn, f, u, rtol, maxit, check, host):
        m = len(self.contexts) * self.nrhs
        it = (C.c_int * m)()
        rr = (C.c_double * m)()
        ms = C.c_float()
        total = self.layout(0)[2] if self.contexts else None
        dev = None if host or not self.contexts else self.contexts[0].device
        s = fn(self.h, _ptr(f, "f", host=host, n=total, device=dev),
               _ptr(u, "u", host=host, n=total, device=dev), float(rtol), int(maxit), it, rr,
               C.byref(ms))
        if check and s != AMG_OK:
            raise AmgError(s, lib().amg_batch_last_error(self.h).decode())
        return s, list(it), list(rr), ms.value


AMG_MLP_PARAMS = 5446


class Mlp:
    """amg_mlp: the learned smoother's network (FP32 master weights, BF16
    working copy) with its device training."""

    def __init__(self, device=0, seed=0):
        self.h = _P()
        s = lib().amg_mlp_create(C.byref(self.h), int(device), C.c_uint64(int(seed)))
        if s != AMG_OK:
            raise AmgError(s, "amg_mlp_create failed")

    def close(self):
        if self.h:
            lib().amg_mlp_destroy(self.h)
            self.h = _P()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, s):
        if s != AMG_OK:
            raise AmgError(s, lib().amg_mlp_last_error(self.h).decode())
        return s

    def params(self, working=False):
        out = np.zeros(AMG_MLP_PARAMS, dtype=np.float32)
        self._check(lib().amg_mlp_get_params(self.h, out.ctypes.data, int(bool(working))))
        return out

    def set_params(self, p):
        p = np.ascontiguousarray(p, dtype=np.float32)
        if p.size != AMG_MLP_PARAMS:
            raise ValueError("wrong number of parameters")
        return self._check(lib().amg_mlp_set_params(self.h, p.ctypes.data))

    def loss_grad(self, X, T, n=None):
        n = int(X.shape[0]) if n is None else int(n)
        loss = C.c_double()
        g = np.zeros(AMG_MLP_PARAMS, dtype=np.float32)
        self._check(lib().amg_mlp_loss_grad(self.h, _ptr(X, "X", dtype="float32", n=13 * n),
                                            _ptr(T, "T", dtype="float32", n=9 * n), n,
                                            C.byref(loss), g.ctypes.data))
        return loss.value, g

    def train(self, X, T, epochs=10, batch=4096, lr=1e-3, seed=0, n=None):
        n = int(X.shape[0]) if n is None else int(n)
        hist = np.zeros(max(epochs, 1))
        self._check(lib().amg_mlp_train(self.h, _ptr(X, "X", dtype="float32", n=13 * n),
                                        _ptr(T, "T", dtype="float32", n=9 * n), n, int(epochs), int(batch),
                                        float(lr), C.c_uint64(int(seed)), hist.ctypes.data))
        return hist[:epochs]

    def infer(self, X, out, n=None):
        n = int(X.shape[0]) if n is None else int(n)
        return self._check(lib().amg_mlp_infer(self.h, _ptr(X, "X", dtype="float32", n=13 * n), n,
                                               _ptr(out, "out", dtype="float32", n=6 * n)))
