"""Thin ctypes binding of the C ABI declared in ``include/rsnegf.h``.

Argument marshalling only: every step of the computation runs in the CUDA
library.  PyTorch supplies device memory (output tensors) and the stream.
If the shared library has not been built, :func:`load` raises -- there is no
CPU fallback.
"""
from __future__ import annotations

import ctypes as ct
import dataclasses
import os
from typing import List, Optional, Sequence

import numpy as np

from . import build as _build

RSN_OK, RSN_EINVAL, RSN_ENOMEM, RSN_ECUDA, RSN_ENOCONV, RSN_ETIMEOUT, RSN_EBREAKDOWN, RSN_ESTATE = \
    0, -1, -2, -3, -4, -5, -6, -7
RSN_FP64, RSN_MIXED = 0, 1
_STATUS = {0: "RSN_OK", -1: "RSN_EINVAL", -2: "RSN_ENOMEM", -3: "RSN_ECUDA", -4: "RSN_ENOCONV",
           -5: "RSN_ETIMEOUT", -6: "RSN_EBREAKDOWN", -7: "RSN_ESTATE"}

# every exported entry point and its ctypes signature
_SIGS = {
    "rsn_default_opts": (None, [ct.c_int, ct.c_void_p]),
    "rsn_create": (ct.c_int, [ct.POINTER(ct.c_void_p), ct.c_int, ct.c_void_p]),
    "rsn_destroy": (ct.c_int, [ct.c_void_p]),
    "rsn_set_grid": (ct.c_int, [ct.c_void_p, ct.c_int, ct.c_int, ct.c_int, ct.c_double, ct.c_int]),
    "rsn_set_potential": (ct.c_int, [ct.c_void_p, ct.c_void_p]),
    "rsn_set_projectors": (ct.c_int, [ct.c_void_p, ct.c_int, ct.c_void_p, ct.c_void_p, ct.c_void_p, ct.c_void_p]),
    "rsn_set_cap": (ct.c_int, [ct.c_void_p, ct.c_void_p, ct.c_void_p]),
    "rsn_apply": (ct.c_int, [ct.c_void_p, ct.c_int, ct.c_int, ct.c_void_p, ct.c_void_p, ct.c_void_p]),
    "rsn_apply_noalloc": (ct.c_int, [ct.c_void_p, ct.c_int, ct.c_int, ct.c_void_p, ct.c_void_p, ct.c_void_p]),
    "rsn_solve_columns": (ct.c_int, [ct.c_void_p, ct.c_int, ct.c_void_p, ct.c_int, ct.c_void_p, ct.c_void_p,
                                     ct.c_void_p, ct.c_void_p, ct.c_void_p]),
    "rsn_transmission": (ct.c_int, [ct.c_void_p, ct.c_int, ct.c_void_p, ct.c_int, ct.c_void_p, ct.c_void_p,
                                    ct.c_void_p]),
    "rsn_transmission_vjp": (ct.c_int, [ct.c_void_p, ct.c_int, ct.c_void_p, ct.c_int, ct.c_void_p, ct.c_void_p,
                                        ct.c_void_p, ct.c_void_p, ct.c_int, ct.c_void_p]),
    "rsn_solve_columns_shifted": (ct.c_int, [ct.c_void_p, ct.c_int, ct.c_void_p, ct.c_int, ct.c_void_p,
                                             ct.c_void_p, ct.c_void_p, ct.c_void_p, ct.c_void_p]),
    "rsn_transmission_shifted": (ct.c_int, [ct.c_void_p, ct.c_int, ct.c_void_p, ct.c_int, ct.c_void_p,
                                            ct.c_void_p, ct.c_void_p, ct.c_void_p]),
    "rsn_solve_columns_block": (ct.c_int, [ct.c_void_p, ct.c_int, ct.c_void_p, ct.c_int, ct.c_void_p, ct.c_int,
                                           ct.c_double, ct.c_void_p, ct.c_void_p, ct.c_void_p, ct.c_void_p,
                                           ct.c_void_p]),
    "rsn_transmission_block": (ct.c_int, [ct.c_void_p, ct.c_int, ct.c_void_p, ct.c_int, ct.c_void_p, ct.c_int,
                                          ct.c_double, ct.c_void_p, ct.c_void_p, ct.c_void_p, ct.c_void_p]),
    "rsn_transmission_keep": (ct.c_int, [ct.c_void_p, ct.c_int, ct.c_void_p, ct.c_int, ct.c_void_p, ct.c_void_p,
                                         ct.c_void_p, ct.c_void_p]),
    "rsn_transmission_vjp_reuse": (ct.c_int, [ct.c_void_p, ct.c_int, ct.c_void_p, ct.c_int, ct.c_void_p,
                                              ct.c_void_p, ct.c_void_p, ct.c_void_p, ct.c_void_p, ct.c_int]),
    "rsn_landauer_current": (ct.c_int, [ct.c_void_p, ct.c_int, ct.c_void_p, ct.c_void_p, ct.c_int, ct.c_void_p,
                                        ct.c_double, ct.c_double, ct.c_void_p]),
    "rsn_batch_transmission": (ct.c_int, [ct.c_int, ct.c_void_p, ct.c_void_p, ct.c_void_p, ct.c_void_p, ct.c_void_p,
                                          ct.c_void_p, ct.c_void_p, ct.c_void_p]),
    "rsn_last_stats": (ct.c_int, [ct.c_void_p, ct.c_void_p, ct.c_void_p, ct.c_void_p, ct.c_void_p, ct.c_void_p]),
    "rsn_last_error": (ct.c_char_p, [ct.c_void_p]),
    "rsn_kernel_stats": (ct.c_int, [ct.c_void_p, ct.c_int, ct.c_void_p, ct.c_void_p, ct.c_void_p]),
    "rsn_set_tiling": (ct.c_int, [ct.c_void_p, ct.c_int, ct.c_int, ct.c_int]),
    "rsn_bench_kernel": (ct.c_int, [ct.c_void_p, ct.c_int, ct.c_int, ct.c_int, ct.c_int, ct.c_void_p, ct.c_void_p]),
    "rsn_autotune": (ct.c_int, [ct.c_void_p, ct.c_int, ct.c_int, ct.c_void_p, ct.c_void_p, ct.c_void_p, ct.c_void_p,
                                ct.c_void_p]),
}


class SolverOpts(ct.Structure):
    """Mirror of ``rsn_solver_opts``."""

    _fields_ = [
        ("precision", ct.c_int),
        ("tol", ct.c_double),
        ("tol_inner", ct.c_double),
        ("max_iter", ct.c_int),
        ("max_outer", ct.c_int),
        ("deadline_ms", ct.c_double),
        ("rhs_block", ct.c_int),
        ("use_graph", ct.c_int),
        ("graph_iters", ct.c_int),
        ("timing", ct.c_int),
        ("tol_adjoint", ct.c_double),
        ("tol_T", ct.c_double),
    ]


class RsnError(RuntimeError):
    def __init__(self, fn: str, code: int, msg: str):
        super().__init__(f"{fn} -> {_STATUS.get(code, code)}: {msg}")
        self.code = code


_lib = None


def load(path: Optional[str] = None):
    """Load the shared library (built by ``paper_1401_0782_gb300.build``)."""
    global _lib
    if _lib is not None and path is None:
        return _lib
    path = path or _build.lib_path()
    if not os.path.exists(path):
        raise RuntimeError(f"CUDA library not built: {path} is missing "
                           "(run paper_1401_0782_gb300.build.build() on a machine with nvcc)")
    lib = ct.CDLL(path)
    for name, (res, args) in _SIGS.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    if path == _build.lib_path():
        _lib = lib
    return lib


def exported_symbols():
    return sorted(_SIGS)


def default_opts(precision: int = RSN_FP64, **kw) -> SolverOpts:
    o = SolverOpts()
    load().rsn_default_opts(precision, ct.byref(o))
    for k, v in kw.items():
        if not hasattr(o, k):
            raise AttributeError(k)
        setattr(o, k, v)
    return o


def _ptr(a) -> int:
    return a.ctypes.data if isinstance(a, np.ndarray) else int(a)


def _torch():
    import torch
    return torch


class Context:
    """One junction on one GPU (wraps ``rsn_ctx``)."""

    def __init__(self, device: int = 0, stream=None):
        self.lib = load()
        torch = _torch()
        self.device = device
        if stream is None:
            stream = torch.cuda.current_stream(device)
        self._stream = stream
        h = ct.c_void_p()
        rc = self.lib.rsn_create(ct.byref(h), device, ct.c_void_p(stream.cuda_stream))
        if rc != RSN_OK:
            raise RsnError("rsn_create", rc, self.lib.rsn_last_error(None).decode())
        self.h = h
        self.N = 0
        self.junction = None

    def close(self):
        if getattr(self, "h", None):
            self.lib.rsn_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, fn: str, rc: int):
        if rc != RSN_OK:
            raise RsnError(fn, rc, self.lib.rsn_last_error(self.h).decode())

    # ---- setup ------------------------------------------------------------
    def set_junction(self, j) -> "Context":
        self._check("rsn_set_grid", self.lib.rsn_set_grid(self.h, j.nx, j.ny, j.nz, float(j.h), j.fd_half_order))
        self.N = j.N
        self.set_potential(j.v_loc)
        gl = np.ascontiguousarray(j.gamma_l, dtype=np.float64)
        gr = np.ascontiguousarray(j.gamma_r, dtype=np.float64)
        self._check("rsn_set_cap", self.lib.rsn_set_cap(self.h, _ptr(gl), _ptr(gr)))
        off = np.ascontiguousarray(j.proj_offsets, dtype=np.int64)
        idx = np.ascontiguousarray(j.proj_idx, dtype=np.int32)
        val = np.ascontiguousarray(j.proj_val, dtype=np.float64)
        ekb = np.ascontiguousarray(j.proj_ekb, dtype=np.float64)
        self._check("rsn_set_projectors",
                    self.lib.rsn_set_projectors(self.h, int(ekb.size), _ptr(off), _ptr(idx), _ptr(val), _ptr(ekb)))
        self.junction = j
        return self

    def set_potential(self, v_loc) -> None:
        v = np.ascontiguousarray(v_loc, dtype=np.float64)
        if v.size != self.N:
            raise ValueError("v_loc has the wrong size")
        self._check("rsn_set_potential", self.lib.rsn_set_potential(self.h, _ptr(v)))

    def set_tiling(self, TY: int = 0, Lz: int = 0, ppt: int = 0) -> None:
        self._check("rsn_set_tiling", self.lib.rsn_set_tiling(self.h, TY, Lz, ppt))

    # ---- compute ----------------------------------------------------------
    def apply(self, E: Sequence[float], x, precision: int = RSN_FP64):
        """y[k] = A(E[k]) x[k]; x is a CUDA tensor (n, N), complex128 or complex64."""
        torch = _torch()
        E = np.ascontiguousarray(E, dtype=np.float64)
        want = torch.complex128 if precision == RSN_FP64 else torch.complex64
        if x.dtype != want or not x.is_cuda or not x.is_contiguous() or x.shape != (E.size, self.N):
            raise ValueError("x must be a contiguous CUDA tensor of shape (len(E), N) and matching dtype")
        y = torch.empty_like(x)
        self._check("rsn_apply", self.lib.rsn_apply(self.h, precision, int(E.size), _ptr(E), x.data_ptr(),
                                                    y.data_ptr()))
        return y

    def solve_columns(self, E: Sequence[float], cols: Sequence[int], opts: Optional[SolverOpts] = None,
                      raise_on_noconv: bool = True):
        """Columns G(E[e]) e_{cols[c]} as a CUDA complex128 tensor (n_e, n_cols, N)."""
        torch = _torch()
        opts = opts or default_opts()
        E = np.ascontiguousarray(E, dtype=np.float64)
        cols = np.ascontiguousarray(cols, dtype=np.int32)
        x = torch.empty((E.size, cols.size, self.N), dtype=torch.complex128, device=f"cuda:{self.device}")
        iters = np.zeros(E.size * cols.size, np.int32)
        relres = np.zeros(E.size * cols.size, np.float64)
        rc = self.lib.rsn_solve_columns(self.h, int(E.size), _ptr(E), int(cols.size), _ptr(cols), ct.byref(opts),
                                        x.data_ptr(), _ptr(iters), _ptr(relres))
        if rc != RSN_OK and (raise_on_noconv or rc not in (RSN_ENOCONV, RSN_ETIMEOUT, RSN_EBREAKDOWN)):
            self._check("rsn_solve_columns", rc)
        return x, iters.reshape(E.size, cols.size), relres.reshape(E.size, cols.size)

    def solve_columns_shifted(self, E: Sequence[float], cols: Sequence[int], opts: Optional[SolverOpts] = None):
        """Columns at every energy from one Krylov space per column (FP64):
        (CUDA complex128 tensor (n_e, n_cols, N), iterations, recurrence residuals)."""
        torch = _torch()
        opts = opts or default_opts()
        E = np.ascontiguousarray(E, dtype=np.float64)
        cols = np.ascontiguousarray(cols, dtype=np.int32)
        x = torch.empty((E.size, cols.size, self.N), dtype=torch.complex128, device=f"cuda:{self.device}")
        iters = np.zeros(E.size * cols.size, np.int32)
        relres = np.zeros(E.size * cols.size, np.float64)
        self._check("rsn_solve_columns_shifted",
                    self.lib.rsn_solve_columns_shifted(self.h, int(E.size), _ptr(E), int(cols.size), _ptr(cols),
                                                       ct.byref(opts), x.data_ptr(), _ptr(iters), _ptr(relres)))
        return x, iters.reshape(E.size, cols.size), relres.reshape(E.size, cols.size)

    def transmission_shifted(self, E: Sequence[float], cols: Optional[Sequence[int]] = None,
                             opts: Optional[SolverOpts] = None, return_iters: bool = False):
        """T(E) over an energy window by shifted COCG (FP64)."""
        opts = opts or default_opts()
        E = np.ascontiguousarray(E, dtype=np.float64)
        if cols is None:
            cols = self.junction.right_columns()
        cols = np.ascontiguousarray(cols, dtype=np.int32)
        T = np.zeros(E.size, np.float64)
        iters = np.zeros(E.size * cols.size, np.int32)
        self._check("rsn_transmission_shifted",
                    self.lib.rsn_transmission_shifted(self.h, int(E.size), _ptr(E), int(cols.size), _ptr(cols),
                                                      ct.byref(opts), _ptr(T), _ptr(iters)))
        return (T, iters.reshape(E.size, cols.size)) if return_iters else T

    def solve_columns_block(self, E: Sequence[float], cols: Sequence[int], block: int = 16,
                            tol_inner: float = 0.0, opts: Optional[SolverOpts] = None,
                            raise_on_noconv: bool = True):
        """Columns by block COCG (blocks of ``block`` columns of one energy share one
        Krylov space; FP32 block recurrence under FP64 refinement): (CUDA complex128
        tensor (n_e, n_cols, N), T partials (n_e, n_cols), operator applications,
        relative residuals)."""
        torch = _torch()
        opts = opts or default_opts(RSN_MIXED)
        E = np.ascontiguousarray(E, dtype=np.float64)
        cols = np.ascontiguousarray(cols, dtype=np.int32)
        x = torch.empty((E.size, cols.size, self.N), dtype=torch.complex128, device=f"cuda:{self.device}")
        tc = np.zeros(E.size * cols.size, np.float64)
        iters = np.zeros(E.size * cols.size, np.int32)
        relres = np.zeros(E.size * cols.size, np.float64)
        rc = self.lib.rsn_solve_columns_block(self.h, int(E.size), _ptr(E), int(cols.size), _ptr(cols), int(block),
                                              float(tol_inner), ct.byref(opts), x.data_ptr(), _ptr(tc),
                                              _ptr(iters), _ptr(relres))
        if rc != RSN_OK and (raise_on_noconv or rc not in (RSN_ENOCONV, RSN_ETIMEOUT)):
            self._check("rsn_solve_columns_block", rc)
        sh = (E.size, cols.size)
        return x, tc.reshape(sh), iters.reshape(sh), relres.reshape(sh)

    def transmission_block(self, E: Sequence[float], cols: Optional[Sequence[int]] = None, block: int = 16,
                           tol_inner: float = 0.0, opts: Optional[SolverOpts] = None, return_cols: bool = False):
        """T(E) from block COCG columns; with ``return_cols`` also the per-column T
        partials and operator applications, each (n_e, n_cols)."""
        opts = opts or default_opts(RSN_MIXED)
        E = np.ascontiguousarray(E, dtype=np.float64)
        if cols is None:
            cols = self.junction.right_columns()
        cols = np.ascontiguousarray(cols, dtype=np.int32)
        T = np.zeros(E.size, np.float64)
        tc = np.zeros(E.size * cols.size, np.float64)
        iters = np.zeros(E.size * cols.size, np.int32)
        self._check("rsn_transmission_block",
                    self.lib.rsn_transmission_block(self.h, int(E.size), _ptr(E), int(cols.size), _ptr(cols),
                                                    int(block), float(tol_inner), ct.byref(opts), _ptr(T),
                                                    _ptr(tc), _ptr(iters)))
        sh = (E.size, cols.size)
        return (T, tc.reshape(sh), iters.reshape(sh)) if return_cols else T

    def transmission(self, E: Sequence[float], cols: Optional[Sequence[int]] = None,
                     opts: Optional[SolverOpts] = None) -> np.ndarray:
        opts = opts or default_opts()
        E = np.ascontiguousarray(E, dtype=np.float64)
        if cols is None:
            cols = self.junction.right_columns()
        cols = np.ascontiguousarray(cols, dtype=np.int32)
        T = np.zeros(E.size, np.float64)
        self._check("rsn_transmission", self.lib.rsn_transmission(self.h, int(E.size), _ptr(E), int(cols.size),
                                                                  _ptr(cols), ct.byref(opts), _ptr(T)))
        return T

    def transmission_vjp(self, E: Sequence[float], T_bar: Sequence[float], cols: Optional[Sequence[int]] = None,
                         opts: Optional[SolverOpts] = None, dV_out=None):
        """(T(E), dV) with dV[r] = sum_e T_bar[e] dT(E[e])/dV_loc(r).

        ``dV_out``: optional CUDA float64 tensor (N,) to receive dV on the device;
        otherwise a host array is returned."""
        opts = opts or default_opts()
        E = np.ascontiguousarray(E, dtype=np.float64)
        Tb = np.ascontiguousarray(T_bar, dtype=np.float64)
        if cols is None:
            cols = self.junction.right_columns()
        cols = np.ascontiguousarray(cols, dtype=np.int32)
        T = np.zeros(E.size, np.float64)
        if dV_out is not None:
            dptr, isdev = dV_out.data_ptr(), 1
            dV = dV_out
        else:
            dV = np.zeros(self.N, np.float64)
            dptr, isdev = _ptr(dV), 0
        self._check("rsn_transmission_vjp",
                    self.lib.rsn_transmission_vjp(self.h, int(E.size), _ptr(E), int(cols.size), _ptr(cols),
                                                  ct.byref(opts), _ptr(Tb), dptr, isdev, _ptr(T)))
        return T, dV

    def transmission_keep(self, E: Sequence[float], cols: Sequence[int], opts: Optional[SolverOpts] = None):
        """(T(E), forward columns as a CUDA complex128 tensor (n_e, n_cols, N))."""
        torch = _torch()
        opts = opts or default_opts()
        E = np.ascontiguousarray(E, dtype=np.float64)
        cols = np.ascontiguousarray(cols, dtype=np.int32)
        x = torch.empty((E.size, cols.size, self.N), dtype=torch.complex128, device=f"cuda:{self.device}")
        T = np.zeros(E.size, np.float64)
        self._check("rsn_transmission_keep",
                    self.lib.rsn_transmission_keep(self.h, int(E.size), _ptr(E), int(cols.size), _ptr(cols),
                                                   ct.byref(opts), x.data_ptr(), _ptr(T)))
        return T, x

    def transmission_vjp_reuse(self, E: Sequence[float], T_bar: Sequence[float], cols: Sequence[int], x,
                               opts: Optional[SolverOpts] = None, dV_out=None):
        """dV = sum_e T_bar[e] dT(E[e])/dV_loc from the forward columns ``x`` of
        ``transmission_keep`` (adjoint solves only)."""
        opts = opts or default_opts()
        E = np.ascontiguousarray(E, dtype=np.float64)
        Tb = np.ascontiguousarray(T_bar, dtype=np.float64)
        cols = np.ascontiguousarray(cols, dtype=np.int32)
        if x.shape != (E.size, cols.size, self.N) or not x.is_contiguous():
            raise ValueError("x must be the (n_e, n_cols, N) columns of transmission_keep")
        if dV_out is not None:
            dptr, isdev, dV = dV_out.data_ptr(), 1, dV_out
        else:
            dV = np.zeros(self.N, np.float64)
            dptr, isdev = _ptr(dV), 0
        self._check("rsn_transmission_vjp_reuse",
                    self.lib.rsn_transmission_vjp_reuse(self.h, int(E.size), _ptr(E), int(cols.size), _ptr(cols),
                                                        ct.byref(opts), x.data_ptr(), _ptr(Tb), dptr, isdev))
        return dV

    def landauer_current(self, E: Sequence[float], T: Sequence[float], V: Sequence[float], E_F: float = 0.0,
                         kT: float = 0.0) -> np.ndarray:
        """I(V) of Eq. Landauer in atomic units (e E_h / hbar) from T on the grid E."""
        E = np.ascontiguousarray(E, dtype=np.float64)
        T = np.ascontiguousarray(T, dtype=np.float64)
        V = np.ascontiguousarray(np.atleast_1d(V), dtype=np.float64)
        if T.size != E.size:
            raise ValueError("T must have one value per energy")
        I = np.zeros(V.size, np.float64)
        self._check("rsn_landauer_current",
                    self.lib.rsn_landauer_current(self.h, int(E.size), _ptr(E), _ptr(T), int(V.size), _ptr(V),
                                                  float(E_F), float(kT), _ptr(I)))
        return I

    def kernel_stats(self, kind: int):
        """(launches, ms, algorithmic bytes) of kind 0 (COCG operator) / 1 (COCG update)."""
        la, ms, by = ct.c_int64(), ct.c_double(), ct.c_double()
        self._check("rsn_kernel_stats", self.lib.rsn_kernel_stats(self.h, kind, ct.byref(la), ct.byref(ms),
                                                                  ct.byref(by)))
        return {"launches": la.value, "ms": ms.value, "bytes": by.value}

    def bench_kernel(self, precision: int, kind: int, nslots: int, reps: int = 20):
        """(ms per launch, algorithmic bytes per launch) of one COCG kernel in isolation."""
        ms, by = ct.c_double(), ct.c_double()
        self._check("rsn_bench_kernel", self.lib.rsn_bench_kernel(self.h, precision, kind, nslots, reps,
                                                                  ct.byref(ms), ct.byref(by)))
        return ms.value, by.value

    def autotune(self, precision: int, nslots: int):
        """Pick the fastest operator-kernel tiling; returns the choice and its GB/s."""
        ty, lz, ppt, tma, gbs = ct.c_int(), ct.c_int(), ct.c_int(), ct.c_int(), ct.c_double()
        self._check("rsn_autotune", self.lib.rsn_autotune(self.h, precision, nslots, ct.byref(ty), ct.byref(lz),
                                                          ct.byref(ppt), ct.byref(tma), ct.byref(gbs)))
        return {"TY": ty.value, "Lz": lz.value, "ppt": ppt.value, "tma": tma.value, "gbs": gbs.value}

    def last_stats(self):
        it, sw, la, ms, fb = ct.c_int64(), ct.c_int64(), ct.c_int64(), ct.c_double(), ct.c_int64()
        self._check("rsn_last_stats", self.lib.rsn_last_stats(self.h, ct.byref(it), ct.byref(sw), ct.byref(la),
                                                              ct.byref(ms), ct.byref(fb)))
        return {"krylov_iters": it.value, "sweeps": sw.value, "launches": la.value, "gpu_ms": ms.value,
                "fp64_fallbacks": fb.value}


def batch_transmission(contexts: Sequence["Context"], energies: Sequence[Sequence[float]],
                       cols: Optional[Sequence[Optional[Sequence[int]]]] = None,
                       opts: Optional[SolverOpts] = None) -> List[np.ndarray]:
    """T(E) of several junctions at once (``rsn_batch_transmission``).

    ``contexts[k]`` holds junction k; it gets ``energies[k]`` and ``cols[k]``
    (default: its right-lead columns).  Returns one T array per junction;
    raises RsnError naming the first junction that failed.
    """
    lib = load()
    n = len(contexts)
    if len(energies) != n or (cols is not None and len(cols) != n):
        raise ValueError("one energy list and one column list per context")
    opts = opts or default_opts(RSN_MIXED)
    Es = [np.ascontiguousarray(e, dtype=np.float64) for e in energies]
    Cs = [np.ascontiguousarray(ctx.junction.right_columns() if (cols is None or cols[k] is None) else cols[k],
                               dtype=np.int32) for k, ctx in enumerate(contexts)]
    Ts = [np.zeros(e.size, np.float64) for e in Es]
    ctxs = (ct.c_void_p * max(n, 1))(*[c.h.value for c in contexts])
    n_e = (ct.c_int * max(n, 1))(*[e.size for e in Es])
    n_c = (ct.c_int * max(n, 1))(*[c.size for c in Cs])
    Ep = (ct.c_void_p * max(n, 1))(*[_ptr(e) for e in Es])
    Cp = (ct.c_void_p * max(n, 1))(*[_ptr(c) for c in Cs])
    Tp = (ct.c_void_p * max(n, 1))(*[_ptr(t) for t in Ts])
    st = (ct.c_int * max(n, 1))()
    rc = lib.rsn_batch_transmission(n, ctxs, n_e, Ep, n_c, Cp, ct.byref(opts), Tp, st)
    if rc != RSN_OK:
        bad = [k for k in range(n) if st[k] != RSN_OK]
        k = bad[0] if bad else 0
        msg = lib.rsn_last_error(contexts[k].h).decode() if n else ""
        raise RsnError("rsn_batch_transmission", rc, f"junction {k}: {msg}")
    return Ts

