"""Thin ctypes binding of the FAM C ABI (include/fam.h).

Argument marshalling only: every step of the FAM time step runs in the CUDA
kernels of libfam.so.  The library must have been built
(``python -m paper_2609_26194_b300.build``); loading fails loudly otherwise.

States are numpy arrays (host) or torch CUDA tensors (device) in the layout
U[c, m, j, i] (1D: U[c, m, i]); float64 for precision 64, float32 for 32.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libfam.so")

ADVECTION, BURGERS, EULER, BUCKLEY = 0, 1, 2, 3
PERIODIC, OUTFLOW, REFLECTIVE, INFLOW, FRONT = 0, 1, 2, 3, 4
# 2D tile shapes (cells per CTA in x, y) selectable with the "tile2d" option / tune()
TILES_2D = ((32, 8), (32, 4), (16, 8))
STATUS = {0: "FAM_OK", 1: "FAM_E_INVAL", 2: "FAM_E_NOMEM", 3: "FAM_E_CUDA", 4: "FAM_E_NONPHYSICAL",
          5: "FAM_E_TIMEOUT", 6: "FAM_E_STATE", 7: "FAM_E_UNSUPPORTED"}

# every function declared in include/fam.h
EXPORTS = ("fam_create", "fam_set_option", "fam_set_state", "fam_get_state", "fam_step", "fam_run_steps",
           "fam_run", "fam_sync", "fam_time", "fam_profile", "fam_residual", "fam_oe", "fam_last_error",
           "fam_status_string", "fam_destroy", "fam_alu_peak", "fam_selftest_math", "fam_selftest_int_fp64",
           "fam_batch_create", "fam_batch_set_option", "fam_batch_set_state", "fam_batch_get_state",
           "fam_batch_run", "fam_batch_sync", "fam_batch_times", "fam_batch_info", "fam_batch_tune",
           "fam_batch_last_error", "fam_batch_destroy", "fam_batch2d_create", "fam_batch_tile",
           "fam_step1d_noalloc", "fam_adjoint",
           "fam_run_fixed", "fam_set_bc", "fam_tune", "fam_nonphysical_traces", "fam_batch_health",
           "fam_set_bc_split", "fam_set_bc_front", "fam_rejected_steps", "fam_batch_rejected_steps")


class FamError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{STATUS.get(code, code)}: {msg}")
        self.code = code


class Grid(ctypes.Structure):
    _fields_ = [("d", ctypes.c_int), ("nx", ctypes.c_int), ("ny", ctypes.c_int),
                ("x0", ctypes.c_double), ("x1", ctypes.c_double),
                ("y0", ctypes.c_double), ("y1", ctypes.c_double)]


_lib = None


def lib() -> ctypes.CDLL:
    """Load libfam.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise FileNotFoundError(f"{LIB_PATH} missing: build it with `python -m paper_2609_26194_b300.build`")
        L = ctypes.CDLL(LIB_PATH)
        vp, dp, i, d, l = ctypes.c_void_p, ctypes.POINTER(ctypes.c_double), ctypes.c_int, ctypes.c_double, ctypes.c_long
        L.fam_create.argtypes = [ctypes.POINTER(vp), ctypes.POINTER(Grid), i, i, i, d, i, vp]
        L.fam_set_option.argtypes = [vp, ctypes.c_char_p, d]
        L.fam_set_state.argtypes = [vp, vp, i]
        L.fam_get_state.argtypes = [vp, vp, i]
        L.fam_step.argtypes = [vp, d]
        L.fam_run_steps.argtypes = [vp, l, d]
        L.fam_run.argtypes = [vp, d, d, l, ctypes.POINTER(l)]
        L.fam_sync.argtypes = [vp]
        L.fam_time.argtypes = [vp, dp, dp, ctypes.POINTER(l)]
        L.fam_profile.argtypes = [vp, dp, ctypes.POINTER(l)]
        L.fam_residual.argtypes = [vp, vp, vp, i]
        L.fam_oe.argtypes = [vp, d, vp, vp, i]
        L.fam_adjoint.argtypes = [vp, l, d, i, vp, vp, vp, i]
        L.fam_run_fixed.argtypes = [vp, l, dp]
        L.fam_set_bc.argtypes = [vp, i, i, dp]
        L.fam_set_bc_split.argtypes = [vp, i, ctypes.c_double, dp]
        L.fam_set_bc_front.argtypes = [vp, i, ctypes.c_double, ctypes.c_double, ctypes.c_double, dp, dp]
        L.fam_tune.argtypes = [vp, d, i, ctypes.c_char_p, ctypes.POINTER(i)]
        L.fam_nonphysical_traces.argtypes = [vp, ctypes.POINTER(ctypes.c_ulonglong)]
        L.fam_rejected_steps.argtypes = [vp, ctypes.POINTER(ctypes.c_ulonglong)]
        L.fam_last_error.argtypes = [vp]
        L.fam_last_error.restype = ctypes.c_char_p
        L.fam_status_string.argtypes = [i]
        L.fam_status_string.restype = ctypes.c_char_p
        L.fam_destroy.argtypes = [vp]
        L.fam_destroy.restype = None
        L.fam_alu_peak.argtypes = [i, dp]
        L.fam_selftest_math.argtypes = [dp, i, dp, dp, dp]
        L.fam_selftest_int_fp64.argtypes = [dp, dp, i, dp]
        for name in EXPORTS:
            if name not in ("fam_last_error", "fam_status_string", "fam_destroy"):
                getattr(L, name).restype = ctypes.c_int
        _lib = L
    return _lib


def _is_torch(x) -> bool:
    return type(x).__module__.startswith("torch")


class Solver:
    """One FAM problem on the GPU (wraps a fam_t handle)."""

    def __init__(self, d: int, nx: int, ny: int = 1, box=(0.0, 1.0, 0.0, 1.0), k: int = 5,
                 equation: int = EULER, bc: int = PERIODIC, gamma: float = 1.4, precision: int = 64,
                 stream: int | None = None, **options):
        self.d, self.nx, self.ny, self.k = d, nx, (ny if d == 2 else 1), k
        self.equation, self.precision = equation, precision
        self.ncomp = d + 2 if equation == EULER else 1
        self.nmom = d + 1
        self.dtype = np.float64 if precision == 64 else np.float32
        g = Grid(d, nx, self.ny, box[0], box[1], box[2], box[3])
        h = ctypes.c_void_p()
        rc = lib().fam_create(ctypes.byref(h), ctypes.byref(g), k, equation, bc, gamma, precision,
                              ctypes.c_void_p(stream or 0))
        if rc != 0:
            raise FamError(rc, "fam_create failed")
        self._h = h
        for key, val in options.items():
            self.set_option(key, val)

    @property
    def shape(self) -> tuple:
        if self.d == 1:
            return (self.ncomp, self.nmom, self.nx)
        return (self.ncomp, self.nmom, self.ny, self.nx)

    def _check(self, rc: int):
        if rc != 0:
            raise FamError(rc, lib().fam_last_error(self._h).decode())

    def close(self):
        if getattr(self, "_h", None):
            lib().fam_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def set_option(self, key: str, value: float):
        self._check(lib().fam_set_option(self._h, key.encode(), float(value)))

    @staticmethod
    def _state4(v):
        arr = (ctypes.c_double * 4)(*([float(x) for x in v] + [0.0] * (4 - len(v))))
        return ctypes.cast(arr, ctypes.POINTER(ctypes.c_double)), arr

    def set_bc(self, side: int, bc: int, inflow=None):
        """Per-side condition: side 0 x-low, 1 x-high, 2 y-low, 3 y-high."""
        st, _keep = (None, None) if inflow is None else self._state4(inflow)
        self._check(lib().fam_set_bc(self._h, int(side), int(bc), st))

    def set_bc_split(self, side: int, position: float, state):
        """Ghost cells of the side whose nearest interior cell's centre along
        the side lies below position hold state (fam_set_bc_split)."""
        st, _keep = self._state4(state)
        self._check(lib().fam_set_bc_split(self._h, int(side), float(position), st))

    def set_bc_front(self, side: int, a: float, b: float, c: float, behind, ahead):
        """Front condition of a y-side: behind where x < a + b y + c t, ahead
        elsewhere (fam_set_bc_front)."""
        pb, _kb = self._state4(behind)
        pa, _ka = self._state4(ahead)
        self._check(lib().fam_set_bc_front(self._h, int(side), float(a), float(b), float(c), pb, pa))

    def _buf(self, U):
        if _is_torch(U):
            if tuple(U.shape) != self.shape or not U.is_contiguous():
                raise ValueError(f"tensor must be contiguous with shape {self.shape}")
            want = "torch.float64" if self.precision == 64 else "torch.float32"
            if str(U.dtype) != want:
                raise TypeError(f"tensor dtype must be {want}")
            return ctypes.c_void_p(U.data_ptr()), (1 if U.is_cuda else 0), U
        A = np.ascontiguousarray(U, dtype=self.dtype)
        if A.shape != self.shape:
            raise ValueError(f"array shape {A.shape} != {self.shape}")
        return ctypes.c_void_p(A.ctypes.data), 0, A

    def set_state(self, U):
        p, dev, keep = self._buf(U)
        self._check(lib().fam_set_state(self._h, p, dev))

    def get_state(self, out=None):
        if out is None:
            out = np.empty(self.shape, dtype=self.dtype)
        p, dev, keep = self._buf(out)
        self._check(lib().fam_get_state(self._h, p, dev))
        return out

    def step(self, cfl: float):
        self._check(lib().fam_step(self._h, float(cfl)))

    def run_steps(self, nsteps: int, cfl: float):
        self._check(lib().fam_run_steps(self._h, int(nsteps), float(cfl)))

    def run(self, T: float, cfl: float, max_steps: int = 0) -> int:
        n = ctypes.c_long()
        self._check(lib().fam_run(self._h, float(T), float(cfl), int(max_steps), ctypes.byref(n)))
        return n.value

    def sync(self):
        self._check(lib().fam_sync(self._h))

    def tune(self, cfl: float, probe_steps: int = 2, cache_path: str | None = None) -> int:
        """Pick the fastest 2D tile shape, with the final stage and OE split or
        fused, on the current state; returns the tile's index into TILES_2D
        and leaves the split / fused choice in ``self.fused_oe`` (the state and
        clock are restored)."""
        c = ctypes.c_int()
        self._check(lib().fam_tune(self._h, float(cfl), int(probe_steps),
                                   cache_path.encode() if cache_path else None, ctypes.byref(c)))
        self.fused_oe = c.value // 3
        return c.value % 3

    def run_fixed(self, dts):
        d = np.ascontiguousarray(dts, dtype=np.float64)
        self._check(lib().fam_run_fixed(self._h, d.size, d.ctypes.data_as(ctypes.POINTER(ctypes.c_double))))

    def record_steps(self, nsteps: int, cfl: float) -> np.ndarray:
        """Take nsteps CFL steps one by one and return the step sizes used."""
        out = np.empty(nsteps)
        self.run_steps(0, cfl)  # make the device step size current without stepping
        for q in range(nsteps):
            out[q] = self.time()[1]
            self.step(cfl)
        return out

    def time(self) -> tuple[float, float, int]:
        t, dt, s = ctypes.c_double(), ctypes.c_double(), ctypes.c_long()
        self._check(lib().fam_time(self._h, ctypes.byref(t), ctypes.byref(dt), ctypes.byref(s)))
        return t.value, dt.value, s.value

    def rejected_steps(self) -> int:
        """Steps discarded and retried with half the step size (safeguard)."""
        n = ctypes.c_ulonglong()
        self._check(lib().fam_rejected_steps(self._h, ctypes.byref(n)))
        return n.value

    def nonphysical_traces(self) -> int:
        """Face quadrature points whose Rusanov trace had no spectral radius,
        summed over the residual evaluations since set_state()."""
        n = ctypes.c_ulonglong()
        self._check(lib().fam_nonphysical_traces(self._h, ctypes.byref(n)))
        return n.value

    def profile(self) -> tuple[list, int]:
        """(ms per kernel [stage1, stage2, stage3, oe], profiled steps)."""
        ms = (ctypes.c_double * 4)()
        n = ctypes.c_long()
        self._check(lib().fam_profile(self._h, ms, ctypes.byref(n)))
        return list(ms), n.value

    def residual(self, U):
        p, dev, keep = self._buf(U)
        out = np.empty(self.shape, dtype=self.dtype) if not dev else keep.new_empty(self.shape)
        q, dev2, keep2 = self._buf(out)
        self._check(lib().fam_residual(self._h, p, q, dev))
        return out

    def adjoint(self, U0, dJdUT, nsteps: int, cfl: float, ckpt_every: int = 20):
        """dJ/dU0 of a terminal functional with dJ/dU_T given (fixed step sizes)."""
        p0, dev, k0 = self._buf(U0)
        pg, dev2, kg = self._buf(dJdUT)
        if dev != dev2:
            raise ValueError("U0 and dJdUT must both be host or both be device buffers")
        out = np.empty(self.shape, dtype=self.dtype) if not dev else k0.new_empty(self.shape)
        q, _, keep = self._buf(out)
        self._check(lib().fam_adjoint(self._h, int(nsteps), float(cfl), int(ckpt_every), p0, pg, q, dev))
        return out

    def oe(self, dt: float, U):
        p, dev, keep = self._buf(U)
        out = np.empty(self.shape, dtype=self.dtype) if not dev else keep.new_empty(self.shape)
        q, dev2, keep2 = self._buf(out)
        self._check(lib().fam_oe(self._h, float(dt), p, q, dev))
        return out


def alu_peak(precision: int = 64) -> float:
    v = ctypes.c_double()
    rc = lib().fam_alu_peak(precision, ctypes.byref(v))
    if rc != 0:
        raise FamError(rc, "fam_alu_peak failed")
    return v.value


def selftest_math(x: np.ndarray):
    x = np.ascontiguousarray(x, dtype=np.float64)
    outs = [np.empty_like(x) for _ in range(3)]
    dp = ctypes.POINTER(ctypes.c_double)
    rc = lib().fam_selftest_math(x.ctypes.data_as(dp), x.size, *(o.ctypes.data_as(dp) for o in outs))
    if rc != 0:
        raise FamError(rc, "fam_selftest_math failed")
    return tuple(outs)


def selftest_int_fp64(a: np.ndarray, b: np.ndarray) -> np.ndarray:
    """The library's integer-pipe binary64 product a * b, elementwise."""
    a = np.ascontiguousarray(a, dtype=np.float64)
    b = np.ascontiguousarray(b, dtype=np.float64)
    if a.shape != b.shape:
        raise ValueError("a and b differ in shape")
    prod = np.empty_like(a)
    dp = ctypes.POINTER(ctypes.c_double)
    rc = lib().fam_selftest_int_fp64(a.ctypes.data_as(dp), b.ctypes.data_as(dp), a.size, prod.ctypes.data_as(dp))
    if rc != 0:
        raise FamError(rc, "fam_selftest_int_fp64 failed")
    return prod


class Batch:
    """Many independent problems advanced in one persistent launch (fam_batch_t).

    1D: Batch(nx, k, ...) -- instance i has nx[i] cells on [x0, x1].
    2D (Euler): Batch(nx, k, ny=ny, ...) -- instance i has nx[i] x ny[i]
    cells on [x0, x1] x [y0, y1].  States are lists of per-instance arrays of
    shape (ncomp, 2, nx) or (4, 3, ny, nx)."""

    def __init__(self, nx, k, x0: float = 0.0, x1: float = 1.0, equation: int = EULER, bc: int = OUTFLOW,
                 gamma: float = 1.4, precision: int = 64, stream: int | None = None, ny=None,
                 y0: float = 0.0, y1: float = 1.0):
        self.nx = [int(v) for v in nx]
        self.k = [int(v) for v in k]
        self.d = 1 if ny is None else 2
        self.ny = [1] * len(self.nx) if ny is None else [int(v) for v in ny]
        if len(self.nx) != len(self.k) or len(self.ny) != len(self.nx):
            raise ValueError("nx, ny and k must have the same length")
        self.n = len(self.nx)
        self.ncomp = (self.d + 2) if equation == EULER else 1
        self.nmom = self.d + 1
        self.precision = precision
        self.dtype = np.float64 if precision == 64 else np.float32
        L = lib()
        _batch_sigs(L)
        h = ctypes.c_void_p()
        anx = (ctypes.c_int * self.n)(*self.nx)
        ak = (ctypes.c_int * self.n)(*self.k)
        if self.d == 1:
            rc = L.fam_batch_create(ctypes.byref(h), self.n, anx, ak, x0, x1, equation, bc, gamma, precision,
                                    ctypes.c_void_p(stream or 0))
        else:
            any_ = (ctypes.c_int * self.n)(*self.ny)
            rc = L.fam_batch2d_create(ctypes.byref(h), self.n, anx, any_, ak, x0, x1, y0, y1, equation, bc, gamma,
                                      precision, ctypes.c_void_p(stream or 0))
        if rc != 0:
            raise FamError(rc, "fam_batch_create failed")
        self._h = h

    def _shape(self, i: int) -> tuple:
        if self.d == 1:
            return (self.ncomp, 2, self.nx[i])
        return (self.ncomp, 3, self.ny[i], self.nx[i])

    def _check(self, rc):
        if rc != 0:
            raise FamError(rc, lib().fam_batch_last_error(self._h).decode())

    def close(self):
        if getattr(self, "_h", None):
            lib().fam_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_option(self, key: str, value: float):
        self._check(lib().fam_batch_set_option(self._h, key.encode(), float(value)))

    def pack(self, states) -> np.ndarray:
        parts = []
        for i, U in enumerate(states):
            U = np.ascontiguousarray(U, dtype=self.dtype)
            if U.shape != self._shape(i):
                raise ValueError(f"instance state shape {U.shape} != {self._shape(i)}")
            parts.append(U.reshape(-1))
        return np.ascontiguousarray(np.concatenate(parts))

    def unpack(self, flat) -> list:
        out, o = [], 0
        for i in range(self.n):
            shp = self._shape(i)
            m = int(np.prod(shp))
            out.append(flat[o:o + m].reshape(shp))
            o += m
        return out

    def set_state(self, states):
        flat = self.pack(states)
        self._check(lib().fam_batch_set_state(self._h, ctypes.c_void_p(flat.ctypes.data), 0))

    def get_state(self) -> list:
        flat = np.empty(sum(int(np.prod(self._shape(i))) for i in range(self.n)), dtype=self.dtype)
        self._check(lib().fam_batch_get_state(self._h, ctypes.c_void_p(flat.ctypes.data), 0))
        return self.unpack(flat)

    def run(self, nsteps: int, cfl: float):
        self._check(lib().fam_batch_run(self._h, int(nsteps), float(cfl)))

    def sync(self):
        self._check(lib().fam_batch_sync(self._h))

    def times(self):
        t = np.empty(self.n)
        dt = np.empty(self.n)
        st = (ctypes.c_long * self.n)()
        dp = ctypes.POINTER(ctypes.c_double)
        self._check(lib().fam_batch_times(self._h, t.ctypes.data_as(dp), dt.ctypes.data_as(dp), st))
        return t, dt, np.array(st[:], dtype=np.int64)

    def health(self):
        """Per instance: (trace counts, status codes, first flagged step)."""
        nt = (ctypes.c_ulonglong * self.n)()
        st = (ctypes.c_int * self.n)()
        bs = (ctypes.c_long * self.n)()
        self._check(lib().fam_batch_health(self._h, nt, st, bs))
        return (np.array(nt[:], dtype=np.int64), np.array(st[:], dtype=np.int32),
                np.array(bs[:], dtype=np.int64))

    def rejected_steps(self) -> np.ndarray:
        """Per instance: attempts the BP/PP safeguard discarded (each retried
        with half the step size) since the state was set."""
        c = (ctypes.c_ulonglong * self.n)()
        self._check(lib().fam_batch_rejected_steps(self._h, c))
        return np.array(c[:], dtype=np.int64)

    def info(self) -> dict:
        tx, g, nt, nc = ctypes.c_int(), ctypes.c_int(), ctypes.c_long(), ctypes.c_long()
        self._check(lib().fam_batch_info(self._h, ctypes.byref(tx), ctypes.byref(g), ctypes.byref(nt),
                                         ctypes.byref(nc)))
        ty = ctypes.c_int()
        self._check(lib().fam_batch_tile(self._h, ctypes.byref(tx), ctypes.byref(ty)))
        return {"tile_x": tx.value, "tile_y": ty.value, "grid": g.value, "tiles": nt.value, "cells": nc.value}

    def tune(self, cfl: float, probe_steps: int = 3, cache_path: str | None = None) -> tuple[int, int]:
        tx, b = ctypes.c_int(), ctypes.c_int()
        self._check(lib().fam_batch_tune(self._h, float(cfl), int(probe_steps),
                                         cache_path.encode() if cache_path else None, ctypes.byref(tx),
                                         ctypes.byref(b)))
        return tx.value, b.value


_batch_ready = False


def _batch_sigs(L):
    global _batch_ready
    if _batch_ready:
        return
    vp, dp, i, d, l = ctypes.c_void_p, ctypes.POINTER(ctypes.c_double), ctypes.c_int, ctypes.c_double, ctypes.c_long
    ip = ctypes.POINTER(ctypes.c_int)
    L.fam_batch_create.argtypes = [ctypes.POINTER(vp), i, ip, ip, d, d, i, i, d, i, vp]
    L.fam_batch2d_create.argtypes = [ctypes.POINTER(vp), i, ip, ip, ip, d, d, d, d, i, i, d, i, vp]
    L.fam_batch_tile.argtypes = [vp, ip, ip]
    L.fam_batch_set_option.argtypes = [vp, ctypes.c_char_p, d]
    L.fam_batch_set_state.argtypes = [vp, vp, i]
    L.fam_batch_get_state.argtypes = [vp, vp, i]
    L.fam_batch_run.argtypes = [vp, l, d]
    L.fam_batch_sync.argtypes = [vp]
    L.fam_batch_times.argtypes = [vp, dp, dp, ctypes.POINTER(l)]
    L.fam_batch_info.argtypes = [vp, ip, ip, ctypes.POINTER(l), ctypes.POINTER(l)]
    L.fam_batch_tune.argtypes = [vp, d, i, ctypes.c_char_p, ip, ip]
    L.fam_batch_health.argtypes = [vp, ctypes.POINTER(ctypes.c_ulonglong), ip, ctypes.POINTER(l)]
    L.fam_batch_rejected_steps.argtypes = [vp, ctypes.POINTER(ctypes.c_ulonglong)]
    L.fam_batch_last_error.argtypes = [vp]
    L.fam_batch_last_error.restype = ctypes.c_char_p
    L.fam_batch_destroy.argtypes = [vp]
    L.fam_batch_destroy.restype = None
    for name in ("fam_batch_create", "fam_batch2d_create", "fam_batch_set_option", "fam_batch_set_state",
                 "fam_batch_get_state", "fam_batch_run", "fam_batch_sync", "fam_batch_times", "fam_batch_info",
                 "fam_batch_tune", "fam_batch_tile", "fam_batch_health", "fam_batch_rejected_steps"):
        getattr(L, name).restype = ctypes.c_int
    _batch_ready = True


def step1d_noalloc(U_in, U_out, nx: int, k: int, x0: float = 0.0, x1: float = 1.0, equation: int = EULER,
                   bc: int = PERIODIC, gamma: float = 1.4, cfl: float = 0.3, stream: int | None = None,
                   return_dt: bool = True) -> float | None:
    """One 1D time step from U_in to U_out (contiguous CUDA tensors of shape
    (ncomp, 2, nx), float64 or float32) without any device allocation by the
    library: its intermediate states live in a fixed static device array
    (at most FAM_NOALLOC_MAX_CELLS = 16384 cells).  Calls share that array,
    so calls whose GPU work may overlap must be serialised by the caller.
    The call waits for its step and raises on a non-physical state.  stream
    defaults to torch's current stream."""
    ncomp = 3 if equation == EULER else 1
    for name, t in (("U_in", U_in), ("U_out", U_out)):
        if not _is_torch(t) or not t.is_cuda:
            raise TypeError(f"{name} must be a CUDA tensor")
        if not t.is_contiguous():
            raise ValueError(f"{name} must be contiguous")
        if tuple(t.shape) != (ncomp, 2, int(nx)):
            raise ValueError(f"{name} has shape {tuple(t.shape)}, expected {(ncomp, 2, int(nx))}")
        if str(t.dtype) not in ("torch.float64", "torch.float32"):
            raise TypeError(f"{name} must be float64 or float32")
    if U_in.dtype != U_out.dtype:
        raise TypeError("U_in and U_out differ in dtype")
    if U_in.device != U_out.device:
        raise ValueError("U_in and U_out are on different devices")
    if stream is None:
        import torch
        stream = torch.cuda.current_stream(U_in.device).cuda_stream
    L = lib()
    _noalloc_sig(L)
    prec = 64 if str(U_in.dtype) == "torch.float64" else 32
    dt = ctypes.c_double()
    import torch
    with torch.cuda.device(U_in.device):
        rc = L.fam_step1d_noalloc(ctypes.c_void_p(U_in.data_ptr()), ctypes.c_void_p(U_out.data_ptr()), int(nx),
                                  float(x0), float(x1), int(k), int(equation), int(bc), float(gamma), prec,
                                  float(cfl), ctypes.byref(dt) if return_dt else None, ctypes.c_void_p(stream))
    if rc != 0:
        raise FamError(rc, "fam_step1d_noalloc failed")
    return dt.value if return_dt else None


def _noalloc_sig(L):
    vp, d, i = ctypes.c_void_p, ctypes.c_double, ctypes.c_int
    L.fam_step1d_noalloc.argtypes = [vp, vp, i, d, d, i, i, i, d, i, d, ctypes.POINTER(d), vp]
    L.fam_step1d_noalloc.restype = ctypes.c_int
