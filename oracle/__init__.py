"""Plain FP64 CPU oracle of the compact FAM time step (ctypes wrapper).

TEST INFRASTRUCTURE ONLY.  The test suite, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` are the only callers.  The oracle is written
in plain C (``fam_oracle.c``) from the paper, Fan & Wu, "Compact
Finite-Average-Moment Schemes with Single-Step Oscillation Elimination for
Hyperbolic Conservation Laws"; it shares no code with the CUDA library.

State layout: ``U[c, m, j, i]`` (component, moment, row, column) as a
C-contiguous float64 array; in one dimension ``U[c, m, i]``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "fam_oracle.c")
_HDR = os.path.join(_HERE, "fam_oracle.h")
_LIB = os.path.join(_HERE, "liboracle.so")

ADVECTION, BURGERS, EULER, BUCKLEY = 0, 1, 2, 3
PERIODIC, OUTFLOW, REFLECTIVE, INFLOW, FRONT = 0, 1, 2, 3, 4
OE_NONE, OE_TYPE1, OE_TYPE2 = 0, 1, 2


def build(force: bool = False) -> str:
    """Compile the oracle into ``oracle/liboracle.so`` (gcc, -O2, OpenMP)."""
    stale = (not os.path.exists(_LIB)) or any(
        os.path.getmtime(p) > os.path.getmtime(_LIB) for p in (_SRC, _HDR))
    if force or stale:
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-fPIC", "-shared", "-fopenmp", "-std=c11",
                               "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


class _Problem(ctypes.Structure):
    _fields_ = [
        ("d", ctypes.c_int), ("nx", ctypes.c_int), ("ny", ctypes.c_int),
        ("x0", ctypes.c_double), ("x1", ctypes.c_double),
        ("y0", ctypes.c_double), ("y1", ctypes.c_double),
        ("k", ctypes.c_int), ("eq", ctypes.c_int), ("bc", ctypes.c_int * 4),
        ("inflow", (ctypes.c_double * 4) * 4),
        ("gamma", ctypes.c_double), ("ax", ctypes.c_double), ("ay", ctypes.c_double),
        ("oe_type", ctypes.c_int), ("gamma_k", ctypes.c_double), ("oe_jump_q6", ctypes.c_int),
        ("oe_mean", ctypes.c_int), ("pp_limiter", ctypes.c_int),
        ("split", ctypes.c_double * 4), ("front", ctypes.c_double * 3), ("front_ahead", ctypes.c_double * 4),
        ("time", ctypes.c_double),
    ]


@dataclass
class Problem:
    """Mirror of ``or_problem``; see fam_oracle.h for the meaning of each field."""
    d: int
    nx: int
    ny: int = 1
    x0: float = 0.0
    x1: float = 1.0
    y0: float = 0.0
    y1: float = 1.0
    k: int = 5
    eq: int = EULER
    bc: tuple = (PERIODIC, PERIODIC, PERIODIC, PERIODIC)
    inflow: tuple = ((0.0,) * 4,) * 4
    gamma: float = 1.4
    ax: float = 1.0
    ay: float = 1.0
    oe_type: int = OE_TYPE2
    gamma_k: float = 0.0
    oe_jump_q6: int = 1
    oe_mean: int = 0
    pp_limiter: int = 0
    split: tuple = (0.0, 0.0, 0.0, 0.0)
    front: tuple = (0.0, 0.0, 0.0)
    front_ahead: tuple = (0.0,) * 4
    time: float = 0.0

    @property
    def ncomp(self) -> int:
        return self.d + 2 if self.eq == EULER else 1

    @property
    def nmom(self) -> int:
        return self.d + 1

    @property
    def shape(self) -> tuple:
        if self.d == 1:
            return (self.ncomp, 2, self.nx)
        return (self.ncomp, 3, self.ny, self.nx)

    def _c(self) -> _Problem:
        p = _Problem()
        p.d, p.nx, p.ny = self.d, self.nx, (1 if self.d == 1 else self.ny)
        p.x0, p.x1, p.y0, p.y1 = self.x0, self.x1, self.y0, self.y1
        p.k, p.eq = self.k, self.eq
        for q in range(4):
            p.bc[q] = int(self.bc[q])
            for c in range(4):
                p.inflow[q][c] = float(self.inflow[q][c])
        p.gamma, p.ax, p.ay = self.gamma, self.ax, self.ay
        p.oe_type, p.gamma_k, p.oe_jump_q6 = self.oe_type, self.gamma_k, self.oe_jump_q6
        p.oe_mean = self.oe_mean
        p.pp_limiter = self.pp_limiter
        for q in range(4):
            p.split[q] = float(self.split[q])
            p.front_ahead[q] = float(self.front_ahead[q])
        for q in range(3):
            p.front[q] = float(self.front[q])
        p.time = float(self.time)
        return p


_lib_handle = None


def lib():
    global _lib_handle
    if _lib_handle is None:
        L = ctypes.CDLL(build())
        dp = ctypes.POINTER(ctypes.c_double)
        pp = ctypes.POINTER(_Problem)
        L.or_recon1d.argtypes = [ctypes.c_int, dp, dp, dp, dp]
        L.or_recon2d.argtypes = [ctypes.c_int, dp, dp, dp, dp]
        L.or_basis1d.argtypes = [ctypes.c_int, ctypes.c_double]
        L.or_basis1d.restype = ctypes.c_double
        L.or_basis2d.argtypes = [ctypes.c_int, ctypes.c_double, ctypes.c_double]
        L.or_basis2d.restype = ctypes.c_double
        L.or_eval1d.argtypes = [ctypes.c_int, dp, ctypes.c_double]
        L.or_eval1d.restype = ctypes.c_double
        L.or_eval2d.argtypes = [ctypes.c_int, dp, ctypes.c_double, ctypes.c_double]
        L.or_eval2d.restype = ctypes.c_double
        L.or_gauss4.argtypes = [dp, dp]
        L.or_residual.argtypes = [pp, dp, dp]
        L.or_max_speed.argtypes = [pp, dp, dp, dp]
        L.or_dt.argtypes = [pp, dp, ctypes.c_double, ctypes.c_int]
        L.or_dt.restype = ctypes.c_double
        L.or_oe.argtypes = [pp, ctypes.c_double, dp, dp]
        L.or_step.argtypes = [pp, dp, ctypes.c_double]
        L.or_rejected_steps.argtypes = [ctypes.c_int]
        L.or_rejected_steps.restype = ctypes.c_long
        L.or_run.argtypes = [pp, dp, ctypes.c_double, ctypes.c_long, ctypes.c_double, ctypes.c_int,
                             dp, ctypes.POINTER(ctypes.c_long)]
        L.or_trace_count.argtypes = []
        L.or_trace_count.restype = ctypes.c_longlong
        L.or_trace_reset.argtypes = []
        L.or_trace_reset.restype = None
        L.or_inadmissible.argtypes = [pp, dp]
        L.or_inadmissible.restype = ctypes.c_longlong
        _lib_handle = L
    return _lib_handle


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _state(P: Problem, U) -> np.ndarray:
    U = np.ascontiguousarray(U, dtype=np.float64)
    if U.shape != P.shape:
        raise ValueError(f"state shape {U.shape} != {P.shape}")
    return U


def recon1d(k: int, um, u0, up) -> tuple[np.ndarray, int]:
    """App. B coefficients c_0..c_5 and the number used by FAM-k."""
    a = [np.ascontiguousarray(v, dtype=np.float64) for v in (um, u0, up)]
    c = np.zeros(6)
    n = lib().or_recon1d(k, _ptr(a[0]), _ptr(a[1]), _ptr(a[2]), _ptr(c))
    return c, n


def recon2d(k: int, avg, mx, my) -> tuple[np.ndarray, int]:
    """App. I coefficients c_0..c_22 from the 3x3 patch (I1..I9 row by row)."""
    a = [np.ascontiguousarray(v, dtype=np.float64).reshape(9) for v in (avg, mx, my)]
    c = np.zeros(23)
    n = lib().or_recon2d(k, _ptr(a[0]), _ptr(a[1]), _ptr(a[2]), _ptr(c))
    return c, n


def basis1d(l: int, xi: float) -> float:
    return lib().or_basis1d(l, xi)


def basis2d(l: int, xi: float, eta: float) -> float:
    return lib().or_basis2d(l, xi, eta)


def eval1d(c: np.ndarray, ncoef: int, xi: float) -> float:
    c = np.ascontiguousarray(c, dtype=np.float64)
    return lib().or_eval1d(ncoef, _ptr(c), xi)


def eval2d(c: np.ndarray, ncoef: int, xi: float, eta: float) -> float:
    c = np.ascontiguousarray(c, dtype=np.float64)
    return lib().or_eval2d(ncoef, _ptr(c), xi, eta)


def gauss4() -> tuple[np.ndarray, np.ndarray]:
    x, w = np.zeros(4), np.zeros(4)
    lib().or_gauss4(_ptr(x), _ptr(w))
    return x, w


def residual(P: Problem, U) -> np.ndarray:
    U = _state(P, U)
    R = np.zeros_like(U)
    if lib().or_residual(ctypes.byref(P._c()), _ptr(U), _ptr(R)):
        raise MemoryError("oracle residual failed")
    return R


def max_speed(P: Problem, U) -> tuple[float, float]:
    U = _state(P, U)
    ax, ay = ctypes.c_double(), ctypes.c_double()
    lib().or_max_speed(ctypes.byref(P._c()), _ptr(U), ctypes.byref(ax), ctypes.byref(ay))
    return ax.value, ay.value


def dt(P: Problem, U, cfl: float, smooth: bool = False) -> float:
    U = _state(P, U)
    return lib().or_dt(ctypes.byref(P._c()), _ptr(U), cfl, int(smooth))


def oe(P: Problem, dt_: float, U) -> tuple[np.ndarray, np.ndarray]:
    """Returns (OE-corrected copy of U, damping exponent theta per cell)."""
    U = _state(P, U).copy()
    theta = np.zeros(U.shape[2:] if P.d == 2 else U.shape[2:], dtype=np.float64)
    if lib().or_oe(ctypes.byref(P._c()), dt_, _ptr(U), _ptr(theta)):
        raise MemoryError("oracle OE failed")
    return U, theta


def step(P: Problem, U, dt_: float) -> np.ndarray:
    U = _state(P, U).copy()
    if lib().or_step(ctypes.byref(P._c()), _ptr(U), dt_):
        raise MemoryError("oracle step failed")
    return U


def run(P: Problem, U, T: float | None = None, nsteps: int | None = None, cfl: float = 0.3,
        smooth: bool = False) -> tuple[np.ndarray, float, int]:
    """Advance to time T (last step clamped) or by exactly nsteps steps."""
    U = _state(P, U).copy()
    t, s = ctypes.c_double(), ctypes.c_long()
    rc = lib().or_run(ctypes.byref(P._c()), _ptr(U), float(T) if T else 0.0, int(nsteps or 0), cfl,
                      int(smooth), ctypes.byref(t), ctypes.byref(s))
    if rc:
        raise FloatingPointError("oracle run produced a non-finite state")
    return U, t.value, s.value


def trace_count(reset: bool = False) -> int:
    """Face quadrature points at which a Rusanov trace had no spectral radius
    (an Euler trace with gamma p / rho < 0), summed over every residual
    evaluation since the last reset (see or_trace_count in fam_oracle.h)."""
    n = int(lib().or_trace_count())
    if reset:
        lib().or_trace_reset()
    return n


def trace_reset() -> None:
    lib().or_trace_reset()


def rejected_steps(reset: bool = False) -> int:
    """Steps run() discarded and retried with half the step size (the
    safeguard's stage check) since the last reset."""
    return int(lib().or_rejected_steps(1 if reset else 0))


def inadmissible(P: Problem, U) -> int:
    """Cells whose averages are not admissible (Euler: rho <= 0 or p <= 0) or
    hold a non-finite value."""
    U = _state(P, U)
    return int(lib().or_inadmissible(ctypes.byref(P._c()), _ptr(U)))
