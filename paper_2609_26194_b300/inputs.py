"""Seeded synthetic initial data for the FAM time step, as moment arrays.

This module holds only input generation: it projects analytic or piecewise
initial data onto the evolved P1 moment state (cell average and scaled first
moments, Sec. 2.1 / Sec. 2.2 of the paper) by Gauss quadrature or closed
forms.  It contains none of the scheme's arithmetic and is shared by the CPU
oracle tests and the CUDA path.

Layout: 1D ``U[c, m, i]``; 2D ``U[c, m, j, i]`` with m = 0 average, 1 scaled
x-moment (1/|I| int u (x-x_i)/dx), 2 scaled y-moment.  Euler variables are
conservative: (rho, rho u, E) in 1D, (rho, rho u, rho v, E) in 2D.

Workload recipes (shapes and value ranges follow the paper's tests):
  * advection_sine: u0 = sin(2 pi x) on [0,1], exact moments (closed form).
  * euler1d_riemann: [0,1], 8 face-snapped discontinuities, 9 states with
    rho ~ U[0.1,2], u ~ U[-1,1], p ~ U[0.1,10]; rho multiplied by
    (1 + 0.2 sin(32 pi x)).
  * euler2d_smooth: [0,1]^2, rho = 1 + 0.2 sin(2 pi (x+y)), u = v = p = 1.
  * euler2d_rectangles: [0,1]^2 background (1,0,0,1) with 64 face-snapped
    periodic rectangles, side lengths U[N/32, N/4] cells, rho, p ~ U[0.1,5],
    u, v ~ U[-1,1].
  * euler2d_fourier: (1, .5, .5, 1) + 16 Fourier modes of amplitude 0.05/16
    per primitive variable, integer wave numbers in [-4,4]^2 \\ {0}.
  * batched_1d: instances with N = round(exp(U[ln 64, ln 16384])) and
    k ~ U{3,4,5,6}, each with euler1d_riemann data (seed + i).
  * smooth accuracy data of the paper's Examples 4.1 and 4.2.
"""
from __future__ import annotations

import numpy as np

GAMMA = 1.4


def gauss_legendre_unit(nq: int) -> tuple[np.ndarray, np.ndarray]:
    """Gauss-Legendre nodes on [-1/2, 1/2] and weights summing to one."""
    x, w = np.polynomial.legendre.leggauss(nq)
    return 0.5 * x, 0.5 * w


# --------------------------------------------------------------------------
# generic projections
# --------------------------------------------------------------------------

def project_1d(func, n: int, x0: float, x1: float, nq: int = 8) -> np.ndarray:
    """Average and scaled first moment of func (returns (ncomp, npts)) per cell."""
    dx = (x1 - x0) / n
    xi, w = gauss_legendre_unit(nq)
    xc = x0 + (np.arange(n) + 0.5) * dx
    X = xc[:, None] + dx * xi[None, :]                      # (n, nq)
    F = np.asarray(func(X.reshape(-1)), dtype=np.float64)   # (ncomp, n*nq)
    F = F.reshape(F.shape[0], n, nq)
    avg = np.einsum("cnq,q->cn", F, w)
    mom = np.einsum("cnq,q->cn", F, w * xi)
    return np.ascontiguousarray(np.stack([avg, mom], axis=1))


def project_2d(func, nx: int, ny: int, box=(0.0, 1.0, 0.0, 1.0), nq: int = 4,
               rows_per_chunk: int = 128) -> np.ndarray:
    """Average and both scaled first moments of func(X, Y) -> (ncomp, ...)."""
    x0, x1, y0, y1 = box
    dx, dy = (x1 - x0) / nx, (y1 - y0) / ny
    xi, w = gauss_legendre_unit(nq)
    xc = x0 + (np.arange(nx) + 0.5) * dx
    out = None
    for r0 in range(0, ny, rows_per_chunk):
        r1 = min(ny, r0 + rows_per_chunk)
        yc = y0 + (np.arange(r0, r1) + 0.5) * dy
        X = (xc[None, :, None, None] + dx * xi[None, None, None, :])      # (1, nx, 1, qx)
        Y = (yc[:, None, None, None] + dy * xi[None, None, :, None])      # (rows, 1, qy, 1)
        X, Y = np.broadcast_arrays(X, Y)                                   # (rows, nx, qy, qx)
        F = np.asarray(func(X, Y), dtype=np.float64)                       # (nc, rows, nx, qy, qx)
        if out is None:
            out = np.empty((F.shape[0], 3, ny, nx), dtype=np.float64)
        ww = w[:, None] * w[None, :]                                       # (qy, qx)
        out[:, 0, r0:r1] = np.einsum("crnab,ab->crn", F, ww)
        out[:, 1, r0:r1] = np.einsum("crnab,ab->crn", F, ww * xi[None, :])
        out[:, 2, r0:r1] = np.einsum("crnab,ab->crn", F, ww * xi[:, None])
    return np.ascontiguousarray(out)


def primitive_to_conservative_1d(rho, u, p, gamma=GAMMA):
    return np.stack([rho, rho * u, p / (gamma - 1.0) + 0.5 * rho * u * u])


def primitive_to_conservative_2d(rho, u, v, p, gamma=GAMMA):
    return np.stack([rho, rho * u, rho * v, p / (gamma - 1.0) + 0.5 * rho * (u * u + v * v)])


# --------------------------------------------------------------------------
# named workloads
# --------------------------------------------------------------------------

def advection_sine(n: int = 200) -> np.ndarray:
    """Exact moments of sin(2 pi x) on [0,1] (closed-form integrals)."""
    dx = 1.0 / n
    xl = np.arange(n) * dx
    xr = xl + dx
    xc = xl + 0.5 * dx
    a = 2.0 * np.pi
    avg = (np.cos(a * xl) - np.cos(a * xr)) / (a * dx)

    def prim(x):  # antiderivative of sin(a x) (x - xc)
        return -(x - xc) * np.cos(a * x) / a + np.sin(a * x) / (a * a)

    mom = (prim(xr) - prim(xl)) / (dx * dx)
    return np.ascontiguousarray(np.stack([avg, mom])[None])


def euler1d_riemann(n: int = 65536, seed: int = 2, gamma: float = GAMMA, rho=(0.1, 2.0), umax: float = 1.0,
                    p=(0.1, 10.0)) -> np.ndarray:
    """8 face-snapped discontinuities, 9 constant states (rho, u, p ranges as
    given) times the density perturbation (1 + 0.2 sin(32 pi x))."""
    rng = np.random.default_rng(seed)
    faces = np.sort(rng.choice(np.arange(1, n), size=min(8, n - 1), replace=False))
    ns = len(faces) + 1
    rho_s = rng.uniform(rho[0], rho[1], ns)
    u_s = rng.uniform(-umax, umax, ns)
    p_s = rng.uniform(p[0], p[1], ns)
    dx = 1.0 / n
    # piece index of every cell (faces are snapped to cell faces)
    piece = np.searchsorted(faces, np.arange(n), side="right")

    def func(x):
        cell = np.minimum((x / dx).astype(np.int64), n - 1)
        pc = piece[cell]
        rho = rho_s[pc] * (1.0 + 0.2 * np.sin(32.0 * np.pi * x))
        return primitive_to_conservative_1d(rho, u_s[pc], p_s[pc], gamma)

    return project_1d(func, n, 0.0, 1.0, nq=8)


def _sincos_moments(n: int, x0: float, x1: float, freq: float, phase: float = 0.0):
    """1D cell averages and scaled moments of sin(freq x + phase), cos(...)."""
    s = project_1d(lambda x: np.stack([np.sin(freq * x + phase), np.cos(freq * x + phase)]), n, x0, x1, 8)
    return s[0, 0], s[0, 1], s[1, 0], s[1, 1]  # As, Ms, Ac, Mc


def euler2d_smooth(n: int = 4096, gamma: float = GAMMA, box=(0.0, 1.0, 0.0, 1.0),
                   amp: float = 0.2, freq: float = 2.0 * np.pi, u: float = 1.0, v: float = 1.0,
                   p: float = 1.0) -> np.ndarray:
    """rho = 1 + amp sin(freq (x + y)), constant u, v, p (separable, exact)."""
    x0, x1, y0, y1 = box
    Asx, Msx, Acx, Mcx = _sincos_moments(n, x0, x1, freq)
    Asy, Msy, Acy, Mcy = _sincos_moments(n, y0, y1, freq)
    # sin(a + b) = sin a cos b + cos a sin b
    avg = 1.0 + amp * (Asx[None, :] * Acy[:, None] + Acx[None, :] * Asy[:, None])
    mx = amp * (Msx[None, :] * Acy[:, None] + Mcx[None, :] * Asy[:, None])
    my = amp * (Asx[None, :] * Mcy[:, None] + Acx[None, :] * Msy[:, None])
    rho = np.stack([avg, mx, my])
    e_const = p / (gamma - 1.0)
    ke = 0.5 * (u * u + v * v)
    E = ke * rho
    E[0] += e_const
    return np.ascontiguousarray(np.stack([rho, u * rho, v * rho, E]))


def euler2d_rectangles(n: int = 4096, seed: int = 3, nrect: int = 64, gamma: float = GAMMA,
                       lo: float = 0.1, hi: float = 5.0, vmax: float = 1.0) -> np.ndarray:
    """Piecewise-constant periodic rectangles painted in order (moments vanish).

    rho, p ~ U[lo, hi], u, v ~ U[-vmax, vmax].  The default ranges are the
    shock-run recipe; without a positivity limiter the scheme admits only
    milder contrasts (``ADMISSIBLE_RECT`` = rho, p in [0.5, 2.5], |u|,|v| <= 0.5).
    """
    rng = np.random.default_rng(seed)
    prim = np.empty((4, n, n))
    prim[0], prim[1], prim[2], prim[3] = 1.0, 0.0, 0.0, 1.0
    wmin, wmax = max(1, n // 32), max(2, n // 4)
    for _ in range(nrect):
        i0, j0 = rng.integers(0, n, 2)
        wx, wy = rng.integers(wmin, wmax + 1, 2)
        st = (rng.uniform(lo, hi), rng.uniform(-vmax, vmax), rng.uniform(-vmax, vmax), rng.uniform(lo, hi))
        ii = (i0 + np.arange(wx)) % n
        jj = (j0 + np.arange(wy)) % n
        for c in range(4):
            prim[c][np.ix_(jj, ii)] = st[c]
    cons = primitive_to_conservative_2d(prim[0], prim[1], prim[2], prim[3], gamma)
    U = np.zeros((4, 3, n, n))
    U[:, 0] = cons
    return U


ADMISSIBLE_RECT = dict(lo=0.5, hi=2.5, vmax=0.5)


def euler2d_fourier(n: int = 1024, seed: int = 5, nmodes: int = 16, amp: float = 0.05,
                    gamma: float = GAMMA) -> np.ndarray:
    rng = np.random.default_rng(seed)
    base = (1.0, 0.5, 0.5, 1.0)
    modes = []
    for var in range(4):
        ms = []
        while len(ms) < nmodes:
            kx, ky = rng.integers(-4, 5, 2)
            if kx == 0 and ky == 0:
                continue
            ms.append((int(kx), int(ky), rng.uniform(0.0, 2.0 * np.pi)))
        modes.append(ms)

    def func(X, Y):
        prim = []
        for var in range(4):
            f = np.full(X.shape, base[var])
            for kx, ky, ph in modes[var]:
                f = f + (amp / nmodes) * np.sin(2.0 * np.pi * (kx * X + ky * Y) + ph)
            prim.append(f)
        return primitive_to_conservative_2d(*prim, gamma=gamma)

    return project_2d(func, n, n, nq=4)


# Milder Riemann states for many small instances: with jumps only tens of
# cells apart the full ranges above produce negative pressures within a few
# steps without a positivity limiter (which the paper cites but does not
# define); these ranges stayed admissible for 200 steps in every sampled
# instance.
BATCH_RIEMANN = dict(rho=(0.7, 1.5), umax=0.3, p=(0.7, 2.0))


def batched_1d(n_inst: int = 4096, seed: int = 4, nmin: int = 64, nmax: int = 16384, **riemann):
    """List of (k, U) instances; U follows euler1d_riemann with seed + i."""
    rng = np.random.default_rng(seed)
    ns = np.rint(np.exp(rng.uniform(np.log(nmin), np.log(nmax), n_inst))).astype(int)
    ks = rng.integers(3, 7, n_inst)
    kw = riemann or BATCH_RIEMANN
    return [(int(ks[i]), euler1d_riemann(int(ns[i]), seed + i, **kw)) for i in range(n_inst)]


def density_wave_2d(nx: int, ny: int, mx_: int, my_: int, phase: float, amp: float, u: float, v: float,
                    p: float, gamma: float = GAMMA) -> np.ndarray:
    """Periodic [0,1]^2 state rho = 1 + amp sin(2 pi (mx x + my y) + phase)
    with constant u, v, p, on nx x ny cells (separable, exact moments)."""
    Asx, Msx, Acx, Mcx = _sincos_moments(nx, 0.0, 1.0, 2.0 * np.pi * mx_, phase)
    Asy, Msy, Acy, Mcy = _sincos_moments(ny, 0.0, 1.0, 2.0 * np.pi * my_)
    avg = 1.0 + amp * (Asx[None, :] * Acy[:, None] + Acx[None, :] * Asy[:, None])
    mx = amp * (Msx[None, :] * Acy[:, None] + Mcx[None, :] * Asy[:, None])
    my = amp * (Asx[None, :] * Mcy[:, None] + Acx[None, :] * Msy[:, None])
    rho = np.stack([avg, mx, my])
    E = 0.5 * (u * u + v * v) * rho
    E[0] += p / (gamma - 1.0)
    return np.ascontiguousarray(np.stack([rho, u * rho, v * rho, E]))


def batched_2d(n_inst: int = 256, seed: int = 6, nmin: int = 32, nmax: int = 512) -> list:
    """List of (k, U) 2D Euler instances on [0,1]^2: nx, ny log-uniform in
    [nmin, nmax] (independently), k uniform in {3..6}, a density wave with
    wavenumbers in 1..3 and amplitude in [0.05, 0.2], u, v in [-0.5, 0.5],
    p in [0.7, 1.5] (density_wave_2d)."""
    rng = np.random.default_rng(seed)
    nxs = np.rint(np.exp(rng.uniform(np.log(nmin), np.log(nmax), n_inst))).astype(int)
    nys = np.rint(np.exp(rng.uniform(np.log(nmin), np.log(nmax), n_inst))).astype(int)
    ks = rng.integers(3, 7, n_inst)
    out = []
    for i in range(n_inst):
        m1, m2 = (int(v) for v in rng.integers(1, 4, 2))
        ph, a = rng.uniform(0, 2 * np.pi), rng.uniform(0.05, 0.2)
        u, v = rng.uniform(-0.5, 0.5, 2)
        p = rng.uniform(0.7, 1.5)
        out.append((int(ks[i]), density_wave_2d(int(nxs[i]), int(nys[i]), m1, m2, ph, a, u, v, p)))
    return out


# shock problems of Examples 4.4 and 4.5 (no positivity limiter needed)

SHU_OSHER_LEFT = (3.857143, 2.629369, 10.333333)


def shu_osher(n: int = 400, gamma: float = GAMMA) -> np.ndarray:
    """[-5,5]: (rho,u,p) = (3.857143, 2.629369, 10.333333) for x < -4, else
    (1 + 0.2 sin(5x), 0, 1); the jump sits on a cell face when n % 10 == 0."""
    def f(x):
        left = x < -4.0
        rho = np.where(left, SHU_OSHER_LEFT[0], 1.0 + 0.2 * np.sin(5.0 * x))
        u = np.where(left, SHU_OSHER_LEFT[1], 0.0)
        p = np.where(left, SHU_OSHER_LEFT[2], 1.0)
        return primitive_to_conservative_1d(rho, u, p, gamma)
    return project_1d(f, n, -5.0, 5.0, nq=8)


def shu_osher_inflow(gamma: float = GAMMA):
    return tuple(primitive_to_conservative_1d(np.array(SHU_OSHER_LEFT[0]), np.array(SHU_OSHER_LEFT[1]),
                                              np.array(SHU_OSHER_LEFT[2]), gamma).tolist())


def lax_tube(n: int = 200, gamma: float = GAMMA) -> np.ndarray:
    """[-0.5,0.5]: (0.445, 0.698, 3.528) for x < 0, (0.5, 0, 0.571) otherwise."""
    def f(x):
        left = x < 0.0
        return primitive_to_conservative_1d(np.where(left, 0.445, 0.5), np.where(left, 0.698, 0.0),
                                            np.where(left, 3.528, 0.571), gamma)
    return project_1d(f, n, -0.5, 0.5, nq=8)


def sedov_1d(n: int = 801, gamma: float = GAMMA) -> np.ndarray:
    """Sedov point blast of Example 4.7 on [-2, 2]: rho = 1, u = 0, total
    energy 1e-12 everywhere except the central cell (n odd: the cell around
    x = 0), whose energy density is 3.2e6 / dx.  Cell averages, zero first
    moments."""
    if n % 2 == 0:
        raise ValueError("n must be odd (one central cell)")
    dx = 4.0 / n
    U = np.zeros((3, 2, n))
    U[0, 0] = 1.0
    U[2, 0] = 1e-12
    U[2, 0, n // 2] = 3.2e6 / dx
    return U


def leblanc_1d(n: int = 800, gamma: float = GAMMA) -> np.ndarray:
    """LeBlanc shock tube of Example 4.7 on [-10, 10]: (rho, u, p) =
    (2, 0, 1e9) for x < 0 and (1e-3, 0, 1) for x > 0 (the jump on a face for
    even n); cell averages, zero first moments."""
    if n % 2:
        raise ValueError("n must be even (the jump on a cell face)")
    U = np.zeros((3, 2, n))
    h = n // 2
    U[0, 0, :h], U[0, 0, h:] = 2.0, 1e-3
    U[2, 0, :h], U[2, 0, h:] = 1e9 / (gamma - 1.0), 1.0 / (gamma - 1.0)
    return U


# double Mach reflection (Example 4.8): states behind / ahead of the Mach 10
# shock (rho, u, v, p) and the shock line x = a + b y + c t (through (1/6, 0)
# at 60 degrees to the x-axis, moving at speed 10 along its normal)
DMR_POST = (8.0, 8.25 * np.cos(np.pi / 6.0), -8.25 * np.sin(np.pi / 6.0), 116.5)
DMR_PRE = (1.4, 0.0, 0.0, 1.0)
DMR_FRONT = (1.0 / 6.0, 1.0 / np.sqrt(3.0), 20.0 / np.sqrt(3.0))
DMR_BOX = (0.0, 3.0, 0.0, 1.0)


def double_mach_states(gamma: float = GAMMA):
    """Conservative (behind, ahead) states of the double Mach shock."""
    post = primitive_to_conservative_2d(*[np.array(v) for v in DMR_POST], gamma)
    pre = primitive_to_conservative_2d(*[np.array(v) for v in DMR_PRE], gamma)
    return tuple(float(v) for v in post), tuple(float(v) for v in pre)


def double_mach(nx: int = 1440, ny: int = 480, gamma: float = GAMMA, nq: int = 8) -> np.ndarray:
    """Double Mach reflection on [0, 3] x [0, 1] at t = 0: the behind state
    left of the shock line x = 1/6 + y / sqrt(3), the ahead state right of it;
    averages and scaled first moments by nq x nq Gauss points per cell."""
    post, pre = double_mach_states(gamma)
    a, b, _ = DMR_FRONT

    def f(X, Y):
        behind = X < a + b * Y
        return np.stack([np.where(behind, post[c], pre[c]) for c in range(4)])
    return project_2d(f, nx, ny, DMR_BOX, nq=nq)


def composite_1d(n: int = 200) -> np.ndarray:
    """A discontinuous advection profile on [-1, 1] (synthetic stand-in for
    the composite profile of the paper's supplementary advection test): a
    Gaussian at -0.7, a square wave on [-0.4, -0.1], a triangle on [0.1, 0.5]
    and a parabolic bump on [0.6, 0.9].  Averages and scaled first moments by
    8-point Gauss per cell."""
    def f(x):
        g = np.exp(-200.0 * (x + 0.7) ** 2)
        sq = ((x >= -0.4) & (x < -0.1)).astype(float)
        tri = np.clip(1.0 - np.abs(x - 0.3) / 0.2, 0.0, None)
        bump = np.clip(1.0 - ((x - 0.75) / 0.15) ** 2, 0.0, None)
        return (g + sq + tri + bump)[None]
    return project_1d(f, n, -1.0, 1.0, nq=8)


def multiscale_lax(n: int = 600, gamma: float = GAMMA) -> np.ndarray:
    """Multiscale Lax problem of Example 4.6 on [-15, 15]: (rho, u, p) =
    (44.5, 0.698, 352.8) on [-15, -10), (50, 0, 57.1) on [-10, 0),
    (0.00445, 0.698, 0.03528) on [0, 10), (0.005, 0, 0.00571) on [10, 15];
    the jumps sit on cell faces when n % 6 == 0.  Cell averages, zero
    moments."""
    if n % 6:
        raise ValueError("n must be a multiple of 6 (the jumps on cell faces)")
    x = -15.0 + (np.arange(n) + 0.5) * (30.0 / n)
    parts = [(x < -10.0, (44.5, 0.698, 352.8)), ((x >= -10.0) & (x < 0.0), (50.0, 0.0, 57.1)),
             ((x >= 0.0) & (x < 10.0), (0.00445, 0.698, 0.03528)), (x >= 10.0, (0.005, 0.0, 0.00571))]
    rho, u, p = (np.select([m for m, _ in parts], [v[q] for _, v in parts]) for q in range(3))
    U = np.zeros((3, 2, n))
    U[:, 0] = primitive_to_conservative_1d(rho, u, p, gamma)
    return U


def buckley_leverett(n: int = 100) -> np.ndarray:
    """Example 4.3 on [-1, 1] (periodic): u = 1 on [-0.5, 0], 0 elsewhere;
    exact cell averages (the jumps may cut cells), zero first moments."""
    dx = 2.0 / n
    xl = -1.0 + np.arange(n) * dx
    U = np.zeros((1, 2, n))
    U[0, 0] = np.clip(np.minimum(xl + dx, 0.0) - np.maximum(xl, -0.5), 0.0, None) / dx
    return U


# smooth accuracy data (Example 4.1 and Example 4.2 of the paper)

def burgers_smooth(n: int) -> np.ndarray:
    """u0 = 0.5 + sin(pi x) on [0,2]."""
    return project_1d(lambda x: (0.5 + np.sin(np.pi * x))[None], n, 0.0, 2.0, nq=8)


def euler1d_smooth(n: int, gamma: float = GAMMA) -> np.ndarray:
    """(rho, u, p) = (1 + 0.2 sin(pi x), 1, 1) on [0,2]."""
    return project_1d(lambda x: primitive_to_conservative_1d(1.0 + 0.2 * np.sin(np.pi * x),
                                                             np.ones_like(x), np.ones_like(x), gamma),
                      n, 0.0, 2.0, nq=8)


def euler2d_smooth_accuracy(n: int, gamma: float = GAMMA) -> np.ndarray:
    """(rho, u, v, p) = (1 + 0.2 sin(pi (x+y)), 1, 1, 1) on [0,2]^2."""
    return euler2d_smooth(n, gamma, box=(0.0, 2.0, 0.0, 2.0), freq=np.pi)
