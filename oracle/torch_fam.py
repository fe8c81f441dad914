"""Differentiable FP64 CPU oracle of the 2D/1D FAM time step (PyTorch CPU ops).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).  This module restates the
forward step of the paper -- eq. (11) / eq. (1dSemi) residual with Rusanov
flux and 4-point Gauss quadrature, SSP-RK3 of eq. (12), Type-II OE of
eq. (2dOE_sol) / eq. (9) with the system forms of Sec. 2.3 -- as whole-array
tensor operations, so that torch.autograd yields the oracle's reverse sweep
(the transpose of every step, taken in reverse order) for the adjoint tests.

The reconstruction is linear: its matrices (stencil moments -> coefficients
of p in the basis of App. B / App. I) and the basis values at the points the
scheme evaluates are read off the pinned C oracle (or_recon*, or_basis*) by
applying it to unit vectors -- a library call as a step, not a second
transcription.  The time-step sizes are inputs (held fixed in the reverse
sweep).  Max and abs use torch's subgradients.
"""
from __future__ import annotations

import numpy as np
import torch

from . import basis1d, basis2d, gauss4, recon1d, recon2d

torch.set_default_dtype(torch.float64)


def _recon_matrix_2d(k: int, q6: bool = False) -> tuple[np.ndarray, int, int]:
    """M (ncoef_eval x 27) with c = M @ [avg(9), mx(9), my(9)]; ncoef for p and for OE jumps."""
    cols = []
    n_p = None
    for j in range(27):
        e = np.zeros(27)
        e[j] = 1.0
        c, n_p = recon2d(k, e[:9], e[9:18], e[18:])
        cols.append(c)
    M = np.array(cols).T  # (23, 27)
    n_oe = 23 if (k == 6 and q6) else n_p
    return M, n_p, n_oe


def _recon_matrix_1d(k: int) -> tuple[np.ndarray, int]:
    cols = []
    for j in range(6):
        e = np.zeros(6)
        e[j] = 1.0
        c, n = recon1d(k, (e[0], e[3]), (e[1], e[4]), (e[2], e[5]))
        cols.append(c)
    return np.array(cols).T, n  # (6, 6): inputs (a_m, a_0, a_p, m_m, m_0, m_p)


class Euler2D:
    """Forward FAM step for the 2D Euler equations on a periodic or outflow grid."""

    def __init__(self, nx: int, ny: int, k: int, box=(0.0, 1.0, 0.0, 1.0), gamma: float = 1.4,
                 bc: str = "periodic", gamma_k: float | None = None, q6: bool = True):
        self.nx, self.ny, self.k, self.g = nx, ny, k, gamma
        self.dx = (box[1] - box[0]) / nx
        self.dy = (box[3] - box[2]) / ny
        self.bc = bc
        self.gk = gamma_k if gamma_k else (25.0 if k <= 4 else 15.0)
        M, self.ncoef, n_oe = _recon_matrix_2d(k, q6)
        self.M = torch.tensor(M)
        x, w = gauss4()
        self.gx, self.gw = torch.tensor(x), torch.tensor(w)
        nc = self.ncoef
        # basis values: volume points (a, b) -> (xi_a, eta_b); faces
        vol = np.array([[basis2d(l, x[a], x[b]) for l in range(nc)] for b in range(4) for a in range(4)])
        self.Bvol = torch.tensor(vol)                                   # (16, nc), index b*4 + a
        self.Bxp = torch.tensor(np.array([[basis2d(l, 0.5, x[g]) for l in range(nc)] for g in range(4)]))
        self.Bxm = torch.tensor(np.array([[basis2d(l, -0.5, x[g]) for l in range(nc)] for g in range(4)]))
        self.Byp = torch.tensor(np.array([[basis2d(l, x[g], 0.5) for l in range(nc)] for g in range(4)]))
        self.Bym = torch.tensor(np.array([[basis2d(l, x[g], -0.5) for l in range(nc)] for g in range(4)]))
        fc = [(-0.5, 0.0), (0.5, 0.0), (0.0, -0.5), (0.0, 0.5)]
        self.Bfc = torch.tensor(np.array([[basis2d(l, a, b) for l in range(n_oe)] for a, b in fc]))
        self.n_oe = n_oe

    # ---- helpers -----------------------------------------------------------
    def pad(self, U: torch.Tensor, g: int) -> torch.Tensor:
        if self.bc == "periodic":
            U = torch.cat([U[..., -g:], U, U[..., :g]], dim=-1)
            return torch.cat([U[..., -g:, :], U, U[..., :g, :]], dim=-2)
        left = U[..., :1].expand(*U.shape[:-1], g)
        right = U[..., -1:].expand(*U.shape[:-1], g)
        U = torch.cat([left, U, right], dim=-1)
        bot = U[..., :1, :].expand(*U.shape[:-2], g, U.shape[-1])
        top = U[..., -1:, :].expand(*U.shape[:-2], g, U.shape[-1])
        return torch.cat([bot, U, top], dim=-2)

    def coeffs(self, Up: torch.Tensor, g: int, r: int, ncoef: int) -> torch.Tensor:
        """Coefficients (4, ncoef, ny+2r, nx+2r) for the cells within r of the grid."""
        ny, nx = self.ny + 2 * r, self.nx + 2 * r
        o = g - r
        parts = []
        for m in range(3):
            for s in range(9):
                dj, di = s // 3 - 1, s % 3 - 1
                parts.append(Up[:, m, o + dj:o + dj + ny, o + di:o + di + nx])
        S = torch.stack(parts, dim=1)  # (4, 27, ny, nx) ordered avg(9), mx(9), my(9)
        return torch.einsum("lk,cknm->clnm", self.M[:ncoef], S)

    def flux(self, u: torch.Tensor, dirn: int):
        rho, mu, mv, E = u[0], u[1], u[2], u[3]
        vx, vy = mu / rho, mv / rho
        p = (self.g - 1.0) * (E - 0.5 * (mu * vx + mv * vy))
        vn = vx if dirn == 0 else vy
        f = torch.stack([rho * vn, mu * vn + (p if dirn == 0 else 0.0), mv * vn + (p if dirn == 1 else 0.0),
                         (E + p) * vn])
        speed = torch.abs(vn) + torch.sqrt(self.g * p / rho)
        return f, speed

    def llf(self, uL, uR, dirn):
        fL, sL = self.flux(uL, dirn)
        fR, sR = self.flux(uR, dirn)
        a = torch.fmax(sL, sR)  # a NaN radius (non-physical trace) is ignored, as C fmax does
        return 0.5 * (fL + fR) - 0.5 * a * (uR - uL)

    # ---- eq. (11) -------------------------------------------------------------
    def residual(self, U: torch.Tensor) -> torch.Tensor:
        Up = self.pad(U, 3)
        C = self.coeffs(Up, 3, 1, self.ncoef)            # cells -1..n (both directions)
        ny, nx = self.ny, self.nx
        # x-faces f = 0..nx between cells f-1 and f, rows 0..ny-1; Gauss points along y
        Cl = C[:, :, 1:ny + 1, 0:nx + 1]
        Cr = C[:, :, 1:ny + 1, 1:nx + 2]
        uL = torch.einsum("gl,clnm->cgnm", self.Bxp, Cl)
        uR = torch.einsum("gl,clnm->cgnm", self.Bxm, Cr)
        Fx = self.llf(uL, uR, 0)                         # (4, 4g, ny, nx+1)
        Cb = C[:, :, 0:ny + 1, 1:nx + 1]
        Ct = C[:, :, 1:ny + 2, 1:nx + 1]
        uB = torch.einsum("gl,clnm->cgnm", self.Byp, Cb)
        uT = torch.einsum("gl,clnm->cgnm", self.Bym, Ct)
        Fy = self.llf(uB, uT, 1)                         # (4, 4g, ny+1, nx)
        Cc = C[:, :, 1:ny + 1, 1:nx + 1]
        uv = torch.einsum("ql,clnm->cqnm", self.Bvol, Cc)  # (4, 16, ny, nx)
        f1, _ = self.flux(uv, 0)
        f2, _ = self.flux(uv, 1)
        W = (self.gw[None, :] * self.gw[:, None]).reshape(16)  # index b*4 + a
        V1 = torch.einsum("q,cqnm->cnm", W, f1)
        V2 = torch.einsum("q,cqnm->cnm", W, f2)
        w, x = self.gw, self.gx
        sxr = torch.einsum("g,cgnm->cnm", w, Fx[..., 1:])
        sxl = torch.einsum("g,cgnm->cnm", w, Fx[..., :-1])
        syt = torch.einsum("g,cgnm->cnm", w, Fy[:, :, 1:, :])
        syb = torch.einsum("g,cgnm->cnm", w, Fy[:, :, :-1, :])
        mx = torch.einsum("g,cgnm->cnm", w * x, Fx[..., 1:] - Fx[..., :-1])
        my = torch.einsum("g,cgnm->cnm", w * x, Fy[:, :, 1:, :] - Fy[:, :, :-1, :])
        R0 = -(sxr - sxl) / self.dx - (syt - syb) / self.dy
        R1 = (V1 - 0.5 * (sxr + sxl)) / self.dx - my / self.dy
        R2 = (V2 - 0.5 * (syt + syb)) / self.dy - mx / self.dx
        return torch.stack([R0, R1, R2], dim=1)

    # ---- Tab. sigma2d (Type II), eq. (2dOE_system) ---------------------------
    def oe(self, U: torch.Tensor, dt: float) -> torch.Tensor:
        Up = self.pad(U, 3)
        C = self.coeffs(Up, 3, 1, self.n_oe)
        ny, nx = self.ny, self.nx
        T = torch.einsum("fl,clnm->cfnm", self.Bfc, C)    # (4, 4 traces, ny+2, nx+2)
        c0 = T[:, :, 1:ny + 1, 1:nx + 1]
        jxl = c0[:, 0] - T[:, 1, 1:ny + 1, 0:nx]
        jxr = T[:, 0, 1:ny + 1, 2:nx + 2] - c0[:, 1]
        jyb = c0[:, 2] - T[:, 3, 0:ny, 1:nx + 1]
        jyt = T[:, 2, 2:ny + 2, 1:nx + 1] - c0[:, 3]
        A = Up[:, 0]                                        # averages, padded by 3
        lam = torch.stack([A[:, 3 + dj:3 + dj + ny, 3 + di:3 + di + nx]
                           for dj in (-1, 0, 1) for di in (-1, 0, 1)], dim=1)  # (4, 9, ny, nx)
        S = lam.sum(dim=1, keepdim=True)
        D = torch.abs(lam - S).max(dim=1).values
        eps = 1e-14 * torch.clamp(torch.abs(lam).max(dim=1).values, min=1.0)
        active = ~(D < eps)
        Dsafe = torch.where(active, D, torch.ones_like(D))
        sx = torch.where(active, self.gk * (torch.abs(jxl) + torch.abs(jxr)) / Dsafe, torch.zeros_like(D))
        sy = torch.where(active, self.gk * (torch.abs(jyb) + torch.abs(jyt)) / Dsafe, torch.zeros_like(D))
        sx = sx.max(dim=0).values
        sy = sy.max(dim=0).values
        ua = torch.stack([A[:, 3 + dj:3 + dj + ny, 3 + di:3 + di + nx]
                          for dj in (-1, 0, 1) for di in (-1, 0, 1)], dim=1)  # (4, 9, ny, nx)
        _, spx = self.flux(ua, 0)
        _, spy = self.flux(ua, 1)
        bx = spx.max(dim=0).values
        by = spy.max(dim=0).values
        theta = bx * dt * sx / self.dx + by * dt * sy / self.dy
        delta = torch.exp(-theta)
        return torch.cat([U[:, :1], U[:, 1:] * delta[None, None]], dim=1)

    # ---- eq. (12) -------------------------------------------------------------
    def step(self, U: torch.Tensor, dt: float) -> torch.Tensor:
        U1 = U + dt * self.residual(U)
        U2 = 0.75 * U + 0.25 * (U1 + dt * self.residual(U1))
        U3 = 1.0 / 3.0 * U + 2.0 / 3.0 * (U2 + dt * self.residual(U2))
        return self.oe(U3, dt)

    def run(self, U: torch.Tensor, dts) -> torch.Tensor:
        for dt in dts:
            U = self.step(U, float(dt))
        return U


def window_functional_grad(shape, window, dx: float, dy: float) -> np.ndarray:
    """dJ/dU for J = dx dy * sum of the density averages over window = (j0, j1, i0, i1)."""
    G = np.zeros(shape)
    j0, j1, i0, i1 = window
    G[0, 0, j0:j1, i0:i1] = dx * dy
    return G


def reverse_sweep(model: Euler2D, U0: np.ndarray, dts, dJdUT: np.ndarray) -> np.ndarray:
    """Oracle gradient dJ/dU0 = (d U_T / d U0)^T dJ/dU_T with the step sizes held fixed."""
    U = torch.tensor(U0, requires_grad=True)
    UT = model.run(U, dts)
    (UT * torch.tensor(dJdUT)).sum().backward()
    return U.grad.numpy().copy()
