"""Pins of the oracle's Buckley-Leverett equation (Example 4.3).

f(u) = 4u^2 / (4u^2 + (1-u)^2), periodic [-1, 1], u0 = 1 on [-0.5, 0] and 0
elsewhere, T = 0.4.  f' vanishes at u = 0 and 1, so every wave speed the
method uses is the bound max |f'| (reading c27).  What fixes the oracle:
  - the flux: the residual of the averages on smooth data equals the exact
    flux difference -(f(u(x+)) - f(u(x-))) / dx to the reconstruction's order;
  - the speed: the time step is cfl dx / max |f'|, max |f'| found here from
    f' on a fine grid refined by Newton on f'' = 0;
  - the entropy solution of both Riemann problems (a rarefaction from the
    sonic state u = 0 up to u_a = 1 - 2/sqrt(5) and a shock into 1; a
    rarefaction from 1 down to u_b = 1/sqrt(5) and a shock into 0 at speed
    (1 + sqrt(5))/2), computed here from the convex / concave hulls of f:
    FAM3 and FAM4 converge to it;
  - the safeguard keeps every average in [0, 1].
"""
import numpy as np
import pytest
from scipy.optimize import brentq

import oracle
from paper_2609_26194_b300 import inputs


def f(u):
    return 4 * u * u / (4 * u * u + (1 - u) ** 2)


def fp(u):
    return 8 * u * (1 - u) / (5 * u * u - 2 * u + 1) ** 2


U_STAR = brentq(lambda u: 10 * u ** 3 - 15 * u ** 2 + 1, 0.1, 0.5)  # f'' = 0 in (0, 1)
U_A, U_B = 1 - 2 / np.sqrt(5), 1 / np.sqrt(5)


def exact(x, T):
    """Entropy solution at time T (no wave interaction before T = 0.4)."""
    u = np.zeros_like(x)
    xi1 = (x + 0.5) / T
    fan1 = (xi1 >= 0) & (xi1 < fp(U_A))
    u[fan1] = [brentq(lambda v: fp(v) - s, 0.0, U_STAR) for s in xi1[fan1]]
    u[(xi1 >= fp(U_A)) & (x < 0)] = 1.0
    xi2 = x / T
    fan2 = (xi2 > 0) & (xi2 < fp(U_B))
    u[fan2] = [brentq(lambda v: fp(v) - s, U_STAR, 1.0) for s in xi2[fan2]]
    return u


def exact_avg(n, T, sub=400):
    dx = 2.0 / n
    xs = -1.0 + (np.arange(n * sub) + 0.5) * dx / sub
    return exact(xs, T).reshape(n, sub).mean(axis=1)


def problem(n, k, **kw):
    return oracle.Problem(d=1, nx=n, x0=-1.0, x1=1.0, k=k, eq=oracle.BUCKLEY, bc=(oracle.PERIODIC,) * 4, **kw)


def test_tangent_states_and_speed_bound():
    """The hull tangents have the closed forms above, and the bound of |f'|
    is attained at U_STAR (the fine-grid maximum agrees)."""
    assert abs(fp(U_A) * (1 - U_A) - (1 - f(U_A))) < 1e-14
    assert abs(fp(U_B) * U_B - f(U_B)) < 1e-14
    assert abs(fp(U_B) - (1 + np.sqrt(5)) / 2) < 1e-13
    grid = np.linspace(-3.0, 4.0, 2_000_001)
    assert abs(np.max(np.abs(fp(grid))) - fp(U_STAR)) < 1e-10


@pytest.mark.parametrize("k", [3, 5])
def test_flux_and_time_step(k):
    n = 200
    U = inputs.project_1d(lambda x: (0.5 + 0.3 * np.sin(np.pi * x))[None], n, -1.0, 1.0)
    P = problem(n, k)
    R = oracle.residual(P, U)
    dx = 2.0 / n
    xf = -1.0 + np.arange(n + 1) * dx
    F = f(0.5 + 0.3 * np.sin(np.pi * xf))
    want = -(F[1:] - F[:-1]) / dx
    assert np.max(np.abs(R[0, 0] - want)) < 2e-6 * np.max(np.abs(want))
    assert oracle.dt(P, U, 0.3) == pytest.approx(0.3 * dx / fp(U_STAR), rel=1e-15)


@pytest.mark.parametrize("k", [3, 4])
def test_fam3_fam4_converge_to_the_entropy_solution(k):
    errs = []
    for n in (100, 400):
        V, t, _ = oracle.run(problem(n, k, pp_limiter=1), inputs.buckley_leverett(n), T=0.4, cfl=1 / 6)
        assert t == 0.4
        errs.append(np.abs(V[0, 0] - exact_avg(n, 0.4)).mean())
    assert errs[0] < 0.02 and errs[0] / errs[1] > 3.0, errs


def test_fam5_with_the_printed_gamma_k_keeps_the_sonic_rarefaction_closed():
    """Reading c27: with the printed OE constant for k >= 5 (gamma_k = 12.5 in
    1D) FAM5 does not open the rarefaction from the sonic state u = 0 under
    refinement: a flat plateau near u = 0.03 stands where the entropy fan
    rises from 0.05 to u_a = 0.106, the shock into 1 leads from it (left of
    the entropy shock at x = -0.5 + 0.4 f'(u_a)), and the L1 error stalls near
    1e-2.  With gamma_k = 25 (the k <= 4 value) it converges."""
    n = 400
    U = inputs.buckley_leverett(n)
    x = -1.0 + (np.arange(n) + 0.5) * (2.0 / n)
    V, _, _ = oracle.run(problem(n, 5, pp_limiter=1), U, T=0.4, cfl=1 / 12)
    ex = exact_avg(n, 0.4)
    assert np.abs(V[0, 0] - ex).mean() > 8e-3
    fan = (x > -0.3) & (x < -0.12)
    assert V[0, 0][fan].max() < 0.04 < ex[fan].min()
    left = (x > -0.5) & (x < 0.0)
    front = x[left][np.argmax(V[0, 0][left] > 0.5)]
    assert front < -0.5 + 0.4 * fp(U_A) - 0.008
    W, _, _ = oracle.run(problem(n, 5, pp_limiter=1, gamma_k=25.0), U, T=0.4, cfl=1 / 12)
    assert np.abs(W[0, 0] - ex).mean() < 6e-3


@pytest.mark.parametrize("k", [3, 5])
def test_safeguard_keeps_the_averages_in_bounds(k):
    n = 100
    U = inputs.buckley_leverett(n)
    cfl = 1 / 6 if k <= 4 else 1 / 12
    V, _, _ = oracle.run(problem(n, k, pp_limiter=1), U, T=0.4, cfl=cfl)
    assert V[0, 0].min() >= 0.0 and V[0, 0].max() <= 1.0
    assert abs(V[0, 0].sum() - U[0, 0].sum()) < 1e-12 * U[0, 0].sum()
    if k == 5:
        W, _, _ = oracle.run(problem(n, k), U, T=0.4, cfl=cfl)
        assert W[0, 0].max() > 1.0 + 1e-3  # the unlimited scheme overshoots
