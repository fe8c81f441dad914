"""Pins of the oracle's optional BP/PP safeguard (option pp_limiter).

The paper applies a bound/positivity-preserving limiter after RK substeps in
the tests that name it (Sec. 2.3 remarks, Alg. 1) and only cites its
construction.  The oracle builds the Zhang--Shu scaling of each stage's
reconstruction towards the cell average, checked at the points of a
Gauss--Lobatto decomposition of the average and at the volume Gauss points,
with the CFL speeds taken at those points.  What fixes it, without any GPU:
  - the decomposition: the Gauss--Lobatto rules used (3 points for k <= 4,
    4 for k = 5, 6) reproduce the cell mean of every polynomial of degree
    k - 1, with end weights 1/6 and 1/12 (textbook rules);
  - on data whose reconstructions are admissible at the points, the
    safeguard changes nothing (the residual is bit-identical);
  - the forward-Euler property it exists for: one Euler step of the averages
    at the bound CFL (dt from the limited point speeds) keeps every average
    admissible, on data where the unlimited scheme loses admissibility;
  - whole runs at the printed shock-run ranges, Shu-Osher at the paper's
    CFL and the extreme tests of Example 4.7 stay admissible with it and
    fail without it.
"""
import numpy as np
import pytest

import oracle
from paper_2609_26194_b300 import inputs

PRINTED_1D = dict(rho=(0.1, 2.0), umax=1.0, p=(0.1, 10.0))


def _lobatto(k):
    if k <= 4:
        return np.array([-0.5, 0.0, 0.5]), np.array([1, 4, 1]) / 6.0
    r = 0.5 / np.sqrt(5.0)
    return np.array([-0.5, -r, r, 0.5]), np.array([1, 5, 5, 1]) / 12.0


@pytest.mark.parametrize("k", [3, 4, 5, 6])
def test_lobatto_decomposition_reproduces_the_mean(k):
    x, w = _lobatto(k)
    rng = np.random.default_rng(k)
    for _ in range(5):
        c = rng.standard_normal(k)  # degree k - 1
        poly = np.polynomial.Polynomial(c)
        mean = poly.integ()(0.5) - poly.integ()(-0.5)
        assert abs(np.dot(w, poly(x)) - mean) < 1e-14 * (1 + abs(mean))
    assert w[0] == w[-1] == (1 / 6 if k <= 4 else 1 / 12)


@pytest.mark.parametrize("d", [1, 2])
@pytest.mark.parametrize("k", [3, 5, 6])
def test_safeguard_inactive_on_admissible_data(d, k):
    n = 60 if d == 1 else (24, 20)
    if d == 1:
        U = inputs.project_1d(lambda x: inputs.primitive_to_conservative_1d(
            1 + 0.2 * np.sin(2 * np.pi * x), 0.3 + 0.0 * x, 1 + 0.1 * np.cos(2 * np.pi * x)), n, 0.0, 1.0)
        P0 = oracle.Problem(d=1, nx=n, k=k, eq=oracle.EULER)
    else:
        U = inputs.euler2d_smooth(n[0])[:, :, :n[1], :]
        U = np.ascontiguousarray(U)
        P0 = oracle.Problem(d=2, nx=n[0], ny=n[1], k=k, eq=oracle.EULER, bc=(oracle.OUTFLOW,) * 4)
    P1 = oracle.Problem(**{**P0.__dict__, "pp_limiter": 1})
    assert np.array_equal(oracle.residual(P0, U), oracle.residual(P1, U))


def _admissible_fraction(U, d):
    rho = U[0, 0]
    m2 = U[1, 0] ** 2 + (U[2, 0] ** 2 if d == 2 else 0.0)
    E = U[d + 1, 0]
    p = 0.4 * (E - 0.5 * m2 / rho)
    return np.mean((rho > 0) & (p > 0) & np.isfinite(p))


@pytest.mark.parametrize("k", [4, 5, 6])
def test_euler_step_of_averages_is_admissible_at_the_bound(k):
    """Rectangles at rho, p in [0.1, 5], |u|, |v| <= 1 (the shock-run ranges):
    one forward-Euler step of the averages at CFL = the end weight of the
    Lobatto rule, dt from the limited point speeds, stays admissible with
    the safeguard; without it the residual is not even finite."""
    n = 48
    U = inputs.euler2d_rectangles(n, seed=3, nrect=64)
    cfl = 1 / 6 if k <= 4 else 1 / 12
    P = oracle.Problem(d=2, nx=n, ny=n, k=k, eq=oracle.EULER, pp_limiter=1)
    dt = oracle.dt(P, U, cfl)
    R = oracle.residual(P, U)
    assert np.all(np.isfinite(R))
    assert _admissible_fraction(U + dt * R, 2) == 1.0
    assert oracle.trace_count(reset=True) >= 0  # (counter reset)
    oracle.residual(P, U)
    assert oracle.trace_count(reset=True) == 0  # every limited trace has a spectral radius
    P0 = oracle.Problem(d=2, nx=n, ny=n, k=k, eq=oracle.EULER)
    R0 = oracle.residual(P0, U)
    assert not np.all(np.isfinite(R0)) or _admissible_fraction(U + dt * R0, 2) < 1.0


@pytest.mark.parametrize("k", [4, 5, 6])
def test_printed_range_rectangles_run_with_the_safeguard(k):
    """The same data advanced 15 steps at the paper's CFL (Sec. 4: 0.4 for
    k = 4, 0.55 for k = 5, 6): admissible throughout with the safeguard; the
    unlimited scheme leaves the admissible set in the first step."""
    n = 48
    U = inputs.euler2d_rectangles(n, seed=3, nrect=64)
    cfl = 0.4 if k == 4 else 0.55
    for pp, ok in ((1, True), (0, False)):
        P = oracle.Problem(d=2, nx=n, ny=n, k=k, eq=oracle.EULER, pp_limiter=pp)
        V, failed = U.copy(), False
        for _ in range(15 if pp else 1):
            V = oracle.step(P, V, oracle.dt(P, V, cfl))
            if oracle.inadmissible(P, V):
                failed = True
                break
        assert failed != ok, (k, pp)


EXTREME = {  # Example 4.7: generator, cells, domain, final time
    "sedov": (inputs.sedov_1d, 201, -2.0, 2.0, 1e-3),
    "leblanc": (inputs.leblanc_1d, 200, -10.0, 10.0, 1e-4),
}


@pytest.mark.parametrize("name", ["sedov", "leblanc"])
@pytest.mark.parametrize("k", [3, 5])
def test_extreme_1d_tests_run_with_the_safeguard(name, k):
    """Example 4.7 (Sedov point blast on [-2, 2] to T = 1e-3; LeBlanc tube
    on [-10, 10] to T = 1e-4; outflow), at the CFL of the guarantee (1/6 for
    k = 3, 1/12 for k = 5).  The unlimited scheme leaves the admissible set
    in its first step; with the safeguard every step stays admissible, mass
    and energy are conserved to rounding (no wave reaches the boundary, whose
    fluxes carry no mass or energy for gas at rest), the Sedov profile stays
    mirror-symmetric, and its peak density lies below the strong-shock limit
    (gamma + 1) / (gamma - 1) = 6."""
    gen, n, x0, x1, T = EXTREME[name]
    U = gen(n)
    cfl = 1 / 6 if k <= 4 else 1 / 12
    P0 = oracle.Problem(d=1, nx=n, x0=x0, x1=x1, k=k, eq=oracle.EULER, bc=(oracle.OUTFLOW,) * 4)
    assert oracle.inadmissible(P0, oracle.step(P0, U, oracle.dt(P0, U, cfl)))
    P = oracle.Problem(**{**P0.__dict__, "pp_limiter": 1})
    V, t = U.copy(), 0.0
    while t < T:
        dt = min(oracle.dt(P, V, cfl), T - t)
        V = oracle.step(P, V, dt)
        t += dt
        assert oracle.inadmissible(P, V) == 0, t
    for c in (0, 2):  # mass, energy
        assert abs(V[c, 0].sum() / U[c, 0].sum() - 1.0) < 1e-12
    rho = V[0, 0]
    if name == "sedov":
        assert np.max(np.abs(rho - rho[::-1])) < 1e-12 * rho.max()
        assert 4.0 < rho.max() < 6.0
    else:
        assert rho.min() > 0.9e-3 and rho.max() < 2.02  # positivity, not a maximum principle


def test_shu_osher_at_the_papers_cfl_runs_with_the_safeguard():
    """Example 4.4 (400 cells on [-5, 5], inflow / outflow) at Sec. 4's
    C = 0.55 with k = 3: the unlimited scheme leaves the admissible set in the
    first step; with the safeguard the run reaches T = 1.8 admissible, with
    the post-shock density of the problem (about 3.86 behind the shock, the
    entropy waves peaking between 4 and 5)."""
    n, cfl = 400, 0.55
    st = inputs.shu_osher_inflow()
    U = inputs.shu_osher(n)
    for pp in (0, 1):
        P = oracle.Problem(d=1, nx=n, x0=-5.0, x1=5.0, k=3, eq=oracle.EULER,
                           bc=(oracle.INFLOW,) + (oracle.OUTFLOW,) * 3, pp_limiter=pp)
        P.inflow = (tuple(float(v) for v in st) + (0.0,),) + ((0.0,) * 4,) * 3
        if pp == 0:
            V = oracle.step(P, U, oracle.dt(P, U, cfl))
            assert oracle.inadmissible(P, V)
            continue
        V, t = U.copy(), 0.0
        while t < 1.8:
            dt = min(oracle.dt(P, V, cfl), 1.8 - t)
            V = oracle.step(P, V, dt)
            t += dt
            assert oracle.inadmissible(P, V) == 0
        rho = V[0, 0]
        assert np.all(rho > 0.5) and 4.0 < rho.max() < 5.0
        assert abs(rho[:40].mean() - 3.857143) < 0.05


def _dmr_problem(nx, ny, k, pp=1):
    post, pre = inputs.double_mach_states()
    P = oracle.Problem(d=2, nx=nx, ny=ny, x0=0.0, x1=3.0, y0=0.0, y1=1.0, k=k, eq=oracle.EULER,
                       bc=(oracle.INFLOW, oracle.OUTFLOW, oracle.REFLECTIVE, oracle.FRONT), pp_limiter=pp)
    P.inflow = (post, (0.0,) * 4, post, post)
    P.split = (0.0, 0.0, inputs.DMR_FRONT[0], 0.0)
    P.front = inputs.DMR_FRONT
    P.front_ahead = pre
    return P


def test_split_and_front_sides_reduce_to_plain_conditions():
    """The side conditions of Example 4.8 in their limits: a split at the
    side's start changes nothing, a split past its end is an inflow side; a
    front beyond the domain is an inflow side with the behind state, one
    before it an inflow side with the ahead state; a moving front at time t
    is the fixed front shifted by c t (no ghost centre near either line)."""
    nx, ny = 24, 12
    post, pre = inputs.double_mach_states()
    U = inputs.double_mach(nx, ny)
    base = oracle.Problem(d=2, nx=nx, ny=ny, x0=0.0, x1=3.0, y0=0.0, y1=1.0, k=5, eq=oracle.EULER,
                          bc=(oracle.INFLOW, oracle.OUTFLOW, oracle.OUTFLOW, oracle.OUTFLOW), pp_limiter=1)
    base.inflow = (post, (0.0,) * 4, post, post)

    def R(**kw):
        return oracle.residual(oracle.Problem(**{**base.__dict__, **kw}), U)

    r0 = R()
    assert np.array_equal(R(split=(0.0, 0.0, 0.0, 0.0)), r0)
    inflow_bottom = R(bc=(oracle.INFLOW, oracle.OUTFLOW, oracle.INFLOW, oracle.OUTFLOW))
    assert np.array_equal(R(split=(0.0, 0.0, 5.0, 0.0)), inflow_bottom)
    inflow_top = R(bc=(oracle.INFLOW, oracle.OUTFLOW, oracle.OUTFLOW, oracle.INFLOW))
    front = dict(bc=(oracle.INFLOW, oracle.OUTFLOW, oracle.OUTFLOW, oracle.FRONT), front_ahead=pre)
    assert np.array_equal(R(front=(10.0, 0.0, 0.0), **front), inflow_top)
    ahead_top = R(bc=(oracle.INFLOW, oracle.OUTFLOW, oracle.OUTFLOW, oracle.INFLOW), inflow=(post, (0.0,) * 4, post, pre))
    assert np.array_equal(R(front=(-10.0, 0.0, 0.0), **front), ahead_top)
    # ghost centres at x = (i + 1/2) / 8: fronts at 1.3 + y / 2 (y = 1.0625, 1.1875) miss them
    moving = R(front=(1.3 - 0.25, 0.5, 2.5), time=0.1, **front)
    assert np.array_equal(moving, R(front=(1.3, 0.5, 0.0), **front))
    assert not np.array_equal(moving, inflow_top)


@pytest.mark.parametrize("k", [3, 5])
def test_double_mach_reflection_runs_with_the_safeguard(k):
    """Example 4.8 on a coarse 60 x 20 mesh of [0, 3] x [0, 1] to T = 0.2 at
    the guarantee's CFL: the unlimited scheme leaves the admissible set in
    its first step; with the safeguard every step stays admissible, the gas
    behind the incident shock near the inflow keeps the post-shock state, and
    the reflection compresses the gas beyond the post-shock density 8."""
    nx, ny = 60, 20
    U = inputs.double_mach(nx, ny)
    cfl = 1 / 6 if k <= 4 else 1 / 12
    P0 = _dmr_problem(nx, ny, k, pp=0)
    assert oracle.inadmissible(P0, oracle.step(P0, U, oracle.dt(P0, U, cfl)))
    P = _dmr_problem(nx, ny, k)
    V, t = U.copy(), 0.0
    while t < 0.2:
        P.time = t
        dt = min(oracle.dt(P, V, cfl), 0.2 - t)
        V = oracle.step(P, V, dt)
        t += dt
        assert oracle.inadmissible(P, V) == 0, t
    rho = V[0, 0]
    assert np.allclose(rho[ny // 2:, :3], 8.0, rtol=1e-3)
    assert rho.max() > 10.0


@pytest.mark.parametrize("k", [3, 5])
def test_multiscale_lax_type1_and_type2_with_the_safeguard(k):
    """Example 4.6 (600 cells on [-15, 15], outflow, T = 1.4) with the
    safeguard at the guarantee's CFL: both OE types run to T with every
    average admissible (run() retries a step whose stages leave the
    admissible set with half its size), and the small-scale copy of the Lax
    tube undershoots less with Type II than with Type I, as the paper
    observes (its minimum density stays higher)."""
    n = 600
    U = inputs.multiscale_lax(n)
    x = -15.0 + (np.arange(n) + 0.5) * (30.0 / n)
    low = {}
    for oe in (oracle.OE_TYPE1, oracle.OE_TYPE2):
        P = oracle.Problem(d=1, nx=n, x0=-15.0, x1=15.0, k=k, eq=oracle.EULER, bc=(oracle.OUTFLOW,) * 4,
                           pp_limiter=1, oe_type=oe)
        V, t, _ = oracle.run(P, U, T=1.4, cfl=1 / 6 if k <= 4 else 1 / 12)
        assert t == 1.4 and oracle.inadmissible(P, V) == 0
        low[oe] = V[0, 0][x > 0].min()
    assert low[oracle.OE_TYPE2] > low[oracle.OE_TYPE1] > 0.0, low


def test_step_rejection_keeps_the_state_and_halves_the_step():
    """The retry rule of run(): one step of k = 5 at 40x the guarantee's step
    size leaves the admissible set on the multiscale Lax data (step() shows
    it); run() at that CFL discards such steps and retries them with half the
    size, so its three accepted steps end admissible, with rejections
    counted."""
    n = 600
    U = inputs.multiscale_lax(n)
    P = oracle.Problem(d=1, nx=n, x0=-15.0, x1=15.0, k=5, eq=oracle.EULER, bc=(oracle.OUTFLOW,) * 4, pp_limiter=1)
    dt = oracle.dt(P, U, 1 / 12)
    # a step 40x the guarantee's size breaks admissibility on this data
    assert oracle.inadmissible(P, oracle.step(P, U, 40.0 * dt)) > 0
    oracle.rejected_steps(reset=True)
    V, t, st = oracle.run(P, U, nsteps=3, cfl=40.0 / 12.0)
    assert st == 3 and oracle.inadmissible(P, V) == 0
    assert oracle.rejected_steps() > 0
