"""The optional BP/PP safeguard (option pp_limiter) on the GPU against the oracle.

Both sides scale each stage's reconstruction towards the cell average until
the density and the pressure are admissible at the points of a
Gauss--Lobatto decomposition and at the volume Gauss points (1D: inline in
the stage kernel; 2D: a per-cell kernel writing the two scaling factors,
read by the stage kernel for its cells and its ring), and take the CFL
speeds at those points.  The scaling is a switch, so whole runs are held to
the parity bar or, where the oracle's own rounding spread is larger, to 10x
that spread (as for reading c21).  The limited states are built by
cancellation down to densities and pressures 1e-6 / 1e-8 of the average, so one
residual moves by up to 5e-10 and one step size by up to 1e-8 (relative)
under 2e-16 input noise: single residuals and step sizes are held to 10x
that spread too, measured on the same data.
"""
import numpy as np
import pytest

import oracle
from paper_2609_26194_b300 import fam, inputs
from test_gpu_parity import comp_err, make, rounding_spread, smooth_state

pytestmark = pytest.mark.gpu

PRINTED_1D = dict(rho=(0.1, 2.0), umax=1.0, p=(0.1, 10.0))
# instances of the printed-range 1D batch (seed 4 + i) whose reconstructions the safeguard scales
CASES_1D = [(29, 221, 5), (346, 143, 6)]


def _noisy(U, seed):
    return U * (1.0 + 2e-16 * np.random.default_rng(seed).standard_normal(U.shape))


def residual_spread(P, U, want, seeds=(1, 2, 3)):
    return max(comp_err(oracle.residual(P, _noisy(U, s)), want) for s in seeds)


def dt_spread(P, U, cfl, want, seeds=(1, 2, 3)):
    return max(abs(oracle.dt(P, _noisy(U, s), cfl) - want) / want for s in seeds)


def _rect(nx, ny):
    n = max(nx, ny)
    return np.ascontiguousarray(inputs.euler2d_rectangles(n, seed=3, nrect=64)[:, :, :ny, :nx])


@pytest.mark.parametrize("i,n,k", CASES_1D)
def test_residual_1d_with_safeguard(i, n, k):
    U = inputs.euler1d_riemann(n, seed=4 + i, **PRINTED_1D)
    s, P = make(1, n, k, "euler", "outflow", pp_limiter=1)
    P.pp_limiter = 1
    got, want = s.residual(U), oracle.residual(P, U)
    s.close()
    spread = residual_spread(P, U, want)
    P.pp_limiter = 0
    assert not np.array_equal(want, oracle.residual(P, U))  # the safeguard acts on this data
    assert comp_err(got, want) < max(1e-12, 10.0 * spread), (comp_err(got, want), spread)


@pytest.mark.parametrize("tile", [0, 2])
@pytest.mark.parametrize("k", [4, 5, 6])
def test_residual_2d_with_safeguard(k, tile):
    """Rectangles at the shock-run ranges, 48 x 40 cells (ragged tiles): the
    unlimited residual is not finite; the limited one matches the oracle's."""
    U = _rect(48, 40)
    s, P = make(2, (48, 40), k, "euler", "periodic", pp_limiter=1, tile2d=tile)
    P.pp_limiter = 1
    got, want = s.residual(U), oracle.residual(P, U)
    s.close()
    assert np.all(np.isfinite(want))
    spread = residual_spread(P, U, want)
    assert comp_err(got, want) < max(1e-12, 10.0 * spread), (comp_err(got, want), spread)


@pytest.mark.parametrize("d", [1, 2])
def test_safeguard_changes_nothing_on_admissible_data(d):
    n = 300 if d == 1 else (70, 45)
    U = smooth_state(d, n, seed=6, amp=0.2)
    outs = []
    for pp in (0, 1):
        s, _ = make(d, n, 5, "euler", "periodic", pp_limiter=pp)
        outs.append(s.residual(U))
        s.close()
    assert np.array_equal(outs[0], outs[1])


@pytest.mark.parametrize("d", [1, 2])
def test_step_size_from_limited_point_speeds(d):
    if d == 1:
        i, n, k = CASES_1D[0]
        U = inputs.euler1d_riemann(n, seed=4 + i, **PRINTED_1D)
        s, P = make(1, n, k, "euler", "outflow", pp_limiter=1)
    else:
        U = _rect(48, 40)
        s, P = make(2, (48, 40), 5, "euler", "periodic", pp_limiter=1)
    P.pp_limiter = 1
    s.set_state(U)
    s.step(0.2)
    s.sync()
    t, _, _ = s.time()
    s.close()
    want = oracle.dt(P, U, 0.2)
    spread = dt_spread(P, U, 0.2, want)
    assert abs(t - want) <= max(1e-12, 10.0 * spread) * want, (t, want, spread)


@pytest.mark.parametrize("k", [4, 5, 6])
def test_printed_range_rectangles_20_steps_with_safeguard(k):
    """The rectangles at the shock-run ranges advance 20 steps at the paper's
    CFL (0.4 / 0.55), admissible throughout, with no face trace lacking a
    spectral radius, and match the oracle within 10x its rounding spread."""
    U = _rect(48, 40)
    cfl = 0.4 if k == 4 else 0.55
    s, P = make(2, (48, 40), k, "euler", "periodic", pp_limiter=1)
    P.pp_limiter = 1
    s.set_state(U)
    s.run_steps(20, cfl)
    s.sync()  # raises if any step left the admissible set
    got = s.get_state()
    assert s.nonphysical_traces() == 0
    s.close()
    want, spread = rounding_spread(P, U, cfl, nsteps=20)
    assert comp_err(got, want) < max(1e-12, 10.0 * spread), (comp_err(got, want), spread)


@pytest.mark.parametrize("i,n,k", CASES_1D)
def test_printed_range_riemann_1d_100_steps_with_safeguard(i, n, k):
    U = inputs.euler1d_riemann(n, seed=4 + i, **PRINTED_1D)
    s, P = make(1, n, k, "euler", "outflow", pp_limiter=1)
    P.pp_limiter = 1
    s.set_state(U)
    s.run_steps(100, 1 / 12)
    s.sync()
    got = s.get_state()
    s.close()
    want, spread = rounding_spread(P, U, 1 / 12, nsteps=100)
    assert comp_err(got, want) < max(1e-12, 10.0 * spread), (comp_err(got, want), spread)


def test_safeguard_in_fp32_keeps_the_rectangles_admissible():
    U = _rect(48, 40).astype(np.float32)
    s, _ = make(2, (48, 40), 5, "euler", "periodic", prec=32, pp_limiter=1)
    s.set_state(U)
    s.run_steps(20, 0.55)
    s.sync()
    s.close()


def test_safeguard_options():
    s, _ = make(2, (32, 16), 5, "adv", "periodic")
    with pytest.raises(fam.FamError) as e:
        s.set_option("pp_limiter", 1)
    assert e.value.code == 7  # FAM_E_UNSUPPORTED: built for the Euler equations
    s.close()
    s, _ = make(2, (32, 16), 5, "euler", "periodic", pp_limiter=1, fused_oe=1)
    U = smooth_state(2, (32, 16), seed=1, amp=0.2)
    s.set_state(U)
    s.set_option("profile", 1)
    s.step(0.4)
    ms, _ = s.profile()
    assert ms[3] > 0.0  # the safeguard runs the final stage and the OE split
    s.close()


def test_printed_range_batch_completes_with_safeguard():
    """A cut-down 1D batch of the Riemann generator at its printed ranges
    (instances that stop without the safeguard included), CFL 1/12: every
    instance completes 60 steps, each equal to its single-problem run with
    the safeguard and within 10x the oracle's spread of the oracle's."""
    rng = np.random.default_rng(4)
    ns = np.rint(np.exp(rng.uniform(np.log(64), np.log(16384), 400))).astype(int)
    ks = rng.integers(3, 7, 400)
    pick = [i for i in range(400) if ns[i] <= 400][:20]
    for i, _, _ in CASES_1D:
        if i not in pick:
            pick.append(i)
    nx = [int(ns[i]) for i in pick]
    kk = [int(ks[i]) for i in pick]
    states = [inputs.euler1d_riemann(n, seed=4 + i, **PRINTED_1D) for n, i in zip(nx, pick)]
    b = fam.Batch(nx, kk, bc=fam.OUTFLOW)
    b.set_option("pp_limiter", 1)
    b.set_state(states)
    b.run(60, 1 / 12)
    b.sync()
    got = b.get_state()
    _, _, steps = b.times()
    b.close()
    assert np.all(steps == 60)
    for q in (0, len(pick) - 2, len(pick) - 1):
        with fam.Solver(1, nx[q], k=kk[q], equation=fam.EULER, bc=fam.OUTFLOW, pp_limiter=1) as s:
            s.set_state(states[q])
            s.run_steps(60, 1 / 12)
            s.sync()
            single = s.get_state()
        assert np.array_equal(got[q], single), q
        P = oracle.Problem(d=1, nx=nx[q], k=kk[q], eq=oracle.EULER, bc=(oracle.OUTFLOW,) * 4, pp_limiter=1)
        want, spread = rounding_spread(P, states[q], 1 / 12, nsteps=60)
        assert comp_err(got[q], want) < max(1e-12, 10.0 * spread), (q, comp_err(got[q], want), spread)


@pytest.mark.parametrize("k", [3, 4])
def test_shu_osher_at_the_papers_cfl_with_safeguard(k):
    """Example 4.4 (400 cells, inflow / outflow) at Sec. 4's C = 0.55 for
    k = 3, 4, which the unlimited scheme cannot run (it leaves the admissible
    set in the first step, in the oracle too): with the safeguard the GPU run
    reaches T = 1.8 admissible, in the post-shock density band.  One step is
    held to 10x the oracle's rounding spread; at T = 1.8 the OE switch makes
    the run discontinuous in its data (reading c21), so the bar there is 10x
    the oracle's spread over the whole run."""
    n, cfl = 400, 0.55
    st = inputs.shu_osher_inflow()
    s = fam.Solver(1, n, box=(-5.0, 5.0, 0.0, 1.0), k=k, equation=fam.EULER, bc=fam.OUTFLOW, pp_limiter=1)
    s.set_bc(0, fam.INFLOW, st)
    P = oracle.Problem(d=1, nx=n, x0=-5.0, x1=5.0, k=k, eq=oracle.EULER,
                       bc=(oracle.INFLOW,) + (oracle.OUTFLOW,) * 3, pp_limiter=1)
    P.inflow = (tuple(float(v) for v in st) + (0.0,),) + ((0.0,) * 4,) * 3
    U = inputs.shu_osher(n)
    s.set_state(U)
    s.run_steps(1, cfl)
    s.sync()
    want, spread = rounding_spread(P, U, cfl, nsteps=1)
    got = s.get_state()
    assert comp_err(got, want) < max(1e-12, 10.0 * spread), (comp_err(got, want), spread)

    s.set_state(U)
    s.run(1.8, cfl)
    s.sync()  # raises if a step left the admissible set
    t, _, _ = s.time()
    got = s.get_state()
    s.close()
    assert t == 1.8
    want, spread = rounding_spread(P, U, cfl, T=1.8)
    assert comp_err(got, want) < 10.0 * spread, (comp_err(got, want), spread)
    rho = got[0, 0]
    assert np.all(rho > 0.5) and 4.0 < rho.max() < 5.0


EXTREME = {  # Example 4.7: generator, cells, domain, final time
    "sedov": (inputs.sedov_1d, 201, -2.0, 2.0, 1e-3),
    "leblanc": (inputs.leblanc_1d, 200, -10.0, 10.0, 1e-4),
}


@pytest.mark.parametrize("name", ["sedov", "leblanc"])
@pytest.mark.parametrize("k", [3, 5, 6])
def test_extreme_1d_tests_with_safeguard(name, k):
    """Example 4.7 with the safeguard at the CFL of its guarantee, run to
    the final time through fam_run: every step admissible, the oracle's
    result within 10x its rounding spread (these runs are not sensitive:
    the spread stays below 1e-13 at T), mass and energy conserved, the
    Sedov profile mirror-symmetric."""
    gen, n, x0, x1, T = EXTREME[name]
    U = gen(n)
    cfl = 1 / 6 if k <= 4 else 1 / 12
    s = fam.Solver(1, n, box=(x0, x1, 0.0, 1.0), k=k, equation=fam.EULER, bc=fam.OUTFLOW, pp_limiter=1)
    s.set_state(U)
    s.run(T, cfl)
    s.sync()
    t, _, nst = s.time()
    got = s.get_state()
    s.close()
    P = oracle.Problem(d=1, nx=n, x0=x0, x1=x1, k=k, eq=oracle.EULER, bc=(oracle.OUTFLOW,) * 4, pp_limiter=1)
    want, spread = rounding_spread(P, U, cfl, T=T)
    assert t == T
    assert comp_err(got, want) < max(1e-12, 10.0 * spread), (comp_err(got, want), spread)
    for c in (0, 2):
        assert abs(got[c, 0].sum() / U[c, 0].sum() - 1.0) < 1e-12
    if name == "sedov":
        rho = got[0, 0]
        assert np.max(np.abs(rho - rho[::-1])) < 1e-12 * rho.max()


def test_sedov_batch_with_safeguard_equals_single_runs():
    """Sedov blasts at four resolutions and orders in one batch on [-2, 2],
    safeguard on, CFL 1/12, 300 steps each with its own step size: each
    instance equals its single-problem run bit for bit."""
    ns, ks = [101, 201, 301, 401], [3, 4, 5, 6]
    states = [inputs.sedov_1d(n) for n in ns]
    b = fam.Batch(ns, ks, x0=-2.0, x1=2.0, bc=fam.OUTFLOW)
    b.set_option("pp_limiter", 1)
    b.set_state(states)
    b.run(300, 1 / 12)
    b.sync()
    got = b.get_state()
    _, _, steps = b.times()
    b.close()
    assert np.all(steps == 300)
    for q, (n, k) in enumerate(zip(ns, ks)):
        with fam.Solver(1, n, box=(-2.0, 2.0, 0.0, 1.0), k=k, equation=fam.EULER, bc=fam.OUTFLOW,
                        pp_limiter=1) as s:
            s.set_state(states[q])
            s.run_steps(300, 1 / 12)
            s.sync()
            assert np.array_equal(got[q], s.get_state()), q


def _mslax(k, oe):
    n = 600
    s = fam.Solver(1, n, box=(-15.0, 15.0, 0.0, 1.0), k=k, equation=fam.EULER, bc=fam.OUTFLOW, pp_limiter=1,
                   oe_type=oe)
    P = oracle.Problem(d=1, nx=n, x0=-15.0, x1=15.0, k=k, eq=oracle.EULER, bc=(oracle.OUTFLOW,) * 4, pp_limiter=1,
                       oe_type=oe)
    return s, P, inputs.multiscale_lax(n)


@pytest.mark.parametrize("k", [3, 5])
def test_multiscale_lax_type2_with_safeguard(k):
    """Example 4.6 (600 cells, T = 1.4) with Type-II OE: the GPU run through
    fam_run against the oracle's within 10x its rounding spread."""
    s, P, U = _mslax(k, 2)
    cfl = 1 / 6 if k <= 4 else 1 / 12
    s.set_state(U)
    s.run(1.4, cfl)
    s.sync()
    got = s.get_state()
    s.close()
    want, spread = rounding_spread(P, U, cfl, T=1.4)
    assert comp_err(got, want) < max(1e-12, 10.0 * spread), (comp_err(got, want), spread)


@pytest.mark.parametrize("k", [3, 5])
def test_multiscale_lax_type1_undershoots_more_than_type2(k):
    """Type-I OE makes this run chaotic in its data (2e-16 input noise moves
    the oracle's result by ~1e-3), so the GPU's Type-I run is held to what
    the paper fixes: it reaches T admissible, and its small-scale copy's
    minimum density lies below the Type-II run's (Type II undershoots less)."""
    cfl = 1 / 6 if k <= 4 else 1 / 12
    low = {}
    for oe in (1, 2):
        s, _, U = _mslax(k, oe)
        s.set_state(U)
        s.run(1.4, cfl)
        s.sync()  # raises if a step left the admissible set
        t, _, _ = s.time()
        V = s.get_state()
        s.close()
        assert t == 1.4
        x = -15.0 + (np.arange(600) + 0.5) * (30.0 / 600)
        low[oe] = V[0, 0][x > 0].min()
    assert low[2] > low[1] > 0.0, low


def test_step_rejection_matches_the_oracle():
    """k = 5 with Type-I OE at 40x the guarantee's step size on the
    multiscale Lax data: the GPU discards every step whose stage averages
    leave the admissible set and retries it with half the size (the OE
    writes nothing, the clock stays).  Single attempts until 3 steps are
    accepted: the rejected count equals the oracle run()'s, and the state
    its result within 10x its rounding spread (1.5e-9 here: the limited
    check points of this run lie near vacuum)."""
    s, P, U = _mslax(5, 1)
    cfl = 40.0 / 12.0
    s.set_state(U)
    attempts = 0
    while s.time()[2] < 3 and attempts < 200:
        s.step(cfl)
        s.sync()
        attempts += 1
    _, _, accepted = s.time()
    rejected = s.rejected_steps()
    got = s.get_state()
    s.close()
    oracle.rejected_steps(reset=True)
    want, _, st = oracle.run(P, U, nsteps=3, cfl=cfl)
    assert accepted == 3 and st == 3
    assert rejected == oracle.rejected_steps() and rejected > 0
    assert attempts == accepted + rejected
    _, spread = rounding_spread(P, U, cfl, nsteps=3)
    assert comp_err(got, want) < max(1e-12, 10.0 * spread), (comp_err(got, want), spread)


def test_batch_step_rejection_matches_single_runs_and_the_oracle():
    """The first 80 printed-range Riemann instances of at most 300 cells,
    safeguard on, 40 attempts at CFL 1/2 (6x the guarantee's size for k = 5,
    6): each instance discards and retries its own steps, so the batch
    equals every instance's single-problem run of 40 attempts bit for bit
    (state, time, accepted and rejected counts).  Against the oracle: the
    state equals its run to the same number of accepted steps within 10x its
    rounding spread, and the batch's rejected count r lies between the
    oracle's count at those steps and at one step more (attempts after the
    last accepted one are all rejected)."""
    rng = np.random.default_rng(4)
    ns = np.rint(np.exp(rng.uniform(np.log(64), np.log(16384), 4096))).astype(int)
    ks = rng.integers(3, 7, 4096)
    pick = [i for i in range(4096) if ns[i] <= 300][:80]
    nx = [int(ns[i]) for i in pick]
    kk = [int(ks[i]) for i in pick]
    states = [inputs.euler1d_riemann(n, seed=4 + i, **PRINTED_1D) for n, i in zip(nx, pick)]
    cfl, attempts = 0.5, 40
    b = fam.Batch(nx, kk, bc=fam.OUTFLOW)
    b.set_option("pp_limiter", 1)
    b.set_state(states)
    b.run(attempts, cfl)
    b.sync()
    got = b.get_state()
    t, dt, steps = b.times()
    rej = b.rejected_steps()
    _, status, _ = b.health()
    b.close()
    assert np.all(status == 0)
    assert np.all(steps + rej == attempts)
    assert np.sum(rej > 0) >= 10, rej
    for q in range(len(pick)):
        if rej[q] == 0 and q % 8:
            continue  # every rejecting instance, and every 8th one
        with fam.Solver(1, nx[q], k=kk[q], equation=fam.EULER, bc=fam.OUTFLOW, pp_limiter=1) as s:
            s.set_state(states[q])
            s.run_steps(attempts, cfl)
            s.sync()
            assert np.array_equal(got[q], s.get_state()), q
            t1, _, st1 = s.time()
            assert (t1, st1) == (t[q], steps[q]), q
            assert s.rejected_steps() == rej[q], q
        P = oracle.Problem(d=1, nx=nx[q], k=kk[q], eq=oracle.EULER, bc=(oracle.OUTFLOW,) * 4, pp_limiter=1)
        oracle.rejected_steps(reset=True)
        want, t_or, st = oracle.run(P, states[q], nsteps=int(steps[q]), cfl=cfl)
        r_at = oracle.rejected_steps(reset=True)
        oracle.run(P, states[q], nsteps=int(steps[q]) + 1, cfl=cfl)
        r_next = oracle.rejected_steps(reset=True)
        assert st == steps[q] and r_at <= rej[q] <= r_next, (q, r_at, rej[q], r_next)
        assert abs(t_or - t[q]) <= 1e-9 * t_or, q
        _, spread = rounding_spread(P, states[q], cfl, nsteps=int(steps[q]))
        assert comp_err(got[q], want) < max(1e-12, 10.0 * spread), (q, comp_err(got[q], want), spread)


def test_printed_range_rectangles_full_size_sampled_step_with_safeguard():
    """4096^2 rectangles at the shock-run ranges, k = 5, safeguard on: one
    step of the full grid on the GPU (the unlimited scheme leaves the
    admissible set in it).  The step size from the limited point speeds
    equals the oracle's over the whole grid within its rounding spread; the
    oracle recomputes sampled cells on windows (radius 10 > 3 stages x 2 +
    OE 2) with the GPU's step size, each within 10x its window's rounding
    spread."""
    n, cfl = 4096, 0.55
    U = inputs.euler2d_rectangles(n, seed=3, nrect=64)
    s = fam.Solver(2, n, n, k=5, equation=fam.EULER, bc=fam.PERIODIC, pp_limiter=1)
    s.set_state(U)
    s.step(cfl)
    s.sync()
    dt, _, nst = s.time()
    assert nst == 1 and s.rejected_steps() == 0
    V = s.get_state()
    s.close()
    P = oracle.Problem(d=2, nx=n, ny=n, k=5, eq=oracle.EULER, pp_limiter=1)
    want_dt = oracle.dt(P, U, cfl)
    assert abs(dt - want_dt) <= 1e-7 * want_dt, (dt, want_dt)
    rng = np.random.default_rng(7)
    pts = [(0, 0), (n - 1, n - 1)] + [tuple(rng.integers(0, n, 2)) for _ in range(10)]
    R = 10
    dx = 1.0 / n
    Pw = oracle.Problem(**{**P.__dict__, "nx": 2 * R + 1, "ny": 2 * R + 1, "x1": dx * (2 * R + 1),
                           "y1": dx * (2 * R + 1)})
    for j, i in pts:
        jj, ii = (j + np.arange(-R, R + 1)) % n, (i + np.arange(-R, R + 1)) % n
        W = np.ascontiguousarray(U[:, :, jj][:, :, :, ii])
        want = oracle.step(Pw, W, dt)[:, :, R, R]
        noisy = oracle.step(Pw, _noisy(W, j * n + i), dt)[:, :, R, R]
        scale = np.abs(want).max(axis=1, keepdims=True) + 1e-300  # per component
        spread = np.max(np.abs(noisy - want) / scale)
        err = np.max(np.abs(V[:, :, j, i] - want) / scale)
        assert err < max(1e-12, 10.0 * spread), ((j, i), err, spread)


def test_step_rejection_2d_matches_the_oracle():
    """The printed-range rectangles (48 x 40, k = 5) at 1000x the guarantee's
    step size (their near-vacuum check points keep the size small, so a
    smaller factor breaks nothing): the 2D stage kernels flag output averages
    outside the admissible set and the OE discards the step; single attempts
    until 3 steps are accepted: the rejected count equals the oracle run()'s,
    and the state its result within 10x its rounding spread."""
    U = _rect(48, 40)
    cfl = 1000.0 / 12.0
    s, P = make(2, (48, 40), 5, "euler", "periodic", pp_limiter=1)
    P.pp_limiter = 1
    s.set_state(U)
    attempts = 0
    while s.time()[2] < 3 and attempts < 200:
        s.step(cfl)
        s.sync()
        attempts += 1
    rejected = s.rejected_steps()
    got = s.get_state()
    s.close()
    oracle.rejected_steps(reset=True)
    want, _, st = oracle.run(P, U, nsteps=3, cfl=cfl)
    assert st == 3 and rejected == oracle.rejected_steps() and rejected > 0
    assert attempts == 3 + rejected
    _, spread = rounding_spread(P, U, cfl, nsteps=3)
    assert comp_err(got, want) < max(1e-12, 10.0 * spread), (comp_err(got, want), spread)
