"""Health reporting of the CUDA path against the FP64 oracle.

Without the paper's optional positivity limiter (Sec. 2.3 remarks, Alg. 1),
a reconstructed face trace can leave the admissible set while every cell
average stays admissible; its spectral radius is then undefined and the
Rusanov flux takes the other trace's (IEEE maxNum).  Both sides count the
face quadrature points where that happens, and both stop at the first step
whose averages are no longer admissible (rho <= 0 or p <= 0, or a non-finite
value).  The counts must be equal, and so must the step at which a run
stops: the shock-run ranges of the rectangle workload (rho, p in [0.1, 5],
|u|, |v| <= 1) and of the 1D Riemann workload (rho in [0.1, 2], |u| <= 1,
p in [0.1, 10]) are run here on cut-down grids.

The batched path's grid barrier has a bounded wait; a test hook makes the
barrier wait for one block more than were launched, so that the wait runs
out after a 1 ms limit and the launch reports FAM_E_TIMEOUT.
"""
import time

import numpy as np
import pytest

import oracle
from paper_2609_26194_b300 import fam, inputs

pytestmark = pytest.mark.gpu

PRINTED_1D = dict(rho=(0.1, 2.0), umax=1.0, p=(0.1, 10.0))


def _solver2d(n, k, bc=fam.PERIODIC, tile=None):
    nx, ny = n
    s = fam.Solver(2, nx, ny, k=k, equation=fam.EULER, bc=bc)
    if tile is not None:
        s.set_option("tile2d", tile)
    obc = oracle.PERIODIC if bc == fam.PERIODIC else oracle.OUTFLOW
    P = oracle.Problem(d=2, nx=nx, ny=ny, k=k, eq=oracle.EULER, bc=(obc,) * 4)
    return s, P


def _rect(nx, ny, seed=3):
    """Rectangles at the shock-run ranges on an nx x ny grid (periodic
    painting on the square, cropped)."""
    n = max(nx, ny)
    return np.ascontiguousarray(inputs.euler2d_rectangles(n, seed=seed, nrect=64)[:, :, :ny, :nx])


@pytest.mark.parametrize("tile", [0, 1, 2])
@pytest.mark.parametrize("bc", [fam.PERIODIC, fam.OUTFLOW])
def test_trace_count_of_one_residual_2d(tile, bc):
    """70 x 45 cells: several tiles in each direction with ragged last tiles,
    so every face is counted once whichever tile computes it."""
    k = 5
    U = _rect(70, 45)
    s, P = _solver2d((70, 45), k, bc, tile)
    oracle.trace_reset()
    want_R = oracle.residual(P, U)
    want = oracle.trace_count()
    got_R = s.residual(U)
    got = s.nonphysical_traces()
    s.close()
    assert want > 0
    assert got == want, (got, want)
    assert np.array_equal(np.isnan(got_R), np.isnan(want_R))


@pytest.mark.parametrize("k", [3, 4, 5, 6])
def test_trace_count_of_one_residual_1d(k):
    n = 1000  # 7 full 128-cell tiles and a ragged one
    U = inputs.euler1d_riemann(n, seed=11, **PRINTED_1D)
    with fam.Solver(1, n, k=k, equation=fam.EULER, bc=fam.OUTFLOW) as s:
        P = oracle.Problem(d=1, nx=n, k=k, eq=oracle.EULER, bc=(oracle.OUTFLOW,) * 4)
        oracle.trace_reset()
        oracle.residual(P, U)
        want = oracle.trace_count()
        s.residual(U)
        assert s.nonphysical_traces() == want


def _oracle_steps(P, U, cfl, nmax):
    """Oracle steps until the averages leave the admissible set: returns
    (steps taken, 1-based step that failed or 0, trace count, state)."""
    oracle.trace_reset()
    for s in range(1, nmax + 1):
        U = oracle.step(P, U, oracle.dt(P, U, cfl))
        if oracle.inadmissible(P, U):
            return s, s, oracle.trace_count(), U
    return nmax, 0, oracle.trace_count(), U


def _gpu_steps(solver, U, cfl, nmax):
    solver.set_state(U)
    for s in range(1, nmax + 1):
        solver.step(cfl)
        try:
            solver.sync()
        except fam.FamError as e:
            assert e.code == 4  # FAM_E_NONPHYSICAL
            return s, s, solver.nonphysical_traces()
    return nmax, 0, solver.nonphysical_traces()


@pytest.mark.parametrize("k", [4, 5, 6])
def test_rectangles_at_printed_ranges_stop_at_the_oracles_step(k):
    cfl = 0.4 if k == 4 else 0.55
    U = _rect(48, 40)
    s, P = _solver2d((48, 40), k)
    _, o_bad, o_tr, _ = _oracle_steps(P, U, cfl, 20)
    _, g_bad, g_tr = _gpu_steps(s, U, cfl, 20)
    s.close()
    assert o_bad > 0, "the printed ranges are expected to leave the admissible set"
    assert g_bad == o_bad
    assert g_tr == o_tr


def test_riemann_1d_at_printed_ranges_count_or_stop_like_the_oracle():
    """The 1D shock workload's generator at its printed ranges, 3000 cells,
    k = 5, CFL 0.3, up to 60 steps: the GPU completes or stops where the
    oracle does, with the same count of traces without a spectral radius."""
    n, k, cfl = 3000, 5, 0.3
    U = inputs.euler1d_riemann(n, seed=2, **PRINTED_1D)
    P = oracle.Problem(d=1, nx=n, k=k, eq=oracle.EULER, bc=(oracle.OUTFLOW,) * 4)
    with fam.Solver(1, n, k=k, equation=fam.EULER, bc=fam.OUTFLOW) as s:
        o_n, o_bad, o_tr, o_U = _oracle_steps(P, U, cfl, 60)
        g_n, g_bad, g_tr = _gpu_steps(s, U, cfl, 60)
        assert (g_n, g_bad, g_tr) == (o_n, o_bad, o_tr)
        if g_bad == 0:
            got = s.get_state()
            nc = 3
            err = np.max(np.max(np.abs(got - o_U).reshape(nc, -1), axis=1) /
                         np.max(np.abs(o_U).reshape(nc, -1), axis=1))
            assert err < 1e-12


def test_batch_at_printed_ranges_reports_each_instance_like_the_oracle():
    """A cut-down 1D batch of the Riemann generator at its printed ranges:
    per instance, the step at which it stops (or none) and the trace count
    equal the oracle's; instances that complete match the oracle's state."""
    rng = np.random.default_rng(40)
    n_inst, steps, cfl = 24, 40, 0.3
    nx = [int(v) for v in np.rint(np.exp(rng.uniform(np.log(64), np.log(600), n_inst)))]
    ks = [int(v) for v in rng.integers(3, 7, n_inst)]
    states = [inputs.euler1d_riemann(n, seed=100 + i, **PRINTED_1D) for i, n in enumerate(nx)]
    b = fam.Batch(nx, ks, bc=fam.OUTFLOW)
    b.set_state(states)
    b.run(steps, cfl)
    try:
        b.sync()
        any_bad = False
    except fam.FamError as e:
        assert e.code == 4
        any_bad = True
    ntr, st, bad = b.health()
    got = b.get_state()
    _, _, nsteps = b.times()
    b.close()
    seen_bad = False
    for i in range(n_inst):
        P = oracle.Problem(d=1, nx=nx[i], k=ks[i], eq=oracle.EULER, bc=(oracle.OUTFLOW,) * 4)
        o_n, o_bad, o_tr, o_U = _oracle_steps(P, states[i], cfl, steps)
        assert bad[i] == o_bad, (i, bad[i], o_bad)
        assert (st[i] != 0) == (o_bad != 0)
        assert ntr[i] == o_tr, (i, ntr[i], o_tr)
        assert nsteps[i] == o_n
        seen_bad |= o_bad != 0
        if o_bad == 0:
            err = np.max(np.max(np.abs(got[i] - o_U).reshape(3, -1), axis=1) /
                         np.max(np.abs(o_U).reshape(3, -1), axis=1))
            assert err < 1e-12, (i, err)
    assert any_bad == seen_bad


def _smooth_batch(n_inst=10, seed=5):
    rng = np.random.default_rng(seed)
    nx = [int(v) for v in rng.integers(60, 700, n_inst)]
    ks = [3, 4, 5, 6] * (n_inst // 4) + [5] * (n_inst % 4)
    states = []
    for n in nx:
        ph = rng.uniform(0, 2 * np.pi, 2)
        f = lambda x, ph=ph: inputs.primitive_to_conservative_1d(
            1 + 0.1 * np.sin(2 * np.pi * x + ph[0]), 0.2 + 0.1 * np.cos(2 * np.pi * x + ph[1]), np.ones_like(x))
        states.append(inputs.project_1d(f, n, 0.0, 1.0))
    return nx, ks, states


def test_batch_grid_barrier_wait_runs_out_and_reports_timeout():
    nx, ks, states = _smooth_batch()
    b = fam.Batch(nx, ks, bc=fam.PERIODIC)
    b.set_state(states)
    b.run(1, 0.3)
    b.sync()
    b.set_option("wait_limit_ns", 1e6)  # 1 ms
    b.set_option("test_barrier_extra", 1)
    t0 = time.perf_counter()
    b.run(2, 0.3)
    with pytest.raises(fam.FamError) as e:
        b.sync()
    assert e.value.code == 5  # FAM_E_TIMEOUT
    assert time.perf_counter() - t0 < 5.0
    # the same handle runs again once the hook is off and the state is set
    b.set_option("test_barrier_extra", 0)
    b.set_option("wait_limit_ns", 0)
    b.set_state(states)
    b.run(3, 0.3)
    b.sync()
    again = b.get_state()
    b.close()
    # and a fresh handle runs normally, to the same result
    f = fam.Batch(nx, ks, bc=fam.PERIODIC)
    f.set_state(states)
    f.run(3, 0.3)
    f.sync()
    fresh = f.get_state()
    f.close()
    for a, c in zip(again, fresh):
        assert np.array_equal(a, c)
    P = oracle.Problem(d=1, nx=nx[0], k=ks[0], eq=oracle.EULER, bc=(oracle.PERIODIC,) * 4)
    want, _, _ = oracle.run(P, states[0], nsteps=3, cfl=0.3)
    assert np.max(np.abs(fresh[0] - want)) < 1e-12 * np.max(np.abs(want))
