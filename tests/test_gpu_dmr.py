"""Double Mach reflection (Example 4.8) on the GPU against the oracle.

The set-up needs two side conditions beyond the plain ones: the bottom wall
imposes the post-shock state on its part x < 1/6 (fam_set_bc_split) and the
top side follows the exact motion of the incident shock (fam_set_bc_front,
rewritten before every stage for its input's time).  The unlimited scheme
leaves the admissible set in its first step, so every run here has the
BP/PP safeguard on.  The oracle's own rounding spread on these runs stays
near 1e-14, so the parity bar is the plain one.
"""
import numpy as np
import pytest

import oracle
from paper_2609_26194_b300 import fam, inputs
from test_gpu_parity import assert_parity, comp_err
from test_oracle_pp import _dmr_problem

pytestmark = pytest.mark.gpu

POST, PRE = inputs.double_mach_states()


def dmr_solver(nx, ny, k, prec=64, tile=None, pp=1, **opt):
    s = fam.Solver(2, nx, ny, box=inputs.DMR_BOX, k=k, equation=fam.EULER, bc=fam.OUTFLOW, precision=prec,
                   pp_limiter=pp, **opt)
    if tile is not None:
        s.set_option("tile2d", tile)
    s.set_bc(0, fam.INFLOW, POST)
    s.set_bc(2, fam.REFLECTIVE)
    s.set_bc_split(2, inputs.DMR_FRONT[0], POST)
    s.set_bc_front(3, *inputs.DMR_FRONT, POST, PRE)
    return s


@pytest.mark.parametrize("k", [3, 4, 5, 6])
def test_residual_at_the_start(k):
    nx, ny = 48, 16
    U = inputs.double_mach(nx, ny)
    s = dmr_solver(nx, ny, k)
    got = s.residual(U)
    s.close()
    assert_parity(got, oracle.residual(_dmr_problem(nx, ny, k), U))


@pytest.mark.parametrize("tile", [0, 2])
@pytest.mark.parametrize("k", [3, 5])
def test_100_steps(k, tile):
    """100 steps at the guarantee's CFL on 48 x 16 (ragged tiles in x and
    y): the front ghosts at t, t + dt, t + dt/2 of every stage and the split
    wall against the oracle's."""
    nx, ny = 48, 16
    U = inputs.double_mach(nx, ny)
    cfl = 1 / 6 if k <= 4 else 1 / 12
    s = dmr_solver(nx, ny, k, tile=tile)
    s.set_state(U)
    s.run_steps(100, cfl)
    s.sync()
    got = s.get_state()
    t, _, nst = s.time()
    s.close()
    want, tw, _ = oracle.run(_dmr_problem(nx, ny, k), U, nsteps=100, cfl=cfl)
    assert nst == 100
    assert_parity(got, want)
    assert abs(t - tw) <= 1e-12 * tw


def test_run_to_T_96x32():
    """The whole run to T = 0.2 (k = 3, CFL 1/6) through fam_run: admissible
    throughout, landing on T, and the oracle's result."""
    nx, ny, k = 96, 32, 3
    U = inputs.double_mach(nx, ny)
    s = dmr_solver(nx, ny, k)
    s.set_state(U)
    s.run(0.2, 1 / 6)
    s.sync()
    t, _, nst = s.time()
    got = s.get_state()
    s.close()
    want, tw, nw = oracle.run(_dmr_problem(nx, ny, k), U, T=0.2, cfl=1 / 6)
    assert t == 0.2 and nst == nw
    assert comp_err(got, want) < 1e-11, comp_err(got, want)
    assert got[0, 0].max() > 10.0


def test_split_and_front_limits_match_plain_conditions():
    """A split at the side's start leaves the run bit-identical to the plain
    wall; a front beyond the domain to an inflow side of the behind state."""
    nx, ny, k = 48, 16, 5
    U = inputs.double_mach(nx, ny)

    def run(setup):
        s = fam.Solver(2, nx, ny, box=inputs.DMR_BOX, k=k, equation=fam.EULER, bc=fam.OUTFLOW, pp_limiter=1)
        s.set_bc(0, fam.INFLOW, POST)
        setup(s)
        s.set_state(U)
        s.run_steps(20, 1 / 12)
        s.sync()
        out = s.get_state()
        s.close()
        return out

    plain = run(lambda s: None)
    assert np.array_equal(run(lambda s: s.set_bc_split(2, 0.0, POST)), plain)
    inflow_top = run(lambda s: s.set_bc(3, fam.INFLOW, POST))
    assert np.array_equal(run(lambda s: s.set_bc_front(3, 10.0, 0.0, 0.0, POST, PRE)), inflow_top)


def test_front_runs_split_even_with_fused_requested():
    nx, ny = 48, 16
    U = inputs.double_mach(nx, ny)
    s = dmr_solver(nx, ny, 5, fused_oe=1, profile=1)
    s.set_state(U)
    s.step(1 / 12)
    ms, steps = s.profile()
    s.close()
    assert steps == 1 and ms[3] > 0.0


def test_fp32_run_stays_admissible():
    nx, ny = 96, 32
    U = inputs.double_mach(nx, ny).astype(np.float32)
    s = dmr_solver(nx, ny, 5, prec=32)
    s.set_state(U)
    s.run(0.2, 1 / 12)
    s.sync()  # raises if a step left the admissible set
    t, _, _ = s.time()
    got = s.get_state()
    s.close()
    assert abs(t - 0.2) < 1e-12
    assert got[0, 0].min() > 1.0 and got[0, 0].max() > 10.0


def test_side_condition_errors():
    s = fam.Solver(2, 32, 16, k=5, equation=fam.EULER, bc=fam.PERIODIC)
    with pytest.raises(fam.FamError) as e:
        s.set_bc_split(2, 0.5, POST)  # a periodic side cannot be split
    assert e.value.code == 1
    with pytest.raises(fam.FamError) as e:
        s.set_bc_front(0, 0.1, 0.0, 0.0, POST, PRE)  # fronts are built for the y-sides
    assert e.value.code == 1
    s.close()
    s = fam.Solver(1, 64, k=5, equation=fam.EULER, bc=fam.OUTFLOW)
    with pytest.raises(fam.FamError) as e:
        s.set_bc_split(0, 0.5, POST[:3])
    assert e.value.code == 7
    s.close()
    # a split side turned periodic afterwards is refused when a step uses it
    s = fam.Solver(2, 32, 16, k=5, equation=fam.EULER, bc=fam.OUTFLOW)
    s.set_bc_split(2, 0.5, POST)
    s.set_bc(2, fam.PERIODIC)
    s.set_bc(3, fam.PERIODIC)
    s.set_state(inputs.double_mach(32, 16))
    with pytest.raises(fam.FamError) as e:
        s.step(0.1)
    assert e.value.code == 1
    s.close()
