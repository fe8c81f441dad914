"""The final RK stage and the OE in one persistent launch (option "fused_oe").

The fused launch computes the same final stage (eq. 12) and the same OE
(eq. 2dOE_sol / 2dOE_system, Tab. sigma2d) as the two split kernels, tile by
tile, ordered by a task list; it must meet the FP64 parity bar against the
oracle wherever the split path does, and agree with the split path to
rounding.  Grids span many tiles with ragged last tiles in both directions,
and every side condition is exercised, since the task order follows the
ghost images through the sides.
"""
import numpy as np
import pytest

import oracle
from paper_2609_26194_b300 import fam, inputs
from test_gpu_parity import assert_parity, comp_err, make, rounding_spread, smooth_state

pytestmark = pytest.mark.gpu


def _run(d, n, k, bc, U, steps, cfl, fused, tile=None, prec=64, **opt):
    s, P = make(d, n, k, "euler", bc, prec=prec, **opt)
    if tile is not None:
        s.set_option("tile2d", tile)
    s.set_option("fused_oe", fused)
    s.set_state(U)
    s.run_steps(steps, cfl)
    s.sync()
    out = s.get_state()
    t, _, nst = s.time()
    s.close()
    return out, t, nst, P


@pytest.mark.parametrize("tile", [0, 1, 2])
@pytest.mark.parametrize("k", [3, 4, 5, 6])
def test_fused_100_steps_smooth_periodic(k, tile):
    n = (70, 45)
    U = smooth_state(2, n, seed=12, amp=0.2)
    got, t, nst, P = _run(2, n, k, "periodic", U, 100, 0.4, 1, tile)
    split, ts, _, _ = _run(2, n, k, "periodic", U, 100, 0.4, 0, tile)
    want, tw, _ = oracle.run(P, U, nsteps=100, cfl=0.4)
    assert nst == 100
    assert_parity(got, want)
    assert comp_err(got, split) < 1e-13
    assert abs(t - tw) <= 1e-13 * tw


@pytest.mark.parametrize("bc", ["periodic", "outflow"])
@pytest.mark.parametrize("k", [4, 5, 6])
def test_100_steps_multi_tile_256x192_split_and_fused(k, bc):
    """256 x 192 cells: 8 x 24 tiles of 32 x 8 (and 16 x 24 of 16 x 8),
    100 steps; both the split and the fused path against the oracle.  k = 5,
    6: the 1e-12 bar.  k = 4 at CFL 0.4: the OE amplifies rounding on this
    state (the oracle moves by 6e-15, 5e-13, 1e-11, 2.5e-11 after 10, 30, 60,
    100 steps under 2e-16 input noise; 3e-15 after 100 steps without OE), so
    the bar is 10x the oracle's own spread, as for the runs of reading c21."""
    n = (256, 192)
    U = smooth_state(2, n, seed=21 + k, amp=0.2)
    cfl = 0.4 if k == 4 else 0.55
    s, P = make(2, n, k, "euler", bc)
    s.close()
    if k == 4:
        want, spread = rounding_spread(P, U, cfl, nsteps=100)
    else:
        want, _, _ = oracle.run(P, U, nsteps=100, cfl=cfl)
    for fused, tile in ((0, 0), (1, 0), (1, 2)):
        got, _, nst, _ = _run(2, n, k, bc, U, 100, cfl, fused, tile)
        assert nst == 100
        if k == 4:
            assert comp_err(got, want) < max(1e-12, 10.0 * spread), (comp_err(got, want), spread)
        else:
            assert_parity(got, want)


@pytest.mark.parametrize("case", ["reflective", "inflow_outflow", "mixed"])
def test_fused_side_conditions(case):
    """Reflective walls, an inflow side next to outflow sides, and a grid
    periodic in x with walls in y; 30 steps against the oracle."""
    n = (72, 50)
    k, cfl = 5, 0.4
    U = smooth_state(2, n, seed=8, amp=0.2)
    sides = {"reflective": (2, 2, 2, 2), "inflow_outflow": (3, 1, 1, 1), "mixed": (0, 0, 2, 2)}[case]
    inflow = inputs.primitive_to_conservative_2d(np.array(1.1), np.array(0.3), np.array(0.0), np.array(1.0))
    inflow = [float(v) for v in inflow]
    results = []
    for fused in (0, 1):
        s, P = make(2, n, k, "euler", "outflow")
        for side, b in enumerate(sides):
            s.set_bc(side, b, inflow if b == 3 else None)
        s.set_option("fused_oe", fused)
        s.set_state(U)
        s.run_steps(30, cfl)
        s.sync()
        results.append(s.get_state())
        s.close()
    P.bc = sides
    P.inflow = tuple(tuple(inflow) if b == 3 else (0.0,) * 4 for b in sides)
    want, _, _ = oracle.run(P, U, nsteps=30, cfl=cfl)
    assert_parity(results[1], want)
    assert comp_err(results[1], results[0]) < 1e-13


def test_fused_graph_replays_and_single_steps():
    """Odd step counts through graphs, then single steps: the state never
    leaves the handle's state buffer."""
    n, k = (64, 40), 5
    U = smooth_state(2, n, seed=5, amp=0.2)
    s, P = make(2, n, k, "euler", "periodic", fused_oe=1)
    s.set_state(U)
    s.run_steps(7, 0.5)
    s.run_steps(7, 0.5)
    s.step(0.5)
    s.sync()
    got = s.get_state()
    _, _, nst = s.time()
    s.close()
    want, _, _ = oracle.run(P, U, nsteps=15, cfl=0.5)
    assert nst == 15
    assert_parity(got, want)


def test_fused_run_to_T_lands_on_T():
    n, k = (48, 48), 4
    U = smooth_state(2, n, seed=9, amp=0.2)
    s, P = make(2, n, k, "euler", "periodic", fused_oe=1)
    s.set_state(U)
    s.run(0.05, 0.4)
    t, _, nst = s.time()
    got = s.get_state()
    s.close()
    want, tw, nw = oracle.run(P, U, T=0.05, cfl=0.4)
    assert t == 0.05 and nst == nw
    assert_parity(got, want)


def test_fused_full_size_4096_one_step_equals_split():
    """4096^2, k = 5: 131072 tiles of 16 x 8 in one launch; the fused step
    equals the split step to rounding (the split step is held to the oracle
    on sampled cells by the parity suite)."""
    n = 4096
    U = inputs.euler2d_smooth(n)
    outs = []
    for fused in (0, 1):
        s = fam.Solver(2, n, n, k=5, equation=fam.EULER, bc=fam.PERIODIC, tile2d=2, fused_oe=fused)
        s.set_state(U)
        s.run_steps(2, 0.55)
        s.sync()
        outs.append(s.get_state())
        s.close()
    assert comp_err(outs[1], outs[0]) < 1e-13


def test_fused_fp32_matches_split_fp32():
    n = (96, 64)
    U = smooth_state(2, n, seed=3, amp=0.2).astype(np.float32)
    a, _, _, _ = _run(2, n, 5, "periodic", U, 50, 0.5, 0, prec=32)
    b, _, _, _ = _run(2, n, 5, "periodic", U, 50, 0.5, 1, prec=32)
    assert comp_err(b, a) < 1e-5


def test_fused_counts_the_same_traces():
    n = (64, 48)
    U = np.ascontiguousarray(inputs.euler2d_rectangles(64, seed=3, nrect=64, **inputs.ADMISSIBLE_RECT)[:, :, :48])
    counts = []
    for fused in (0, 1):
        s, _ = make(2, n, 5, "euler", "periodic", fused_oe=fused)
        s.set_state(U)
        s.run_steps(5, 0.55)
        s.sync()
        counts.append(s.nonphysical_traces())
        s.close()
    assert counts[0] == counts[1]


def test_fused_profile_and_type1_falls_back_to_split():
    n = (64, 40)
    U = smooth_state(2, n, seed=2, amp=0.2)
    s, P = make(2, n, 5, "euler", "periodic", fused_oe=1, profile=1)
    s.set_state(U)
    s.step(0.5)
    ms, steps = s.profile()
    assert steps == 1 and ms[2] > 0 and ms[3] == 0.0
    s.set_option("oe_type", 1)  # Type I needs grid statistics of the final stage: split
    s.set_option("profile", 1)
    s.set_state(U)
    s.step(0.5)
    ms, _ = s.profile()
    assert ms[3] > 0.0
    got = s.get_state()
    s.close()
    P.oe_type = oracle.OE_TYPE1
    want, _, _ = oracle.run(P, U, nsteps=1, cfl=0.5)
    assert_parity(got, want)


def test_tuner_chooses_among_split_and_fused(tmp_path):
    n = (128, 96)
    U = smooth_state(2, n, seed=4, amp=0.2)
    s, P = make(2, n, 5, "euler", "periodic")
    s.set_state(U)
    cache = str(tmp_path / "tune.txt")
    tile = s.tune(0.5, probe_steps=2, cache_path=cache)
    assert tile in (0, 1, 2) and s.fused_oe in (0, 1)
    line = open(cache).read().strip().split("\t")
    assert int(line[1]) == tile + 3 * s.fused_oe
    s.run_steps(10, 0.5)
    s.sync()
    got = s.get_state()
    s.close()
    want, _, _ = oracle.run(P, U, nsteps=10, cfl=0.5)
    assert_parity(got, want)
