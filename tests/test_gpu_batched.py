"""Batched persistent 1D path (fam_batch_*) on the GPU.

Each instance must evolve exactly (bit for bit) as the single-problem path
does, match the FP64 oracle at the parity bar, take its own step size, and
conserve its averages on periodic grids.  The autotuner must not change
results."""
import numpy as np
import pytest

import oracle
from paper_2609_26194_b300 import fam, inputs

pytestmark = pytest.mark.gpu


def _instances(seed=0, n_inst=14):
    rng = np.random.default_rng(seed)
    nx = [int(v) for v in np.rint(np.exp(rng.uniform(np.log(40), np.log(900), n_inst)))]
    ks = [3, 4, 5, 6] * (n_inst // 4) + [5] * (n_inst % 4)
    states = []
    for i, n in enumerate(nx):
        ph = rng.uniform(0, 2 * np.pi, 3)
        amp = rng.uniform(0.05, 0.2)
        f = lambda x, ph=ph, amp=amp: inputs.primitive_to_conservative_1d(
            1 + amp * np.sin(2 * np.pi * x + ph[0]), 0.2 + amp * np.cos(2 * np.pi * x + ph[1]),
            1 + amp * np.sin(4 * np.pi * x + ph[2]))
        states.append(inputs.project_1d(f, n, 0.0, 1.0))
    return nx, ks, states


def _comp_err(a, b):
    nc = b.shape[0]
    A, B = a.reshape(nc, -1), b.reshape(nc, -1)
    return float(np.max(np.max(np.abs(A - B), axis=1) / np.max(np.abs(B), axis=1)))


@pytest.mark.parametrize("bc", [fam.OUTFLOW, fam.PERIODIC])
def test_batch_matches_single_problem_bitwise_and_oracle(bc):
    nx, ks, states = _instances(1)
    b = fam.Batch(nx, ks, bc=bc)
    b.set_state(states)
    b.run(30, 0.3)
    b.sync()
    got = b.get_state()
    t, dt, steps = b.times()
    assert np.all(steps == 30)
    assert len(set(np.round(dt, 15))) > 1  # instances take their own step sizes
    obc = oracle.OUTFLOW if bc == fam.OUTFLOW else oracle.PERIODIC
    for i, (n, k, U) in enumerate(zip(nx, ks, states)):
        with fam.Solver(1, n, k=k, equation=fam.EULER, bc=bc) as s:
            s.set_state(U)
            s.run_steps(30, 0.3)
            single = s.get_state()
            ts, _, _ = s.time()
        assert np.array_equal(got[i], single), i
        assert ts == t[i]
        if i % 3 == 0:
            P = oracle.Problem(d=1, nx=n, k=k, eq=oracle.EULER, bc=(obc,) * 4)
            want, tw, _ = oracle.run(P, U, nsteps=30, cfl=0.3)
            assert _comp_err(got[i], want) < 1e-12
            assert abs(tw - t[i]) < 1e-13
        if bc == fam.PERIODIC:
            for c in range(3):
                assert abs(got[i][c, 0].sum() - U[c, 0].sum()) < 1e-12 * abs(U[c, 0].sum())


def test_batch_riemann_instances_and_tuner():
    rng = np.random.default_rng(4)
    nx = [int(v) for v in np.rint(np.exp(rng.uniform(np.log(64), np.log(2000), 24)))]
    ks = [int(v) for v in rng.integers(4, 7, 24)]
    states = [inputs.euler1d_riemann(n, seed=40 + i) for i, n in enumerate(nx)]
    b = fam.Batch(nx, ks, bc=fam.OUTFLOW)
    b.set_state(states)
    b.run(20, 0.3)
    b.sync()
    ref = b.get_state()
    clock = b.times()
    tx, bps = b.tune(0.3, probe_steps=2)
    assert tx in (64, 128, 256) and bps >= 1
    # the tuner restores the state and every instance's clock
    for r, a in zip(ref, b.get_state()):
        assert np.array_equal(r, a)
    for before, after in zip(clock, b.times()):
        assert np.array_equal(before, after)
    b.set_state(states)
    b.run(20, 0.3)
    b.sync()
    again = b.get_state()
    for r, a in zip(ref, again):
        assert np.array_equal(r, a)
    for i in (0, 7, 13):
        P = oracle.Problem(d=1, nx=nx[i], k=ks[i], eq=oracle.EULER, bc=(oracle.OUTFLOW,) * 4)
        want, _, _ = oracle.run(P, states[i], nsteps=20, cfl=0.3)
        assert _comp_err(again[i], want) < 1e-12
    info = b.info()
    assert info["tile_x"] == tx and info["cells"] == sum(nx)


def test_batch_reports_nonphysical_state():
    nx, ks, states = _instances(2, n_inst=4)
    states[2] = states[2].copy()
    states[2][0, 0, 5] = -1.0
    b = fam.Batch(nx, ks)
    b.set_state(states)
    b.run(2, 0.3)
    with pytest.raises(fam.FamError) as e:
        b.sync()
    assert e.value.code == 4


# ----------------------------------------------------------------------------
# 2D batches (2D Euler)
# ----------------------------------------------------------------------------

def _instances_2d(seed=0):
    rng = np.random.default_rng(seed)
    shapes = [(40, 24, 3), (33, 17, 4), (64, 40, 5), (20, 36, 6), (48, 48, 5), (70, 45, 4), (17, 9, 6)]
    states = []
    for nx, ny, _ in shapes:
        ph = rng.uniform(0, 2 * np.pi, 4)
        amp = rng.uniform(0.05, 0.15)
        f = lambda X, Y, ph=ph, amp=amp: inputs.primitive_to_conservative_2d(
            1 + amp * np.sin(2 * np.pi * (X + Y) + ph[0]), 0.3 + amp * np.cos(2 * np.pi * X + ph[1]),
            -0.2 + amp * np.sin(2 * np.pi * Y + ph[2]), 1 + amp * np.cos(2 * np.pi * (X - Y) + ph[3]))
        states.append(inputs.project_2d(f, nx, ny))
    return [s[0] for s in shapes], [s[1] for s in shapes], [s[2] for s in shapes], states


@pytest.mark.parametrize("bc", [fam.PERIODIC, fam.OUTFLOW])
def test_batch2d_matches_single_problem_bitwise_and_oracle(bc):
    nx, ny, ks, states = _instances_2d(3)
    b = fam.Batch(nx, ks, ny=ny, bc=bc)
    b.set_state(states)
    b.run(20, 0.4)
    b.sync()
    got = b.get_state()
    t, dt, steps = b.times()
    assert np.all(steps == 20)
    assert len(set(np.round(dt, 15))) > 1  # instances take their own step sizes
    info = b.info()
    tile = fam.TILES_2D.index((info["tile_x"], info["tile_y"]))
    obc = oracle.OUTFLOW if bc == fam.OUTFLOW else oracle.PERIODIC
    for i, (n, m, k, U) in enumerate(zip(nx, ny, ks, states)):
        with fam.Solver(2, n, m, k=k, equation=fam.EULER, bc=bc, tile2d=tile) as s:
            s.set_state(U)
            s.run_steps(20, 0.4)
            single = s.get_state()
            ts, _, _ = s.time()
        assert np.array_equal(got[i], single), i
        assert ts == t[i]
        if i % 2 == 0:
            P = oracle.Problem(d=2, nx=n, ny=m, k=k, eq=oracle.EULER, bc=(obc,) * 4)
            want, tw, _ = oracle.run(P, U, nsteps=20, cfl=0.4)
            assert _comp_err(got[i], want) < 1e-12, (i, _comp_err(got[i], want))
            assert abs(tw - t[i]) < 1e-13
        if bc == fam.PERIODIC:
            for c in range(4):
                assert abs(got[i][c, 0].sum() - U[c, 0].sum()) < 1e-12 * abs(U[c, 0].sum())


def test_batch2d_tuner_and_tile_shapes():
    nx, ny, ks, states = _instances_2d(5)
    P = [oracle.Problem(d=2, nx=n, ny=m, k=k, eq=oracle.EULER) for n, m, k in zip(nx, ny, ks)]
    want = [oracle.run(p, U, nsteps=8, cfl=0.4)[0] for p, U in zip(P, states)]
    b = fam.Batch(nx, ks, ny=ny, bc=fam.PERIODIC)
    for tile in (0, 1, 2):
        b.set_option("tile2d", tile)
        b.set_state(states)
        b.run(8, 0.4)
        b.sync()
        for g, w in zip(b.get_state(), want):
            assert _comp_err(g, w) < 1e-12
    b.set_state(states)
    tx, bps = b.tune(0.4, probe_steps=2)
    info = b.info()
    assert tx == info["tile_x"] and (info["tile_x"], info["tile_y"]) in fam.TILES_2D and bps >= 1
    b.set_state(states)
    b.run(8, 0.4)
    b.sync()
    for g, w in zip(b.get_state(), want):
        assert _comp_err(g, w) < 1e-12


def test_batch2d_reports_nonphysical_state():
    nx, ny, ks, states = _instances_2d(6)
    states[1] = states[1].copy()
    states[1][0, 0, 5, 5] = -1.0
    b = fam.Batch(nx, ks, ny=ny)
    b.set_state(states)
    b.run(2, 0.4)
    with pytest.raises(fam.FamError) as e:
        b.sync()
    assert e.value.code == 4


def test_batches_fp32_match_single_problem_bitwise():
    """FP32 batches (1D and 2D) evolve every instance exactly as the FP32
    single-problem kernels do."""
    nx, ks, states = _instances(7, n_inst=6)
    b = fam.Batch(nx, ks, bc=fam.PERIODIC, precision=32)
    b.set_state([U.astype(np.float32) for U in states])
    b.run(10, 0.3)
    b.sync()
    got = b.get_state()
    for i, (n, k, U) in enumerate(zip(nx, ks, states)):
        with fam.Solver(1, n, k=k, equation=fam.EULER, bc=fam.PERIODIC, precision=32) as s:
            s.set_state(U.astype(np.float32))
            s.run_steps(10, 0.3)
            assert np.array_equal(got[i], s.get_state()), i
    nx, ny, ks, states = _instances_2d(8)
    b = fam.Batch(nx, ks, ny=ny, bc=fam.OUTFLOW, precision=32)
    b.set_state([U.astype(np.float32) for U in states])
    b.run(10, 0.4)
    b.sync()
    got = b.get_state()
    info = b.info()
    tile = fam.TILES_2D.index((info["tile_x"], info["tile_y"]))
    for i, (n, m, k, U) in enumerate(zip(nx, ny, ks, states)):
        with fam.Solver(2, n, m, k=k, equation=fam.EULER, bc=fam.OUTFLOW, precision=32, tile2d=tile) as s:
            s.set_state(U.astype(np.float32))
            s.run_steps(10, 0.4)
            assert np.array_equal(got[i], s.get_state()), i
