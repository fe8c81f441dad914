"""Buckley-Leverett (Example 4.3) on the GPU against the oracle.

The equation's physics (flux 4u^2 / (4u^2 + (1-u)^2), the speed bound
max |f'| everywhere, reading c27) and the bound-preserving form of the
safeguard (every check point in [0, 1]) run in the 1D stage kernels.
"""
import numpy as np
import pytest

import oracle
from paper_2609_26194_b300 import fam, inputs
from test_gpu_parity import assert_parity, comp_err, rounding_spread

pytestmark = pytest.mark.gpu


def solver(n, k, **opt):
    return fam.Solver(1, n, box=(-1.0, 1.0, 0.0, 1.0), k=k, equation=fam.BUCKLEY, bc=fam.PERIODIC, **opt)


def problem(n, k, **kw):
    return oracle.Problem(d=1, nx=n, x0=-1.0, x1=1.0, k=k, eq=oracle.BUCKLEY, bc=(oracle.PERIODIC,) * 4, **kw)


@pytest.mark.parametrize("pp", [0, 1])
@pytest.mark.parametrize("k", [3, 4, 5, 6])
def test_residual(k, pp):
    n = 300
    for U in (inputs.buckley_leverett(n),
              inputs.project_1d(lambda x: (0.5 + 0.45 * np.sin(np.pi * x))[None], n, -1.0, 1.0)):
        with solver(n, k, pp_limiter=pp) as s:
            got = s.residual(U)
        assert_parity(got, oracle.residual(problem(n, k, pp_limiter=pp), U))


@pytest.mark.parametrize("k", [3, 5])
def test_run_to_T_with_safeguard(k):
    """The run of Example 4.3 (100 and 400 cells, T = 0.4) through fam_run:
    the oracle's result within 10x its rounding spread, every average in
    [0, 1] to rounding, and mass conserved."""
    cfl = 1 / 6 if k <= 4 else 1 / 12
    for n in (100, 400):
        U = inputs.buckley_leverett(n)
        with solver(n, k, pp_limiter=1) as s:
            s.set_state(U)
            s.run(0.4, cfl)
            s.sync()
            t, _, _ = s.time()
            got = s.get_state()
        assert t == 0.4
        want, spread = rounding_spread(problem(n, k, pp_limiter=1), U, cfl, T=0.4)
        assert comp_err(got, want) < max(1e-12, 10.0 * spread), (n, comp_err(got, want), spread)
        # in [0, 1] to rounding (a convex combination near 0 may round to -1e-93)
        assert got[0, 0].min() >= -1e-14 and got[0, 0].max() <= 1.0 + 1e-14
        assert abs(got[0, 0].sum() - U[0, 0].sum()) < 1e-12 * U[0, 0].sum()


def test_100_steps_without_safeguard_and_in_fp32():
    n, k = 200, 5
    U = inputs.buckley_leverett(n)
    with solver(n, k) as s:
        s.set_state(U)
        s.run_steps(100, 1 / 12)
        s.sync()
        got = s.get_state()
    want, _, _ = oracle.run(problem(n, k), U, nsteps=100, cfl=1 / 12)
    assert_parity(got, want)
    with solver(n, k, precision=32, pp_limiter=1) as s:
        s.set_state(U.astype(np.float32))
        s.run(0.4, 1 / 12)
        s.sync()
        v = s.get_state()[0, 0]
    assert v.min() >= -1e-6 and v.max() <= 1.0 + 1e-6


def test_two_dimensional_grids_are_refused():
    with pytest.raises(fam.FamError) as e:
        fam.Solver(2, 32, 16, k=5, equation=fam.BUCKLEY, bc=fam.PERIODIC)
    assert e.value.code == 7  # FAM_E_UNSUPPORTED
