"""Smooth-accuracy runs of the paper (Examples 4.1, 4.2) on the GPU path.

Same setups and bounds as the oracle pins in test_oracle_pins.py (Type-II
OE, C_CFL = 0.1 with dx^(k/3), L1 error = mean over cells), and the GPU
errors must equal the oracle's errors for the same run to 1 % (the runs
differ only by rounding, which over thousands of steps is a visible part of
errors of 1e-10)."""
import numpy as np
import pytest

import oracle
from golden_io import accuracy
from paper_2609_26194_b300 import fam, inputs

pytestmark = pytest.mark.gpu
ACC = accuracy()


def _gpu_run(d, n, k, U, T, box):
    with fam.Solver(d, n, n if d == 2 else 1, box=box, k=k, equation=fam.EULER, bc=fam.PERIODIC,
                    smooth_dt=1) as s:
        s.set_state(U)
        s.run(T, 0.1)
        t, _, _ = s.time()
        assert t == T
        return s.get_state()


@pytest.mark.parametrize("k", [3, 4, 5, 6])
def test_smooth_euler_1d_gpu_matches_printed_table(k):
    errs = {}
    for n in (20, 40):
        U = inputs.euler1d_smooth(n)
        V = _gpu_run(1, n, k, U, 2.0, (0.0, 2.0, 0.0, 1.0))
        ea, em = np.abs(V[0, 0] - U[0, 0]).mean(), np.abs(V[0, 1] - U[0, 1]).mean()
        ga, gm = ACC[("eu1_avg", n)][k - 3], ACC[("eu1_mom", n)][k - 3]
        assert 0.6 < em / gm < 1.4 and 0.5 < ea / ga < 2.5, (k, n, ea, ga, em, gm)
        P = oracle.Problem(d=1, nx=n, x0=0, x1=2, k=k, eq=oracle.EULER)
        W, _, _ = oracle.run(P, U, T=2.0, cfl=0.1, smooth=True)
        ow = np.abs(W[0, 0] - U[0, 0]).mean()
        assert abs(ea - ow) < 1e-2 * ow
        errs[n] = ea
    order = np.log2(errs[20] / errs[40])
    printed = np.log(ACC[("eu1_avg", 20)][k - 3] / ACC[("eu1_avg", 40)][k - 3]) / np.log(2)
    assert abs(order - printed) < 0.35


@pytest.mark.parametrize("k,ns", [(3, (20, 40)), (4, (20, 40)), (5, (20, 40)), (6, (20,))])
def test_smooth_euler_2d_gpu_matches_printed_table(k, ns):
    errs = []
    for n in ns:
        U = inputs.euler2d_smooth_accuracy(n)
        V = _gpu_run(2, n, k, U, 2.0, (0.0, 2.0, 0.0, 2.0))
        e = np.abs(V[0, 0] - U[0, 0]).mean()
        g = ACC[("eu2_avg", n)][k - 3]
        assert 0.5 < e / g < 2.5, (k, n, e, g)
        errs.append(e)
    if len(ns) == 2:
        order = np.log(errs[0] / errs[1]) / np.log(ns[1] / ns[0])
        printed = np.log(ACC[("eu2_avg", ns[0])][k - 3] / ACC[("eu2_avg", ns[1])][k - 3]) / np.log(ns[1] / ns[0])
        assert abs(order - printed) < 0.3


@pytest.mark.parametrize("k", [5, 6])
def test_smooth_burgers_gpu_matches_oracle_and_table(k):
    from test_oracle_pins import _burgers_exact_avg
    T = 0.5 / np.pi
    for n in (30, 60, 90):
        U = inputs.burgers_smooth(n)
        with fam.Solver(1, n, box=(0.0, 2.0, 0, 1), k=k, equation=fam.BURGERS, bc=fam.PERIODIC, smooth_dt=1) as s:
            s.set_state(U)
            s.run(T, 0.1)
            V = s.get_state()
        e = np.abs(V[0, 0] - _burgers_exact_avg(n, T)).mean()
        g = ACC[("bur_avg", n)][k - 3]
        assert 0.4 < e / g < 2.2, (k, n, e, g)
