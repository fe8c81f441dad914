"""Pins of the oracle's reverse sweep (oracle/torch_fam.py), CPU only.

The differentiable forward is checked against the C oracle (same step to
round-off), and its reverse sweep against central finite differences of the
C oracle's forward with the step sizes held fixed."""
import numpy as np
import pytest
import torch

import oracle
from oracle import torch_fam as tf
from paper_2609_26194_b300 import inputs

RNG = np.random.default_rng(11)


def _state(nx, ny, amp=0.1, mom_noise=0.01, seed=0):
    rng = np.random.default_rng(seed)
    U = inputs.project_2d(lambda X, Y: inputs.primitive_to_conservative_2d(
        1 + 2 * amp * np.sin(2 * np.pi * (X + 2 * Y)), 0.3 + amp * np.cos(2 * np.pi * X),
        -0.2 + amp * np.sin(4 * np.pi * Y), 1 + amp * np.cos(2 * np.pi * (X - Y))), nx, ny)
    U[:, 1:] += mom_noise * rng.standard_normal(U[:, 1:].shape)
    return U


@pytest.mark.parametrize("k", [3, 4, 5, 6])
@pytest.mark.parametrize("bc", ["periodic", "outflow"])
def test_differentiable_forward_equals_c_oracle(k, bc):
    U = _state(11, 9)
    m = tf.Euler2D(11, 9, k, bc=bc)
    obc = oracle.PERIODIC if bc == "periodic" else oracle.OUTFLOW
    P = oracle.Problem(d=2, nx=11, ny=9, k=k, eq=oracle.EULER, bc=(obc,) * 4)
    R = oracle.residual(P, U)
    assert np.max(np.abs(m.residual(torch.tensor(U)).numpy() - R)) < 1e-14 * np.max(np.abs(R))
    assert np.max(np.abs(m.oe(torch.tensor(U), 0.013).numpy() - oracle.oe(P, 0.013, U)[0])) < 1e-15
    assert np.max(np.abs(m.step(torch.tensor(U), 0.013).numpy() - oracle.step(P, U, 0.013))) < 1e-14


@pytest.mark.parametrize("k", [4, 5])
def test_reverse_sweep_matches_central_differences(k):
    nx, ny, steps = 10, 8, 3
    U0 = _state(nx, ny, mom_noise=0.02, seed=k)
    m = tf.Euler2D(nx, ny, k)
    P = oracle.Problem(d=2, nx=nx, ny=ny, k=k, eq=oracle.EULER)
    dts = [0.011, 0.012, 0.0105]
    G = tf.window_functional_grad(U0.shape, (2, 6, 3, 7), 1.0 / nx, 1.0 / ny)
    grad = tf.reverse_sweep(m, U0, dts, G)

    def J(U):
        for dt in dts:
            U = oracle.step(P, U, dt)
        return float((G * U).sum())

    h = 1e-6
    for trial in range(6):
        v = RNG.standard_normal(U0.shape)
        v[:, 1:] *= 0.05
        fd = (J(U0 + h * v) - J(U0 - h * v)) / (2 * h)
        ad = float((grad * v).sum())
        assert abs(fd - ad) < 1e-6 * max(abs(fd), 1e-8), (trial, fd, ad)
    # single entries, including moments
    for (c, mm, j, i) in [(0, 0, 4, 5), (3, 0, 2, 2), (1, 1, 5, 4), (2, 2, 3, 6)]:
        e = np.zeros_like(U0)
        e[c, mm, j, i] = 1.0
        fd = (J(U0 + h * e) - J(U0 - h * e)) / (2 * h)
        assert abs(fd - grad[c, mm, j, i]) < 1e-6 * max(abs(fd), 1e-7), (c, mm, j, i, fd, grad[c, mm, j, i])


def test_reverse_sweep_is_linear_in_the_cotangent():
    nx, ny = 9, 9
    U0 = _state(nx, ny, seed=3)
    m = tf.Euler2D(nx, ny, 5)
    a = RNG.standard_normal(U0.shape)
    b = RNG.standard_normal(U0.shape)
    ga = tf.reverse_sweep(m, U0, [0.01], a)
    gb = tf.reverse_sweep(m, U0, [0.01], b)
    gab = tf.reverse_sweep(m, U0, [0.01], 2 * a - 3 * b)
    assert np.allclose(gab, 2 * ga - 3 * gb, rtol=0, atol=1e-12 * np.abs(gab).max())
