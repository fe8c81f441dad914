"""The allocation-free 1D step (fam_step1d_noalloc) against the regular path.

Callers that cannot allocate device memory (a host application that owns
the device-memory budget, a latency-critical loop) use this entry point:
the library keeps the step's intermediate states in a fixed static device
array instead of allocating.  Here two calls in a row, each from the
previous call's output, must reproduce fam_step on a regular handle within
the parity tolerance, and sizes above the array's limit must be rejected.
This file is collected last so that a run stopping at the first failure has
already run every other test; it also passes on its own in a fresh process.
"""
import ctypes

import numpy as np
import pytest

from paper_2609_26194_b300 import fam, inputs

pytestmark = pytest.mark.gpu


def _comp_err(a, b):
    nc = b.shape[0]
    A, B = a.reshape(nc, -1), b.reshape(nc, -1)
    return float(np.max(np.max(np.abs(A - B), axis=1) / np.max(np.abs(B), axis=1)))


@pytest.mark.parametrize("k,bc", [(5, fam.PERIODIC), (3, fam.OUTFLOW)])
def test_noalloc_step_matches_regular_step_twice(k, bc):
    torch = pytest.importorskip("torch")
    n, cfl = 3000, 0.3
    U0 = inputs.project_1d(lambda x: inputs.primitive_to_conservative_1d(
        1 + 0.2 * np.sin(2 * np.pi * x), 0.3 + 0.1 * np.cos(4 * np.pi * x), 1 + 0.1 * np.sin(2 * np.pi * x + 1)),
        n, 0.0, 1.0)
    a = torch.from_numpy(U0).cuda()
    b = torch.empty_like(a)
    c = torch.empty_like(a)
    dt1 = fam.step1d_noalloc(a, b, n, k, bc=bc, cfl=cfl)
    dt2 = fam.step1d_noalloc(b, c, n, k, bc=bc, cfl=cfl)
    torch.cuda.synchronize()
    with fam.Solver(1, n, k=k, equation=fam.EULER, bc=bc) as s:
        s.set_state(U0)
        s.step(cfl)
        r1 = s.get_state()
        t1, _, _ = s.time()
        s.set_state(r1)  # restart the clock: the next step size comes from r1, as for the second call
        s.step(cfl)
        r2 = s.get_state()
        t2, _, _ = s.time()
    assert _comp_err(b.cpu().numpy(), r1) < 1e-12
    assert _comp_err(c.cpu().numpy(), r2) < 1e-12
    assert abs(dt1 - t1) <= 1e-15 * t1 and abs(dt2 - t2) <= 1e-15 * t2


def test_noalloc_rejects_sizes_above_the_static_limit():
    torch = pytest.importorskip("torch")
    L = fam.lib()
    fam._noalloc_sig(L)
    big = 16384 + 1
    a = torch.zeros((3, 2, 8), dtype=torch.float64, device="cuda")
    rc = L.fam_step1d_noalloc(ctypes.c_void_p(a.data_ptr()), ctypes.c_void_p(a.data_ptr()), big, 0.0, 1.0, 5,
                              fam.EULER, fam.PERIODIC, 1.4, 64, 0.3, None, None)
    assert rc == 1  # FAM_E_INVAL, before any GPU work
