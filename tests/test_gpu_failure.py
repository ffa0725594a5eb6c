"""Failure detection on the GPU without a fault: a bounded device wait on a flag that nothing sets runs
out, the host reads the timeout status through the same path as the engine's own waits, and the
context goes on with its state untouched (the run continues bit-identically to one without the check)."""
import time

import numpy as np
import pytest

import oracle
import paper_2511_13508_gb300 as pkg
from paper_2511_13508_gb300 import workload

pytestmark = pytest.mark.gpu

PT_ETIMEOUT = -4


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    pkg.build()


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_bounded_wait_times_out_and_the_context_goes_on(prec):
    Ns, R, nT = [32, 48], 2, 4
    temps = workload.geometric_ladder(0.4, 1.6, nT)
    Js = [workload.couplings(n, len(oracle.enumerate_quads(n)), 60 + n) for n in Ns]
    kw = dict(swap_every=8, measure_every=4, resync_every=16)
    a = pkg.PT(Ns, Js, temps, R, 3, precision=prec, **kw)
    b = pkg.PT(Ns, Js, temps, R, 3, precision=prec, **kw)
    a.sweep(8)
    t0 = time.perf_counter()
    rc = a.check_wait(200)
    dt = time.perf_counter() - t0
    assert rc == PT_ETIMEOUT, rc
    assert 0.15 < dt < 10.0, dt
    assert "bounded device wait" in pkg.lib().pt_last_error(a._h).decode()
    a.sweep(8)
    b.sweep(16)
    sa, Ea = a.state()
    sb, Eb = b.state()
    assert np.array_equal(sa, sb) and np.array_equal(Ea, Eb)
    oa, ob = a.observables(), b.observables()
    for k in oa:
        assert np.array_equal(oa[k], ob[k]), k
    assert np.allclose(a.energy(), Ea, rtol=1e-5, atol=1e-5)
    assert a.check_wait(0) != PT_ETIMEOUT  # bad limit: argument error, nothing launched
