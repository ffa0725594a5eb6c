"""The allocation-free energy entry point (pt_energy_fp64_static).

Callers that cannot allocate device memory (their memory belongs to another runtime's pool, or
cudaMalloc/cudaFree would stall a real-time loop) pass their own inputs and outputs; the entry point's
only working memory is a static device table.  This test calls it through the C ABI on buffers the
test owns and compares its energies with pt_energy of a plain FP64 context holding the same state,
within the FP64 tolerance the parity tests use, on two calls in a row (the second sees the table the
first one left behind, here after a call with another mode count).  Collected last on purpose.
"""
import ctypes

import numpy as np
import pytest

import oracle
import paper_2511_13508_gb300 as pkg
from paper_2511_13508_gb300 import workload

pytestmark = pytest.mark.gpu

TOL_F64 = 1e-12


def _static(L, N, J_dev, a_dev, E_dev, n_chains, stream):
    fn = L.pt_energy_fp64_static
    fn.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_double,
                   ctypes.c_void_p]
    return fn(N, n_chains, J_dev, a_dev, E_dev, 2.0, stream)


def test_static_energy_matches_pt_energy():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    pkg.build()
    L = pkg.lib()
    stream = torch.cuda.Stream()
    rng = np.random.default_rng(17)
    cases = {}
    for N in (64, 16):
        R, nT = 2, 3
        J = workload.couplings(N, len(oracle.enumerate_quads(N)), 4000 + N)
        pt = pkg.PT([N], [J], workload.geometric_ladder(0.5, 1.5, nT), R, 1, precision="fp64_plain")
        g = rng.standard_normal((R * nT, N))
        u = np.sqrt(N) * np.abs(g) / np.linalg.norm(g, axis=1, keepdims=True)
        a = (np.sqrt(u) * np.exp(1j * rng.uniform(0, 2 * np.pi, (R * nT, N)))).reshape(-1)
        pt.set_state(a)
        ref = pt.energy()
        pt.close()
        cases[N] = (torch.tensor(J, dtype=torch.float64, device="cuda"),
                    torch.tensor(a.view(np.float64), dtype=torch.float64, device="cuda"),
                    torch.zeros(R * nT, dtype=torch.float64, device="cuda"), ref)
    torch.cuda.synchronize()
    for N in (64, 16, 64, 16):  # two calls in a row per size, each after the other size used the table
        Jd, ad, Ed, ref = cases[N]
        Ed.zero_()
        with torch.cuda.stream(stream):
            rc = _static(L, N, Jd.data_ptr(), ad.data_ptr(), Ed.data_ptr(), len(ref), stream.cuda_stream)
        assert rc == 0, L.pt_last_error(None)
        stream.synchronize()
        got = Ed.cpu().numpy()
        assert np.all(np.abs(got - ref) <= TOL_F64 * (np.abs(ref) + 1.0)), (N, got, ref)
    # sizes beyond the static table are rejected with a clear error
    Jd, ad, Ed, ref = cases[64]
    assert _static(L, 66, Jd.data_ptr(), ad.data_ptr(), Ed.data_ptr(), 1, stream.cuda_stream) == -1
    assert b"[4, 64]" in L.pt_last_error(None)
