"""Statistics of the CUDA path through the C ABI against the FP64 oracle: the kurtosis of the overlap
K_N(T) (Eq. (kurt)) and the disorder-averaged specific heat (Eq. (21)) with jackknife errors over samples,
and the symmetry of the per-sample overlap distributions P_J(q) (Sec. III.B.1)."""
import numpy as np
import pytest

import oracle
import paper_2511_13508_gb300 as pkg
from paper_2511_13508_gb300 import analysis, workload

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    pkg.build()


def test_kurtosis_and_specific_heat_match_the_oracle():
    N, S, R, nT = 16, 8, 2, 8
    temps = workload.geometric_ladder(0.4, 1.6, nT)
    Js = [workload.couplings(N, len(oracle.enumerate_quads(N)), 700 + s) for s in range(S)]
    kw = dict(swap_every=16, measure_every=4, resync_every=64)
    gpu = pkg.PT([N] * S, Js, temps, R, 17, precision="fp32", **kw)
    ref = oracle.OraclePT([N] * S, Js, temps, R, 18, **kw)
    for sim in (gpu, ref):
        sim.sweep(1024)
        sim.reset_observables()
        sim.sweep(4096)
    og, oo = gpu.observables(), ref.observables()
    Kg, dKg = analysis.kurtosis(og)
    Ko, dKo = analysis.kurtosis(oo)
    z = (Kg - Ko) / np.sqrt(dKg ** 2 + dKo ** 2)
    assert np.abs(z).max() < 4.0, np.round(z, 2)
    Cg, dCg = analysis.specific_heat(og, temps)
    Co, dCo = analysis.specific_heat(oo, temps)
    zc = (Cg - Co) / np.sqrt(dCg ** 2 + dCo ** 2)
    assert np.abs(zc).max() < 4.0, np.round(zc, 2)
    # P_J(q) = P_J(-q) at every temperature (loosely: counts of one run are correlated in time)
    chi_g = analysis.pq_symmetry(og["qhist"])
    chi_o = analysis.pq_symmetry(oo["qhist"])
    assert np.nanmedian(chi_g) < 4.0 and np.nanmedian(chi_o) < 4.0, (np.nanmedian(chi_g), np.nanmedian(chi_o))
