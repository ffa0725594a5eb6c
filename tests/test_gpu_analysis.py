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


def _swap_rates(N, S, R, Js, temps, sweeps=8192, burn=2048):
    pt = pkg.PT([N] * S, Js, temps, R, 5, precision="fp32", swap_every=16, measure_every=4, resync_every=64)
    pt.sweep(burn)
    pt.reset_observables()
    pt.sweep(sweeps)
    o = pt.observables()
    acc = o["swap_acc"].sum((0, 1)) / np.maximum(o["swap_att"].sum((0, 1)), 1)
    cv, _ = analysis.specific_heat(o, temps)
    pt.close()
    return acc, cv


def test_adaptive_ladder_equalises_swap_acceptance():
    """App. A: C_V(T) measured on a ladder of fixed Delta T gives, through T_i = T_{i-1}/(1 - C/sqrt(C_V)),
    a ladder whose neighbouring swaps are accepted at a nearly uniform rate, unlike a geometric ladder of
    the same size and end points."""
    N, S, R = 64, 8, 2
    Js = [workload.couplings(N, len(pkg.enumerate_quads(N)), 800 + s) for s in range(S)]
    Tlin = np.linspace(0.2, 1.6, 32)
    _, cv = _swap_rates(N, S, R, Js, Tlin)
    Tad = analysis.adaptive_ladder(Tlin, cv, 0.2, 1.6, 0.6)
    Tgeo = workload.geometric_ladder(0.2, 1.6, len(Tad))
    a_ad, _ = _swap_rates(N, S, R, Js, Tad)
    a_geo, _ = _swap_rates(N, S, R, Js, Tgeo)
    inner = slice(0, len(Tad) - 2)  # the last step is cut at T_max
    spread_ad = a_ad[inner].std() / a_ad[inner].mean()
    spread_geo = a_geo[inner].std() / a_geo[inner].mean()
    print(f"adaptive ladder ({len(Tad)} T): swap acceptance mean {a_ad[inner].mean():.3f} spread {spread_ad:.3f}; "
          f"geometric: mean {a_geo[inner].mean():.3f} spread {spread_geo:.3f}")
    assert spread_ad < 0.5 * spread_geo
    assert a_ad[inner].min() > a_geo[inner].min()
