"""The random-frequency mode-locked graph on the GPU (pt_create_graph, quadruplet-list FP64 path)
against the FP64 oracle running the same graphs: same seeds and Philox counters give the same Markov
chain (moves, swaps, resync) and the same observables."""
import numpy as np
import pytest

import oracle
import paper_2511_13508_gb300 as pkg
from paper_2511_13508_gb300 import workload

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    pkg.build()


def _graphs(Ns, seed0):
    graphs = [pkg.fmc_graph(workload.random_frequencies(n, seed0 + s)) for s, n in enumerate(Ns)]
    Js = [workload.couplings(n, len(g), seed0 + 50 + s) for s, (n, g) in enumerate(zip(Ns, graphs))]
    return graphs, Js


@pytest.mark.parametrize("Ns,R,nT,sweeps", [([16, 16], 2, 4, 24), ([32, 24, 40], 2, 3, 12), ([64], 3, 2, 6)])
def test_graph_trajectory_matches_oracle(Ns, R, nT, sweeps):
    temps = workload.geometric_ladder(0.3, 1.6, nT)
    graphs, Js = _graphs(Ns, 300)
    kw = dict(swap_every=4, measure_every=2, resync_every=8)
    ref = oracle.OraclePT(Ns, Js, temps, R, 77, graphs=graphs, **kw)
    ref.sweep(sweeps)
    pt = pkg.PT(Ns, Js, temps, R, 77, precision="fp64_plain", graphs=graphs, **kw)
    pt.sweep(sweeps)
    a0, E0 = ref.state()
    a1, E1 = pt.state()
    assert np.abs(a1 - a0).max() < 1e-9
    assert np.allclose(E1, E0, rtol=1e-9, atol=1e-11)
    o0, o1 = ref.observables(), pt.observables()
    for key in ("qhist", "swap_acc", "swap_att", "mc_acc", "mc_att"):
        assert np.array_equal(o0[key], o1[key]), key
    assert np.allclose(o0["stat"], o1["stat"], rtol=1e-9, atol=1e-10)
    # full recomputation on the device equals the oracle's energy of the same state
    assert np.allclose(pt.energy(), E0, rtol=1e-9, atol=1e-11)


def test_graph_creation_checks():
    Ns = [16]
    graphs, Js = _graphs(Ns, 5)
    temps = workload.geometric_ladder(0.5, 1.5, 2)
    with pytest.raises(pkg.PTError):  # explicit graphs run on the quadruplet-list path only
        pkg.PT(Ns, Js, temps, 2, 1, precision="fp32", graphs=graphs)
    bad = graphs[0].copy(); bad[0, 1] = bad[0, 0]
    with pytest.raises(pkg.PTError):
        pkg.PT(Ns, Js, temps, 2, 1, precision="fp64_plain", graphs=[bad])
    bad = graphs[0].copy(); bad[3, 2] = 16
    with pytest.raises(pkg.PTError):
        pkg.PT(Ns, Js, temps, 2, 1, precision="fp64_plain", graphs=[bad])
    with pytest.raises(ValueError):
        pkg.PT(Ns, [Js[0][:-1]], temps, 2, 1, precision="fp64_plain", graphs=graphs)
