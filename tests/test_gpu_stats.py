"""Long-run statistical parity and scheduling checks of the CUDA path through the C ABI.

FP32 trajectories leave the FP64 oracle's after a few hundred updates (accept decisions at the margin),
so agreement is statistical: per (sample, temperature) thermal averages of E, C_V, <q^2>, Y_4 from
independent GPU and oracle runs on the same couplings agree within their block-averaging errors.
"""
import math

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


def couplings(Ns, seed0=1000):
    return [workload.couplings(N, len(oracle.enumerate_quads(N)), seed0 + s) for s, N in enumerate(Ns)]


def block_stats(pt, nblocks, sweeps):
    """Per block: <E>, C_V = b^2 (<E^2> - <E>^2), <q^2>, <Y4> for every (sample, T)."""
    out = []
    for _ in range(nblocks):
        pt.reset_observables()
        pt.sweep(sweeps)
        o = pt.observables()
        st, qs = o["stat"], o["qstat"]
        n = st[..., 0]
        E = st[..., 1] / n
        out.append(np.stack([E, st[..., 2] / n - E ** 2, qs[..., 2] / qs[..., 0], st[..., 4] / n], -1))
    return np.array(out)  # [block, S, T, 4]


def test_fp32_long_run_matches_oracle_statistically():
    Ns, R, nT = [16] * 4, 2, 8
    temps = workload.geometric_ladder(0.4, 1.6, nT)
    Js = couplings(Ns)
    kw = dict(swap_every=64, measure_every=4, resync_every=64)
    gpu = pkg.PT(Ns, Js, temps, R, 7, precision="fp32", **kw)
    ref = oracle.OraclePT(Ns, Js, temps, R, 8, **kw)  # independent stream
    gpu.sweep(1024)
    ref.sweep(1024)
    nb, sw = 16, 512
    g = block_stats(gpu, nb, sw)
    o = block_stats(ref, nb, sw)
    mg, mo = g.mean(0), o.mean(0)
    se = np.sqrt(g.var(0, ddof=1) / nb + o.var(0, ddof=1) / nb) + 1e-12
    z = (mg - mo) / se
    # 4 samples x 8 T x 4 observables; blocks of 512 sweeps are long against the correlation time
    assert np.mean(np.abs(z) > 3.0) < 0.05, np.round(z, 2)
    assert np.abs(z).max() < 5.5, np.round(z, 2)
    assert np.mean(z ** 2) < 2.0


@pytest.mark.parametrize("prec", ["fp64", "fp64_plain"])
def test_ragged_batch_fp64_trajectory(prec):
    """One launch over samples of N = 32, 48, 64, 96, 128 follows the oracle chain (ragged batch)."""
    Ns, R, nT = [32, 128, 48, 96, 64], 2, 3
    temps = workload.geometric_ladder(0.3, 1.6, nT)
    Js = couplings(Ns)
    kw = dict(swap_every=2, measure_every=1, resync_every=4)
    ref = oracle.OraclePT(Ns, Js, temps, R, 31, **kw)
    ref.sweep(4)
    pt = pkg.PT(Ns, Js, temps, R, 31, precision=prec, **kw)
    pt.sweep(4)
    a0, E0 = ref.state()
    a1, E1 = pt.state()
    assert np.abs(a1 - a0).max() < 1e-9
    assert np.allclose(E1, E0, rtol=1e-9, atol=1e-10)
    o0, o1 = ref.observables(), pt.observables()
    for key in ("qhist", "swap_acc", "swap_att", "mc_acc", "mc_att"):
        assert np.array_equal(o0[key], o1[key]), key


def test_autotune_keeps_the_ensemble_and_picks_a_valid_shape():
    Ns, R, nT = [64] * 4, 2, 16
    temps = workload.geometric_ladder(0.3, 1.6, nT)
    Js = couplings(Ns)
    kw = dict(swap_every=16, measure_every=4, resync_every=32, precision="fp32")
    a = pkg.PT(Ns, Js, temps, R, 3, **kw)
    a.sweep(20)
    blob = a.save()
    s0, E0 = a.state()
    o0 = a.observables()
    shape = a.autotune(4)
    s1, E1 = a.state()
    assert np.array_equal(s0, s1) and np.array_equal(E0, E1) and a.counters == (20, 1)
    o1 = a.observables()
    for k in o0:
        assert np.array_equal(o0[k], o1[k]), k
    G, ncw, spu = shape
    assert G in (8, 16, 32) and ncw > 0 and spu >= 1
    a.sweep(24)
    b = pkg.PT(Ns, Js, temps, R, 3, chains_per_block=G, consumer_warps=ncw, sweeps_per_unit=spu, **kw)
    b.load(blob)
    b.sweep(24)
    assert np.array_equal(a.state()[0], b.state()[0])


def _oracle_blocks(args):
    """One disorder sample on the oracle (spawned process): burn-in, then per block of sweeps the observables."""
    import os, sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import oracle as orc
    N, J, temps, R, seed, burn, nb, sw = args
    pt = orc.OraclePT([N], [J], temps, R, seed, swap_every=64, measure_every=4, resync_every=64)
    pt.sweep(burn)
    out = []
    for _ in range(nb):
        pt.reset_observables()
        pt.sweep(sw)
        o = pt.observables()
        out.append((o["stat"][0], o["qstat"][0], o["qhist"][0]))
    return out


def _block_observables(blocks, temps, N):
    """Per block [nb, S, T]: E/N, C_V/N, <q^2>, Y2, Y4 and P(q) on coarse bins of width 0.1 [nb, S, T, 20]."""
    from paper_2511_13508_gb300 import analysis
    res = []
    for st, qs, qh in blocks:
        ta = analysis.thermal_averages({"stat": st, "qstat": qs}, temps)
        obs = np.stack([ta["E"] / N, ta["CV"] / N, ta["q2"], ta["Y2"], ta["Y4"]], -1)
        res.append((obs, analysis.overlap_distribution(qh, 10)))
    return np.array([r[0] for r in res]), np.array([r[1] for r in res])


N64 = dict(N=64, S=4, R=2, nT=8, burn=1024, nb=16, sw=256)


@pytest.fixture(scope="module")
def oracle_n64_blocks():
    """The oracle's block observables for the N = 64 long-run comparison (one spawned process per sample)."""
    import multiprocessing as mp
    N, S, R, nT, burn, nb, sw = (N64[k] for k in ("N", "S", "R", "nT", "burn", "nb", "sw"))
    temps = workload.geometric_ladder(0.3, 1.6, nT)
    Js = couplings([N] * S, 8100)
    with mp.get_context("spawn").Pool(S) as pool:
        per_sample = pool.map(_oracle_blocks, [(N, Js[s], temps, R, 500 + s, burn, nb, sw) for s in range(S)])
    return [(np.stack([per_sample[s][b][0] for s in range(S)]), np.stack([per_sample[s][b][1] for s in range(S)]),
             np.stack([per_sample[s][b][2] for s in range(S)])) for b in range(nb)]


@pytest.mark.parametrize("cpb,cw", [(32, 11), (16, 11)])
def test_fp32_long_run_matches_oracle_at_n64_production_shapes(cpb, cw, oracle_n64_blocks):
    """N = 64 on the batched workload's block shapes (32 x 11, 16 x 11: packed FP32 blocks, B_jk gathered by
    the copy warp): independent FP32 GPU and FP64 oracle runs on the same couplings; per (sample, T) block means of
    E/N, C_V/N (Eq. (21)), <q^2> (Sec. IV.C), Y2 and Y4 (Sec. IV.D), and P(q) per T pooled over samples, agree
    within their block errors."""
    N, S, R, nT, burn, nb, sw = (N64[k] for k in ("N", "S", "R", "nT", "burn", "nb", "sw"))
    temps = workload.geometric_ladder(0.3, 1.6, nT)
    Js = couplings([N] * S, 8100)
    gpu = pkg.PT([N] * S, Js, temps, R, 71, precision="fp32", chains_per_block=cpb, consumer_warps=cw,
                 swap_every=64, measure_every=4, resync_every=64)
    gpu.sweep(burn)
    gblocks = []
    for _ in range(nb):
        gpu.reset_observables()
        gpu.sweep(sw)
        o = gpu.observables()
        gblocks.append((o["stat"], o["qstat"], o["qhist"]))
    g, gp = _block_observables(gblocks, temps, N)
    o, op = _block_observables(oracle_n64_blocks, temps, N)
    se = np.sqrt(g.var(0, ddof=1) / nb + o.var(0, ddof=1) / nb) + 1e-15
    z = (g.mean(0) - o.mean(0)) / se          # [S, T, 5]
    print("\nN=64 %dx%d vs oracle: max |z| %.2f, mean z^2 %.2f" % (cpb, cw, np.abs(z).max(), (z ** 2).mean()))
    assert np.mean(np.abs(z) > 3.0) < 0.05, np.round(z, 2)
    assert np.abs(z).max() < 5.0 and np.mean(z ** 2) < 2.0
    # P(q) per temperature pooled over samples, on coarse bins holding at least 1% of the mass
    gq, oq = gp.mean(1), op.mean(1)           # [nb, T, 20]
    use = oq.mean(0) >= 0.01
    seq = np.sqrt(gq.var(0, ddof=1) / nb + oq.var(0, ddof=1) / nb) + 1e-15
    zq = ((gq.mean(0) - oq.mean(0)) / seq)[use]
    print("P(q): %d cells, max |z| %.2f, mean z^2 %.2f" % (zq.size, np.abs(zq).max(), (zq ** 2).mean()))
    assert zq.size >= 2 * nT
    assert np.abs(zq).max() < 5.0 and np.mean(zq ** 2) < 2.0
