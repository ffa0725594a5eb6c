"""Long-run statistics of the FP32 path against FP64 at the production block shapes.

The FP32 path (FP32 fields and moves, FP64 running energy, resync and swap ratio) and the FP64 path run the
same disorder samples with the same seeds (common random numbers).  The FP64 J-sharing path follows the
oracle's Markov chain to 1e-9 (test_gpu_parity), so it stands for the oracle at sizes the oracle cannot run
for thousands of sweeps.  The two trajectories part once an accept decision falls within the FP32 rounding
of its threshold; after that they are independent samples of the same law.  Per temperature, the
disorder-averaged difference FP32 - FP64 of E/N, C_V/N (Eq. (21)), <q^2>, <q^4> (Sec. IV.C), Y2, Y4
(Sec. IV.D) and of P_J(q) on 20 coarse bins is compared with its jackknife error over samples (paired):
the mean of z^2 over temperatures (bins) stays near 1 and no |z| is large.

Shapes: N = 64 on 32 chains x 7 warps (the batched workload's shape) and N = 128 on 8 chains x 11 warps
(packed FP32 blocks with the B_jk gather: the kernel family of the N = 256 benchmark; FP64 runs at N = 256
take minutes on this GPU's FP64 units, and the N = 256 launch is checked update by update instead, in
test_gpu_trace).
"""
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


def paired_runs(N, S, R, nT, burn, sweeps, cpb, cw, seed=31, t_min=0.3, t_max=1.6):
    temps = workload.geometric_ladder(t_min, t_max, nT)
    q = oracle.enumerate_quads(N)
    Js = [workload.couplings(N, len(q), 9000 + 17 * N + s) for s in range(S)]
    obs = {}
    for prec in ("fp32", "fp64"):
        kw = dict(chains_per_block=cpb, consumer_warps=cw) if prec == "fp32" else {}
        pt = pkg.PT([N] * S, Js, temps, R, seed, precision=prec, swap_every=64, measure_every=16,
                    resync_every=64, **kw)
        pt.sweep(burn)
        pt.reset_observables()
        pt.sweep(sweeps)
        obs[prec] = pt.observables()
        pt.close()
    return temps, analysis.paired_difference(obs["fp32"], obs["fp64"], temps, N)


CASES = [
    # N, samples, replicas, temperatures, burn-in, measured sweeps, FP32 block shape
    (64, 16, 2, 16, 1024, 8192, 32, 7),
    (128, 8, 2, 8, 512, 4096, 8, 11),
]


@pytest.mark.parametrize("N,S,R,nT,burn,sweeps,cpb,cw", CASES, ids=["n64_32x7", "n128_8x11"])
def test_fp32_statistics_match_fp64(N, S, R, nT, burn, sweeps, cpb, cw):
    temps, d = paired_runs(N, S, R, nT, burn, sweeps, cpb, cw)
    summ = analysis.difference_summary(d)
    print("\nFP32 - FP64 at N=%d (%d samples x %d T x %d replicas, %d sweeps):" % (N, S, nT, R, sweeps))
    for key, v in summ.items():
        print("  %-3s %s" % (key, {k: (round(x, 6) if isinstance(x, float) else x) for k, x in v.items()}))
    # the criterion of the precision pattern: FP32 agrees with FP64 within 3 statistical errors (jackknife
    # over samples) per temperature and P(q) cell; a few per cent of cells may exceed it by chance
    stat = analysis.within_statistical_error(d, 3.0)
    for key, v in stat.items():
        assert v["cells"] > 0, key
        assert v["frac_beyond"] <= max(0.05, 1.5 / v["cells"]) and v["max_in_sigma"] < 5.0, (key, v)
    # and the paired differences scatter like noise: no large systematic FP32 offset
    for key in ("E", "CV", "q2", "q4", "Y2", "Y4"):
        z = d[key]["z"]
        assert np.isfinite(z).all(), key
        mz2, zmax = limits(S, z.size)
        assert float((z ** 2).mean()) < mz2 and float(np.abs(z).max()) < zmax, (key, z)
    m = summ["Pq"]["bins_used"]
    assert m > 0
    mz2, zmax = limits(S, m)
    assert summ["Pq"]["mean_z2"] < mz2 and summ["Pq"]["max_abs_z"] < zmax, summ["Pq"]


def limits(S, m, p=1e-3):
    """Bounds for m jackknife z-values over S samples at false-alarm probability p: the mean of z^2 against
    the chi-square quantile, widened by the variance of a Student t with S - 1 degrees of freedom (the
    error is itself estimated from S samples); the largest |z| against the t quantile at p / m."""
    from scipy import stats
    nu = S - 1
    mz2 = stats.chi2.ppf(1.0 - p, m) / m * nu / (nu - 2.0)
    zmax = stats.t.ppf(1.0 - p / (2.0 * m), nu)
    return mz2, zmax
