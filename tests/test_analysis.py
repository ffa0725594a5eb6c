"""Pins of the host-side statistics (Sec. III.B, IV) against closed forms, and of the kurtosis of the
overlap against its exact beta = 0 value on oracle runs."""
import math

import numpy as np
import pytest
from scipy import special

import oracle
from paper_2511_13508_gb300 import analysis, workload


def test_jackknife_of_a_mean_is_the_standard_error():
    rng = np.random.default_rng(1)
    x = rng.standard_normal((40, 3)) * [1.0, 2.0, 0.5] + [0.0, 1.0, -2.0]
    est, err = analysis.jackknife(x)
    assert np.allclose(est, x.mean(0), rtol=0, atol=1e-12)
    assert np.allclose(err, x.std(0, ddof=1) / math.sqrt(len(x)), rtol=1e-12)


def test_jackknife_removes_the_bias_of_a_squared_mean():
    """For theta = mean(x)^2 the jackknife estimate is mean^2 - s^2/n exactly (s^2 unbiased variance)."""
    rng = np.random.default_rng(2)
    x = rng.normal(0.3, 1.0, 25)
    est, _ = analysis.jackknife(x, lambda v: v.mean(0) ** 2)
    assert abs(est - (x.mean() ** 2 - x.var(ddof=1) / len(x))) < 1e-12


def _qstat_from_samples(q):
    """Accumulators of one (sample, T) cell from overlap values."""
    return np.array([len(q), q.sum(), (q ** 2).sum(), (q ** 3).sum(), (q ** 4).sum()])


def test_kurtosis_of_gaussian_and_two_point_overlaps():
    rng = np.random.default_rng(3)
    S, T = 16, 2
    stat = np.ones((S, T, 7))
    qg = np.stack([np.stack([_qstat_from_samples(rng.normal(0, 0.2, 20000)) for _ in range(T)]) for _ in range(S)])
    K, dK = analysis.kurtosis({"stat": stat, "qstat": qg})
    assert np.all(np.abs(K - 3.0) < 4 * dK + 0.02)
    q2 = np.stack([np.stack([_qstat_from_samples(rng.choice([-0.4, 0.4], 1000)) for _ in range(T)]) for _ in range(S)])
    K2, dK2 = analysis.kurtosis({"stat": stat, "qstat": q2})
    assert np.allclose(K2, 1.0, atol=1e-12) and np.all(dK2 < 1e-12)


def test_crossings_of_straight_lines():
    T = np.linspace(0.2, 1.0, 9)
    K1 = 2.0 + 3.0 * (T - 0.43)
    K2 = 2.0 - 1.0 * (T - 0.43)
    c = analysis.crossings(T, K1, K2)
    assert len(c) == 1 and abs(c[0] - 0.43) < 1e-12
    assert len(analysis.crossings(T, K1, K1 + 1.0)) == 0


def test_pq_symmetry_separates_symmetric_and_shifted_histograms():
    rng = np.random.default_rng(4)
    centres = np.arange(201) / 100 - 1
    p = np.exp(-centres ** 2 / (2 * 0.15 ** 2)); p /= p.sum()
    sym = rng.multinomial(200000, p, size=(3, 2))
    ps = np.exp(-(centres - 0.05) ** 2 / (2 * 0.15 ** 2)); ps /= ps.sum()
    shifted = rng.multinomial(200000, ps, size=(3, 2))
    assert np.all(analysis.pq_symmetry(sym) < 1.6)
    assert np.all(analysis.pq_symmetry(shifted) > 10.0)


def kurtosis_beta0(N):
    """Exact kurtosis of q = Re sum_k conj(a_k) b_k / N for two independent draws of the beta = 0 law of
    Eq. (8): intensities s = |a|^4/N ~ Dirichlet(1/2) (so E|a_k|^4 = 1, E|a_k|^2|a_l|^2 = 2/pi for k != l)
    and independent uniform phases (E cos^2 = 1/2, E cos^4 = 3/8)."""
    Eq2 = special.gamma(N / 2) ** 2 / (2 * math.pi * special.gamma((N + 1) / 2) ** 2)
    Eq4 = (3 * N / 8 + 3 * N * (N - 1) / math.pi ** 2) / N ** 4
    return Eq4 / Eq2 ** 2


def test_kurtosis_at_beta0_matches_the_exact_value_on_oracle_runs():
    N, S, R, nT = 8, 4, 8, 2
    J0 = [np.zeros(len(oracle.enumerate_quads(N)))] * S
    pt = oracle.OraclePT([N] * S, J0, workload.geometric_ladder(0.5, 1.0, nT), R, 5, swap_every=0,
                         measure_every=4, resync_every=64)
    pt.sweep(4000)
    K, dK = analysis.kurtosis(pt.observables())
    K0 = kurtosis_beta0(N)
    assert abs(K0 - 3.0) > 0.2  # the finite-N value is far from the Gaussian one
    # measurements 4 sweeps apart are correlated: allow for an integrated autocorrelation of a few
    assert np.all(np.abs(K - K0) < 5 * dK + 0.03), (K, K0, dK)


def test_doubling_windows_detect_relaxation_on_oracle_runs():
    """From the beta = 0 start the coldest chains relax: the first short windows disagree, the last two
    (thermalised) windows agree."""
    N, S, R, nT = 8, 8, 2, 3
    Js = [workload.couplings(N, len(oracle.enumerate_quads(N)), 30 + s) for s in range(S)]
    temps = workload.geometric_ladder(0.15, 1.0, nT)
    pt = oracle.OraclePT([N] * S, Js, temps, R, 6, swap_every=8, measure_every=1, resync_every=64)
    w = analysis.doubling_windows(pt, 11, first=1)
    assert not analysis.thermalised(w[:2], temps)[0]
    assert np.all(analysis.thermalised(w, temps))
    E = [analysis.disorder_average(analysis.thermal_averages(x, temps)["E"])[0][0] for x in w]
    assert E[-1] < E[0]


def test_adaptive_ladder_is_geometric_for_constant_specific_heat():
    """C_V = c: T_i = T_{i-1} / (1 - C/sqrt(c)) exactly, up to T_max."""
    c, C = 9.0, 0.6
    T = analysis.adaptive_ladder([0.1, 2.0], [c, c], 0.2, 1.0, C)
    r = 1.0 / (1.0 - C / 3.0)
    expect = 0.2 * r ** np.arange(len(T) - 1)
    assert np.allclose(T[:-1], expect, rtol=1e-13) and T[-1] == 1.0 and expect[-1] * r >= 1.0


def test_adaptive_ladder_solves_the_implicit_recursion():
    """C_V(T) = a / T^2 (the high-temperature form beta^2 Var_0(H)): the implicit step
    T_i (1 - C T_i / sqrt(a)) = T_{i-1} has the closed-form root T_i = (1 - sqrt(1 - 4 b T_{i-1})) / (2 b),
    b = C / sqrt(a)."""
    a, C = 400.0, 0.6
    Tg = np.linspace(0.05, 3.0, 20001)
    T = analysis.adaptive_ladder(Tg, a / Tg ** 2, 0.2, 1.0, C)
    b = C / math.sqrt(a)
    prev = 0.2
    for t in T[1:-1]:
        root = (1 - math.sqrt(1 - 4 * b * prev)) / (2 * b)
        assert abs(t - root) < 1e-6 * root
        prev = t


def test_adaptive_ladder_rejects_too_small_specific_heat():
    with pytest.raises(ValueError):
        analysis.adaptive_ladder([0.1, 2.0], [0.25, 0.25], 0.2, 1.0, 0.6)


def _synthetic_obs(rng, S, T, E_shift=0.0, q_sd=0.3, n=400):
    """Accumulators of S samples x T temperatures built from explicit per-sample draws."""
    stat = np.zeros((S, T, 7)); qstat = np.zeros((S, T, 5)); qhist = np.zeros((S, T, 201), np.uint64)
    for s in range(S):
        for t in range(T):
            E = rng.normal(-1.0 + 0.1 * s + E_shift, 0.5, n)
            Y = rng.uniform(0.01, 0.02, n)
            stat[s, t] = [n, E.sum(), (E * E).sum(), Y.sum(), (Y * Y).sum(), n * 8.0, n * 64.0]
            q = np.clip(rng.normal(0.0, q_sd, n), -1, 1)
            qstat[s, t] = _qstat_from_samples(q)
            np.add.at(qhist[s, t], np.floor(100 * (q + 1) + 0.5).astype(int), 1)
    return {"stat": stat, "qstat": qstat, "qhist": qhist}


def test_overlap_distribution_coarse_bins():
    h = np.zeros((1, 1, 201), np.uint64)
    h[0, 0, 0] = 3; h[0, 0, 9] = 1; h[0, 0, 10] = 4; h[0, 0, 200] = 2
    P = analysis.overlap_distribution(h)
    assert P.shape == (1, 1, 20)
    assert np.allclose(P[0, 0, :2], [0.4, 0.4]) and P[0, 0, -1] == pytest.approx(0.2) and P.sum() == pytest.approx(1.0)


def test_paired_difference_recovers_a_known_shift_and_zero():
    rng = np.random.default_rng(11)
    S, T, N = 12, 3, 16
    a = _synthetic_obs(np.random.default_rng(5), S, T)
    b = {k: v.copy() for k, v in a.items()}
    same = analysis.paired_difference(a, b, [0.5, 1.0, 1.5], N)
    for key in ("E", "CV", "q2", "q4", "Y2", "Y4"):
        assert np.all(same[key]["diff"] == 0.0), key
    assert np.all(same["Pq"]["diff"] == 0.0)
    # shift every energy of run a by delta: <E>/N moves by delta/N, C_V (a variance) does not move
    delta = 0.37
    a2 = {k: v.copy() for k, v in a.items()}
    n = a2["stat"][..., 0]
    a2["stat"][..., 2] += 2 * delta * a2["stat"][..., 1] + n * delta ** 2
    a2["stat"][..., 1] += n * delta
    d = analysis.paired_difference(a2, b, [0.5, 1.0, 1.5], N)
    assert np.allclose(d["E"]["diff"], delta / N, rtol=1e-12)
    assert np.allclose(d["CV"]["diff"], 0.0, atol=1e-12)
    assert np.allclose(d["E"]["err"], 0.0, atol=1e-12)
    summ = analysis.difference_summary(d)
    assert summ["E"]["max_abs_diff"] == pytest.approx(delta / N)
    del rng


def test_paired_difference_z_of_independent_runs_is_standard():
    """Two independent runs of the same law: the z of the paired differences are about standard normal
    (mean z^2 near 1), and a real shift of 0.05 in <q^2> gives large z."""
    S, T = 16, 40
    a = _synthetic_obs(np.random.default_rng(21), S, T)
    b = _synthetic_obs(np.random.default_rng(22), S, T)
    d = analysis.paired_difference(a, b, np.linspace(0.5, 1.5, T), 16)
    for key in ("E", "CV", "q2", "Y4"):
        assert 0.5 < float((d[key]["z"] ** 2).mean()) < 1.8, key
    assert 0.5 < analysis.difference_summary(d)["Pq"]["mean_z2"] < 1.8
    c = _synthetic_obs(np.random.default_rng(23), S, T, q_sd=0.38)
    d2 = analysis.paired_difference(c, b, np.linspace(0.5, 1.5, T), 16)
    assert np.abs(d2["q2"]["z"]).min() > 5


def test_within_statistical_error_and_bin_width():
    """Independent runs of one law differ by more than 3 sqrt(2) jackknife errors in about 0.3% of cells; a shift of
    the overlap width is flagged; the coarse P(q) bins follow the spread of q (about half its standard deviation)."""
    S, T = 16, 40
    a = _synthetic_obs(np.random.default_rng(31), S, T)
    b = _synthetic_obs(np.random.default_rng(32), S, T)
    d = analysis.paired_difference(a, b, np.linspace(0.5, 1.5, T), 16)
    st = analysis.within_statistical_error(d)
    for key in ("E", "CV", "q2", "Y4", "Pq"):
        assert st[key]["frac_beyond"] < 0.05, (key, st[key])
    c = _synthetic_obs(np.random.default_rng(33), S, T, q_sd=0.38)
    assert analysis.within_statistical_error(analysis.paired_difference(c, b, np.linspace(0.5, 1.5, T), 16))["q2"][
        "frac_beyond"] == 1.0
    assert analysis.overlap_bin_width(b["qhist"]) == 10        # sd 0.3 -> 15 fine bins, capped at 10
    narrow = _synthetic_obs(np.random.default_rng(34), 2, 2, q_sd=0.04)
    assert analysis.overlap_bin_width(narrow["qhist"]) == 2    # sd 0.04 -> 2 fine bins
