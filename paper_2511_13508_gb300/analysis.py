"""Host-side statistics over the engine's accumulators (arXiv 2511.13508, Sec. III.B and IV).

- thermal averages per disorder sample, Eq. (totave), from the per-(sample, T) sums of `PT.observables()`;
- disorder averages over samples, Eq. (DisAver), with leave-one-sample-out jackknife errors (Sec. III.B.3);
- specific heat C_V = beta^2 (<E^2> - <E>^2) per sample, then averaged (Eq. (21));
- kurtosis of the overlap, K_N(T) = mean<q^4> / (mean<q^2>)^2 (Eq. (kurt), with <q> = 0 exactly by the
  global-phase symmetry), and the temperatures where the curves of two sizes cross;
- thermalisation checks (Sec. III.B.1): averages over windows of doubling length, and the symmetry of the
  per-sample overlap distribution P_J(q) = P_J(-q).

Layouts: stat [S][T][7] = (n, E, E^2, Y2, Y4, I, I^2), qstat [S][T][5] = (n, q, q^2, q^3, q^4),
qhist [S][T][201] with bin b centred at q = b/100 - 1.
"""
from __future__ import annotations

import numpy as np


def thermal_averages(obs: dict, temps) -> dict:
    """Per-sample thermal averages [S, T] (Eq. (totave)) and C_V = beta^2 (<E^2> - <E>^2)."""
    st = np.asarray(obs["stat"], np.float64)
    qs = np.asarray(obs["qstat"], np.float64)
    n = st[..., 0]
    nq = np.maximum(qs[..., 0], 1.0)
    beta = 1.0 / np.asarray(temps, np.float64)
    E, E2 = st[..., 1] / n, st[..., 2] / n
    return {
        "n": n, "E": E, "E2": E2, "CV": beta[None, :] ** 2 * (E2 - E * E),
        "Y2": st[..., 3] / n, "Y4": st[..., 4] / n, "I": st[..., 5] / n, "I2": st[..., 6] / n,
        "q": qs[..., 1] / nq, "q2": qs[..., 2] / nq, "q4": qs[..., 4] / nq,
    }


def jackknife(per_sample: np.ndarray, estimator=lambda x: x.mean(0)):
    """Leave-one-sample-out jackknife over axis 0 of `per_sample` (or of every array in a tuple):
    returns (estimate with first-order bias removed, standard error)."""
    arrays = per_sample if isinstance(per_sample, tuple) else (per_sample,)
    S = arrays[0].shape[0]
    full = np.asarray(estimator(*arrays))
    if S < 2:
        return full, np.full_like(full, np.nan, dtype=np.float64)
    loo = np.stack([np.asarray(estimator(*[np.delete(a, i, axis=0) for a in arrays])) for i in range(S)])
    mean_loo = loo.mean(0)
    est = S * full - (S - 1) * mean_loo
    err = np.sqrt((S - 1) / S * ((loo - mean_loo) ** 2).sum(0))
    return est, err


def disorder_average(per_sample: np.ndarray):
    """Eq. (DisAver) with its jackknife error: mean over samples (axis 0)."""
    return jackknife(np.asarray(per_sample, np.float64))


def specific_heat(obs: dict, temps):
    """Disorder-averaged C_V(T) per temperature and its jackknife error."""
    return disorder_average(thermal_averages(obs, temps)["CV"])


def kurtosis(obs: dict, temps=None):
    """K_N(T) = mean<q^4> / (mean<q^2>)^2 over samples, with its jackknife error."""
    ta = thermal_averages(obs, temps if temps is not None else np.ones(np.asarray(obs["stat"]).shape[1]))
    return jackknife((ta["q4"], ta["q2"]), lambda q4, q2: q4.mean(0) / q2.mean(0) ** 2)


def crossings(T, K1, K2):
    """Temperatures where K1(T) - K2(T) changes sign, by linear interpolation between ladder points."""
    T = np.asarray(T, np.float64)
    d = np.asarray(K1, np.float64) - np.asarray(K2, np.float64)
    out = []
    for i in range(len(T) - 1):
        if d[i] == 0.0:
            out.append(T[i])
        elif d[i] * d[i + 1] < 0.0:
            out.append(T[i] - d[i] * (T[i + 1] - T[i]) / (d[i + 1] - d[i]))
    if len(d) and d[-1] == 0.0:
        out.append(T[-1])
    return np.asarray(out)


def pq_symmetry(qhist: np.ndarray, min_count: int = 5) -> np.ndarray:
    """Chi-square per degree of freedom of P_J(q) against P_J(-q), per (sample, T): bins b and 200 - b
    (b < 100) with at least `min_count` entries together; about 1 for a symmetric distribution.
    NaN where no pair of bins is populated.  (Counts of one run are correlated in time, so a value
    somewhat above 1 is expected for short runs; a broken symmetry gives values far above.)"""
    h = np.asarray(qhist, np.float64)
    a, b = h[..., :100], h[..., 200:100:-1]
    tot = a + b
    use = tot >= min_count
    chi = np.where(use, (a - b) ** 2 / np.where(use, tot, 1.0), 0.0).sum(-1)
    dof = use.sum(-1)
    return np.where(dof > 0, chi / np.maximum(dof, 1), np.nan)


def doubling_windows(pt, n_windows: int, first: int = 1):
    """Runs windows of first, 2 first, 4 first, ... sweeps (Sec. III.B.1) and returns the observables of
    each window (accumulators reset at every window start)."""
    out = []
    length = int(first)
    for _ in range(int(n_windows)):
        pt.reset_observables()
        pt.sweep(length)
        out.append(pt.observables())
        length *= 2
    return out


def thermalised(windows, temps, key: str = "E", z: float = 3.0) -> np.ndarray:
    """Per temperature: True where the disorder averages of `key` over the last two doubling windows agree
    within z jackknife errors of their difference (paired over samples)."""
    a = thermal_averages(windows[-2], temps)[key]
    b = thermal_averages(windows[-1], temps)[key]
    d, err = jackknife(b - a)
    return np.abs(d) <= z * err + 1e-12


def adaptive_ladder(T_grid, CV_grid, T_min: float, T_max: float, C: float = 0.6, tol: float = 1e-12,
                    max_temps: int = 4096) -> np.ndarray:
    """Temperatures of App. A, Eq. (PT_Ti): T_0 = T_min and T_i = T_{i-1} / (1 - C / sqrt(C_V(T_i))) while
    T_i < T_max, then T_max; so that Delta T ~ T / sqrt(C_V(T)) and neighbouring swaps are accepted at a
    similar rate.  C_V(T) is the measured specific heat (per sample, disorder-averaged) interpolated
    linearly on (T_grid, CV_grid) and held constant outside it.  The recursion is implicit (C_V at the
    new temperature) and is solved by fixed-point iteration from C_V(T_{i-1}).
    ValueError where C >= sqrt(C_V) (no finite step)."""
    Tg = np.asarray(T_grid, np.float64)
    Cg = np.asarray(CV_grid, np.float64)
    order = np.argsort(Tg)
    Tg, Cg = Tg[order], Cg[order]

    def cv(T):
        return float(np.interp(T, Tg, Cg))

    def step(Tp, Cv):
        d = 1.0 - C / np.sqrt(Cv)
        if not (Cv > 0.0) or d <= 0.0:
            raise ValueError("adaptive_ladder: C >= sqrt(C_V) near T = %g (C_V = %g)" % (Tp, Cv))
        return Tp / d

    out = [float(T_min)]
    while len(out) < max_temps:
        Tp = out[-1]
        T = step(Tp, cv(Tp))
        for _ in range(200):
            Tn = step(Tp, cv(T))
            if abs(Tn - T) <= tol * max(1.0, abs(T)):
                T = Tn
                break
            T = Tn
        if T >= T_max:
            break
        out.append(T)
    if out[-1] < T_max:
        out.append(float(T_max))
    return np.asarray(out)


def overlap_distribution(qhist: np.ndarray, width: int = 10) -> np.ndarray:
    """P_J(q) per (sample, T), normalised per sample (Sec. IV.C), on coarse bins of `width` fine bins (the
    201 fine bins centred at -1, -0.99, ..., 1; the last coarse bin also takes the fine bin at q = 1)."""
    h = np.asarray(qhist, np.float64)
    nb = (h.shape[-1] - 1) // width
    coarse = h[..., : nb * width].reshape(h.shape[:-1] + (nb, width)).sum(-1)
    coarse[..., -1] += h[..., nb * width:].sum(-1)
    tot = coarse.sum(-1, keepdims=True)
    return coarse / np.where(tot > 0, tot, 1.0)


def overlap_bin_width(qhist: np.ndarray) -> int:
    """Fine bins per coarse bin for P(q) comparisons: about half the pooled standard deviation of q (so the
    bulk of the distribution spans some eight coarse bins), between 1 and 10 fine bins of 0.01."""
    h = np.asarray(qhist, np.float64).reshape(-1, np.asarray(qhist).shape[-1]).sum(0)
    q = np.arange(h.size) / 100.0 - 1.0
    sd = np.sqrt((h * q * q).sum() / max(h.sum(), 1.0))
    return int(np.clip(round(sd / 0.02), 1, 10))


def paired_difference(obs_a: dict, obs_b: dict, temps, N, pq_min_mass: float = 1e-3) -> dict:
    """Disorder-averaged difference a - b of the observables of two runs on the same disorder samples
    (paired over samples, e.g. FP32 against FP64): per temperature the jackknife mean and error of the
    per-sample differences of E/N, C_V/N (Eq. (21)), <q^2>, <q^4> (Sec. IV.C), Y2, Y4 (Sec. IV.D), the
    disorder average of run b and its own jackknife error (the statistical error of the observable), and
    z = difference / error of the difference; for P_J(q) on coarse bins (overlap_bin_width) the same per
    (T, bin) where run b's mass is at least pq_min_mass."""
    ta, tb = thermal_averages(obs_a, temps), thermal_averages(obs_b, temps)
    scale = {"E": 1.0 / N, "CV": 1.0 / N, "q2": 1.0, "q4": 1.0, "Y2": 1.0, "Y4": 1.0}
    out = {}
    for key, f in scale.items():
        d, err = jackknife(f * (ta[key] - tb[key]))
        ref, ref_err = jackknife(f * tb[key])
        with np.errstate(divide="ignore", invalid="ignore"):
            z = np.where(err > 0, d / err, 0.0)
        out[key] = {"diff": d, "err": err, "ref": ref, "ref_err": ref_err, "z": z}
    w = overlap_bin_width(obs_b["qhist"])
    pa, pb = overlap_distribution(obs_a["qhist"], w), overlap_distribution(obs_b["qhist"], w)
    d, err = jackknife(pa - pb)
    ref, ref_err = jackknife(pb)
    use = (ref >= pq_min_mass) & (err > 0)
    with np.errstate(divide="ignore", invalid="ignore"):
        z = np.where(use, d / np.where(err > 0, err, 1.0), 0.0)
    out["Pq"] = {"diff": d, "err": err, "ref": ref, "ref_err": ref_err, "z": z, "used": use, "bin_width": w}
    return out


def within_statistical_error(diff: dict, k: float = 3.0) -> dict:
    """Per observable of paired_difference: the fraction of temperatures (P(q): of used (T, bin) cells) where
    |a - b| exceeds k times the statistical error of the difference of two independent runs, sqrt(2) times
    the jackknife error of run b's disorder average, and the largest |a - b| in units of that error."""
    out = {}
    for key, v in diff.items():
        d, e = np.abs(np.asarray(v["diff"])), np.sqrt(2.0) * np.asarray(v["ref_err"])
        u = np.asarray(v["used"]) if key == "Pq" else np.ones(d.shape, bool)
        u = u & (e > 0)
        r = np.where(u, d / np.where(e > 0, e, 1.0), 0.0)
        out[key] = {"frac_beyond": float((r[u] > k).mean()) if u.any() else 0.0,
                    "max_in_sigma": float(r[u].max()) if u.any() else 0.0, "cells": int(u.sum())}
    return out


def difference_summary(diff: dict) -> dict:
    """Per observable of paired_difference: the largest |difference| over temperatures (and its error), the
    mean over temperatures of |difference| / |disorder average| (P(q): of |difference| summed over bins), the
    mean of z^2 (about 1 when the two runs sample the same law), the largest |z|, and the largest |difference|
    in units of the statistical error of the observable (within_statistical_error)."""
    out = {}
    stat = within_statistical_error(diff)
    for key, v in diff.items():
        d, e, z = np.asarray(v["diff"]), np.asarray(v["err"]), np.asarray(v["z"])
        if key == "Pq":
            u = v["used"]
            out[key] = {"max_abs_diff": float(np.abs(d[u]).max()) if u.any() else 0.0,
                        "l1_diff_mean_over_T": float(np.abs(d).sum(-1).mean()),
                        "mean_z2": float((z[u] ** 2).mean()) if u.any() else 0.0,
                        "max_abs_z": float(np.abs(z[u]).max()) if u.any() else 0.0, "bins_used": int(u.sum()),
                        "bin_width": float(v["bin_width"]) / 100.0,
                        "max_diff_in_stat_sigma": stat[key]["max_in_sigma"]}
            continue
        i = int(np.argmax(np.abs(d)))
        ref = np.abs(np.asarray(v["ref"]))
        rel = np.abs(d) / np.where(ref > 0, ref, np.inf)
        out[key] = {"max_abs_diff": float(abs(d[i])), "err_at_max": float(e[i]),
                    "mean_rel_diff": float(rel.mean()), "mean_z2": float((z ** 2).mean()),
                    "max_abs_z": float(np.abs(z).max()), "max_diff_in_stat_sigma": stat[key]["max_in_sigma"]}
    return out
