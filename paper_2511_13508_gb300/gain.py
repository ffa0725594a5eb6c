"""Effective independent samples per second at the coldest temperature, plain PT against PT with the
learned global move (host orchestration of the library's calls; every step runs in its kernels).

ESS/s = (series per ensemble) x sweeps/s / (2 tau_int x sweeps between measurements), with tau_int from
Sokal's automatic window, for two observables at the coldest temperature: the running energy of every
(sample, replica) ladder, and the squared overlap q^2 of the first two replicas of every sample (Sec. IV.C;
the slow modes of a glassy phase live in q).  Sweep throughput is timed without host synchronisation; the
series are read in between.  The gain's error is a jackknife over disorder samples; the break-even acceptance
is the global-move acceptance per round at which independent proposals every `global_every` sweeps would
decorrelate as fast as plain PT does at the learned run's throughput (gain 1).
"""
from __future__ import annotations

import time

import numpy as np

from . import analysis, stats


def _rate(pt, sweeps):
    pt.sync()
    t0 = time.perf_counter()
    pt.sweep(sweeps)
    pt.sync()
    return sweeps / (time.perf_counter() - t0)


def _series(pt, n, every):
    """Running energies [n, S, R] and q^2 of replicas 0 and 1 [n, S] at the coldest temperature."""
    E = np.zeros((n, pt.S, pt.R))
    q2 = np.zeros((n, pt.S))
    N = int(pt.Ns[0])
    for i in range(n):
        pt.sweep(every)
        a, Ec = pt.state()
        E[i] = Ec.reshape(pt.S, pt.R, pt.nT)[:, :, 0]
        if pt.R >= 2:
            a = a.reshape(pt.S, pt.R, pt.nT, N)
            q2[i] = ((np.conj(a[:, 0, 0]) * a[:, 1, 0]).real.sum(-1) / N) ** 2
    return E, q2


def measure(pt, *, n_cold, global_every, train_configs, train_steps, lr=1e-3, batch=512, burn_in=4096,
            series=4096, every=8, rate_sweeps=4096, blocks=(0, 7), seed=1):
    """Equilibrates the ensemble with plain PT, trains the proposal on configurations PT collects, then measures,
    on the same equilibrated ensemble and with identical series lengths, plain PT (global move off), PT with the
    global move, and plain PT again (A-B-A): the two plain segments bracket the learned one, so a slow drift of
    the ensemble shows as a difference between them (reported) instead of as a gain."""
    pt.sweep(burn_in)
    t0 = time.perf_counter()
    pt.learn_init(n_cold=n_cold, batch=batch, data_per_sample=train_configs, seed=seed)
    rounds = train_configs // (n_cold * pt.R)
    pt.collect(every, rounds)
    losses = pt.train(train_steps, lr=lr)
    t_train = time.perf_counter() - t0
    pt.set_global_blocks(*blocks)

    def plain_segment():
        pt.set_global_every(0)
        r = _rate(pt, rate_sweeps)
        x, q = _series(pt, series, every)
        return r, x, q

    rate0a, x0a, q0a = plain_segment()
    pt.set_global_every(global_every)
    pt.sweep(max(burn_in // 4, global_every))
    rate1 = _rate(pt, rate_sweeps)
    pt.reset_observables()
    x1, q1 = _series(pt, series, every)
    o = pt.observables()
    acc = o["gm_acc"].sum(0)[:n_cold] / np.maximum(o["gm_att"].sum(0)[:n_cold], 1)
    rate0b, x0b, q0b = plain_segment()
    rate0 = 0.5 * (rate0a + rate0b)
    tau0 = 0.5 * (np.array([stats.tau_int(x0a[:, s]) for s in range(pt.S)]) +
                  np.array([stats.tau_int(x0b[:, s]) for s in range(pt.S)]))
    tq0 = 0.5 * (np.array([stats.tau_int(q0a[:, s]) for s in range(pt.S)]) +
                 np.array([stats.tau_int(q0b[:, s]) for s in range(pt.S)]))
    tau1 = np.array([stats.tau_int(x1[:, s]) for s in range(pt.S)])
    tq1 = np.array([stats.tau_int(q1[:, s]) for s in range(pt.S)])
    ess0 = pt.S * pt.R / (2.0 * tau0.mean() * every) * rate0
    ess1 = pt.S * pt.R / (2.0 * tau1.mean() * every) * rate1
    essq0 = pt.S / (2.0 * tq0.mean() * every) * rate0
    essq1 = pt.S / (2.0 * tq1.mean() * every) * rate1
    # the gain is a ratio of mean autocorrelation times over the same disorder samples: jackknife over samples
    ratio = lambda a, b: a.mean(0) / b.mean(0)
    _, gE_err = analysis.jackknife((tau0, tau1), ratio)
    _, gq_err = analysis.jackknife((tq0, tq1), ratio)
    # drift between the two plain segments: difference of the sample means of E against its jackknife error
    dE, dE_err = analysis.jackknife(x0b.mean((0, 2)) - x0a.mean((0, 2)))
    return {
        "ess_per_s_plain": ess0, "ess_per_s_learned": ess1, "gain": ess1 / ess0,
        "gain_err": float(gE_err) * rate1 / rate0,
        "break_even_acceptance": float(global_every / (tau0.mean() * every * rate1 / rate0)),
        "acceptance_mean": float(np.mean(acc)),
        "tau_int_sweeps_plain": float(tau0.mean() * every), "tau_int_sweeps_learned": float(tau1.mean() * every),
        "tau_int_sweeps_plain_before_after": [float(np.mean([stats.tau_int(x0a[:, s]) for s in range(pt.S)]) * every),
                                              float(np.mean([stats.tau_int(x0b[:, s]) for s in range(pt.S)]) * every)],
        "plain_drift_E": {"after_minus_before": float(dE), "err": float(dE_err),
                          "significant": bool(abs(dE) > 3.0 * dE_err)},
        "q2": {"ess_per_s_plain": essq0, "ess_per_s_learned": essq1, "gain": essq1 / essq0,
               "gain_err": float(gq_err) * rate1 / rate0,
               "tau_int_sweeps_plain": float(tq0.mean() * every), "tau_int_sweeps_learned": float(tq1.mean() * every),
               "mean_plain": float(0.5 * (q0a.mean() + q0b.mean())), "mean_learned": float(q1.mean())},
        "sweeps_per_s_plain": rate0, "sweeps_per_s_learned": rate1,
        "acceptance_coldest": [float(v) for v in acc], "train_seconds": t_train, "train_steps": train_steps,
        "train_configs_per_sample": rounds * n_cold * pt.R,
        "nll_first": float(np.mean(losses[:20])), "nll_last": float(np.mean(losses[-100:])),
        "mean_E_coldest_plain": float(0.5 * (x0a.mean() + x0b.mean())), "mean_E_coldest_learned": float(x1.mean()),
        "blocks": list(blocks), "global_every": global_every, "series": series, "every": every,
    }
