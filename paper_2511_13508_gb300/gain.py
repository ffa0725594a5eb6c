"""Effective independent samples per second at the coldest temperature, plain PT against PT with the
learned global move (host orchestration of the library's calls; every step runs in its kernels).

ESS/s = (series per ensemble) x sweeps/s / (2 tau_int(E) x sweeps between measurements), with tau_int from
Sokal's automatic window over the running energy of the coldest temperature of every (sample, replica)
ladder.  Sweep throughput is timed without host synchronisation; the energy series is read in between.
"""
from __future__ import annotations

import time

import numpy as np

from . import stats


def _rate(pt, sweeps):
    pt.sync()
    t0 = time.perf_counter()
    pt.sweep(sweeps)
    pt.sync()
    return sweeps / (time.perf_counter() - t0)


def _series(pt, n, every):
    out = np.zeros((n, pt.S, pt.R))
    for i in range(n):
        pt.sweep(every)
        out[i] = pt.running_energies().reshape(pt.S, pt.R, pt.nT)[:, :, 0]
    return out


def _ess_rate(pt, x, rate, every):
    taus = np.array([stats.tau_int(x[:, s]) for s in range(pt.S)])  # per sample, replicas pooled
    ess_per_sweep = pt.S * pt.R / (2.0 * taus.mean() * every)
    return taus, ess_per_sweep * rate


def measure(pt, *, n_cold, global_every, train_configs, train_steps, lr=1e-3, batch=512, burn_in=4096,
            series=4096, every=8, rate_sweeps=4096, blocks=(0, 7), seed=1):
    """Runs plain PT, then trains the proposal on the same ensemble and runs PT with global moves."""
    pt.sweep(burn_in)
    rate0 = _rate(pt, rate_sweeps)
    x0 = _series(pt, series, every)
    tau0, ess0 = _ess_rate(pt, x0, rate0, every)
    t0 = time.perf_counter()
    pt.learn_init(n_cold=n_cold, batch=batch, data_per_sample=train_configs, seed=seed)
    rounds = train_configs // (n_cold * pt.R)
    pt.collect(every, rounds)
    losses = pt.train(train_steps, lr=lr)
    t_train = time.perf_counter() - t0
    pt.set_global_blocks(*blocks)
    pt.set_global_every(global_every)
    pt.sweep(max(burn_in // 4, global_every))
    rate1 = _rate(pt, rate_sweeps)
    pt.reset_observables()
    x1 = _series(pt, series, every)
    o = pt.observables()
    acc = o["gm_acc"].sum(0)[:n_cold] / np.maximum(o["gm_att"].sum(0)[:n_cold], 1)
    tau1, ess1 = _ess_rate(pt, x1, rate1, every)
    return {
        "ess_per_s_plain": ess0, "ess_per_s_learned": ess1, "gain": ess1 / ess0,
        "tau_int_sweeps_plain": float(tau0.mean() * every), "tau_int_sweeps_learned": float(tau1.mean() * every),
        "sweeps_per_s_plain": rate0, "sweeps_per_s_learned": rate1,
        "acceptance_coldest": [float(v) for v in acc], "train_seconds": t_train, "train_steps": train_steps,
        "train_configs_per_sample": rounds * n_cold * pt.R,
        "nll_first": float(np.mean(losses[:20])), "nll_last": float(np.mean(losses[-100:])),
        "mean_E_coldest_plain": float(x0.mean()), "mean_E_coldest_learned": float(x1.mean()),
        "blocks": list(blocks), "global_every": global_every, "series": series, "every": every,
    }
