"""Sokal's automatic-window estimator against the closed form of an AR(1) process:
x_t = phi x_{t-1} + e_t has rho(t) = phi^t and tau_int = (1 + phi) / (2 (1 - phi))."""
import numpy as np
import pytest

from paper_2511_13508_gb300 import stats


@pytest.mark.parametrize("phi", [0.0, 0.5, 0.9, 0.97])
def test_tau_int_of_ar1(phi):
    rng = np.random.default_rng(int(phi * 100))
    T, M = 20000, 16
    e = rng.standard_normal((T, M))
    x = np.zeros((T, M))
    x[0] = e[0] / np.sqrt(1 - phi * phi)
    for t in range(1, T):
        x[t] = phi * x[t - 1] + e[t]
    exact = (1 + phi) / (2 * (1 - phi))
    est = stats.tau_int(x)
    assert abs(est - exact) < 0.06 * exact + 0.02, (est, exact)
    assert abs(stats.ess(x) - T * M / (2 * exact)) < 0.08 * T * M / (2 * exact)


def test_autocorrelation_of_ar1_matches_phi_powers():
    rng = np.random.default_rng(3)
    phi, T = 0.8, 200000
    e = rng.standard_normal(T)
    x = np.zeros(T)
    for t in range(1, T):
        x[t] = phi * x[t - 1] + e[t]
    rho = stats.autocorrelation(x)
    assert np.allclose(rho[:6], phi ** np.arange(6), atol=0.02)
