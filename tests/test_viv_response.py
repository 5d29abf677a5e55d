"""Effective stiffness of a spring-mounted body (Sec. 3.3) from its
history: exact on signals whose answer is known."""
import math

import numpy as np
import pytest

from paper_1905_05110_gb300.viv import mean_period, viv_response


@pytest.mark.parametrize("period", [97.3, 400.0, 5123.7, 17_000.0])
def test_mean_period_of_a_sampled_sinusoid(period):
    # down to a little more than two periods in the window
    t = np.arange(40_000, dtype=np.float64)
    p, n = mean_period(3.0 + 0.7 * np.sin(2 * math.pi * t / period + 0.4))
    assert abs(n - 2 * (t.size - 1) / period) <= 2
    assert abs(p - period) < 1e-3 * period


def test_response_of_a_free_oscillation_at_the_natural_frequency():
    # a body oscillating at sqrt(k / m): k*_eff = 0 for any mass and U0;
    # amplitude 0.3 D about y0
    d, u0, m = 32.0, 0.04, 5000.0
    omega = 2 * math.pi / 3000.0
    k = m * omega ** 2
    t = np.arange(30_000, dtype=np.float64)
    y0 = 256.0
    y = y0 + 0.3 * d * np.sin(omega * t)
    r = viv_response(y, y0, d, u0, m, k)
    assert abs(r["a_star"] - 0.3) < 1e-6
    assert abs(r["omega_star"] - omega * d / u0) < 1e-4 * omega * d / u0
    assert abs(r["k_eff_star"]) < 1e-3 * r["k_star"]
    assert r["m_star"] == m / (0.5 * d * d) and r["k_star"] == k / (0.5 * u0 * u0)


def test_response_below_and_above_the_natural_frequency():
    # oscillating slower than sqrt(k/m) leaves a positive effective
    # stiffness, faster a negative one, in the units of Sec. 3.3:
    # k*_eff = (k - m w^2) / (rho U0^2 / 2)
    d, u0, m, k = 40.0, 0.05, 1200.0, 0.03
    t = np.arange(50_000, dtype=np.float64)
    for w in (0.5 * math.sqrt(k / m), 2.0 * math.sqrt(k / m)):
        r = viv_response(100.0 + 5.0 * np.sin(w * t), 100.0, d, u0, m, k)
        expect = (k - m * w * w) / (0.5 * u0 * u0)
        assert abs(r["k_eff_star"] - expect) < 2e-3 * abs(expect)


def test_no_oscillation_gives_no_frequency():
    r = viv_response(np.linspace(0.0, 1.0, 1000), 0.0, 10.0, 0.04, 1.0, 1.0)
    assert r["half_periods"] == 0 and math.isnan(r["omega_star"]) and math.isnan(r["k_eff_star"])
