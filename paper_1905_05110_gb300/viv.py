"""Response of a spring-mounted cylinder from its history records (Sec. 3.3).

Post-processing of the records a run returns, not a step of the method:
with the non-dimensional numbers of Sec. 3.3,
    m* = m / (rho D^2 / 2),  k* = k / (rho U0^2 / 2),  y* = y_G / D,
    t* = t U0 / D,
the response of a run is its largest displacement from rest,
A* = max(y*) - y0*, and its angular frequency omega* (per unit t*), taken
from the displacement; the effective stiffness of Shiels et al. is
k*_eff = k* - m* omega*^2 (it is zero when the body oscillates at its
natural frequency in vacuum, sqrt(k / m)).
"""
from __future__ import annotations

import math

import numpy as np


def _crossings(s: np.ndarray, level: float):
    """Times (fractional sample indices) where s crosses `level`, either way,
    by linear interpolation between the samples around each crossing, and
    whether each crossing is upwards."""
    d = s - level
    up = (d[:-1] < 0.0) & (d[1:] >= 0.0)
    k = np.nonzero(up | ((d[:-1] >= 0.0) & (d[1:] < 0.0)))[0]
    return k + d[k] / (d[k] - d[k + 1]), up[k]


def mean_period(s: np.ndarray) -> tuple:
    """Mean period (in samples) of an oscillating s from the spacing of the
    crossings of its centre line (two per period), and the number of half
    periods they span (nan, 0 with fewer than three crossings, i.e. less
    than one period).  The centre line starts as the mean of s and is then
    taken as the mean over the whole periods between its first and last
    upward crossings, which removes the bias of a window that holds a
    fraction of a period."""
    s = np.asarray(s, dtype=np.float64)
    level = s.mean()
    for _ in range(3):
        t, up = _crossings(s, level)
        tu = t[up]
        if tu.size < 2:
            break
        level = s[int(math.ceil(tu[0])):int(math.floor(tu[-1])) + 1].mean()
    t, _ = _crossings(s, level)
    if t.size < 3:
        return math.nan, 0
    return float(2.0 * (t[-1] - t[0]) / (t.size - 1)), int(t.size - 1)


def viv_response(y: np.ndarray, y0: float, diameter: float, u0: float, mass: float, stiffness: float,
                 rho: float = 1.0) -> dict:
    """A*, omega*, k*, m* and k*_eff of a spring-mounted body from its
    transverse positions y (one per time step, lattice units) over the
    analysis window; y0 is the rest position.  half_periods: how many half
    periods of the displacement the frequency was measured over."""
    y = np.asarray(y, dtype=np.float64)
    m_star = mass / (0.5 * rho * diameter ** 2)
    k_star = stiffness / (0.5 * rho * u0 ** 2)
    period, n = mean_period(y)
    omega_star = 2.0 * math.pi / period * diameter / u0 if n else math.nan
    return {"a_star": float((y.max() - y0) / diameter), "omega_star": omega_star, "m_star": m_star,
            "k_star": k_star, "k_eff_star": k_star - m_star * omega_star ** 2, "half_periods": n}
