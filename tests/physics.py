"""Textbook results used to pin the oracle (standard mechanics, not the paper).

Nothing here evaluates the DEM step; these are closed forms of special cases
(Hertz impact, uniformly decelerated rolling/spinning, discrete free fall)
and small state-only diagnostics (momenta, energies) computed from arrays.
"""
from __future__ import annotations

import math

import numpy as np

# integral_0^1 (1 - s^(5/2))^(-1/2) ds = (2/5) B(2/5, 1/2)
HERTZ_TIME_INTEGRAL = 0.4 * math.gamma(0.4) * math.gamma(0.5) / math.gamma(0.9)


def hertz_impact(m_eff, r_eff, e_eff, v):
    """Peak overlap and duration of an elastic Hertz impact.

    Force law F = (4/3) E* sqrt(R*) delta^(3/2) (Hertz); energy balance gives
    delta_max^(5/2) = 15 m* v^2 / (16 E* sqrt(R*)) and the contact lasts
    t_c = 2 (delta_max / v) * integral_0^1 (1 - s^(5/2))^(-1/2) ds.
    """
    dmax = (15.0 * m_eff * v * v / (16.0 * e_eff * math.sqrt(r_eff))) ** 0.4
    return dmax, 2.0 * dmax / v * HERTZ_TIME_INTEGRAL


def sphere_mass(rho, R):
    return 4.0 / 3.0 * math.pi * rho * R ** 3


def linear_momentum(rho, R, v):
    m = 4.0 / 3.0 * math.pi * rho * np.asarray(R) ** 3
    return (m[:, None] * v).sum(axis=0)


def angular_momentum(rho, R, x, v, w):
    R = np.asarray(R)
    m = 4.0 / 3.0 * math.pi * rho * R ** 3
    I = 0.4 * m * R ** 2
    return (m[:, None] * np.cross(x, v) + I[:, None] * w).sum(axis=0)


def kinetic_energy(rho, R, v, w):
    R = np.asarray(R)
    m = 4.0 / 3.0 * math.pi * rho * R ** 3
    I = 0.4 * m * R ** 2
    return 0.5 * (m * (v * v).sum(1)).sum() + 0.5 * (I * (w * w).sum(1)).sum()


def quat_from_axis_angle(axis, angle):
    axis = np.asarray(axis, dtype=np.float64)
    axis = axis / np.linalg.norm(axis)
    return np.concatenate([[math.cos(angle / 2)], math.sin(angle / 2) * axis])


def quat_mul(a, b):
    a0, av = a[0], np.asarray(a[1:])
    b0, bv = b[0], np.asarray(b[1:])
    return np.concatenate([[a0 * b0 - av @ bv], a0 * bv + b0 * av + np.cross(av, bv)])
