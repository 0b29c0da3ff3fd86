"""Closed-form flows and error metrics used to pin the oracle (TEST INFRASTRUCTURE).

Each function cites the passage (or textbook result) it restates.
"""
from __future__ import annotations

import numpy as np


def couette_impulsive(y, t, h, U, nu, nterms=100):
    """Impulsively started plane Couette flow (Sec. III.A, Eq. solution-couette).

    Lower wall at rest at y = 0, upper wall moving with U at y = h from t = 0;
    series truncated at ``nterms`` terms (the paper uses 100).
    """
    y = np.asarray(y, dtype=np.float64)
    s = y / h
    for n in range(1, nterms + 1):
        s = s + (2.0 / np.pi) * ((-1.0) ** n / n) * np.exp(-n * n * np.pi ** 2 * nu * t / h ** 2) \
            * np.sin(n * np.pi * y / h)
    return U * s


def cylindrical_couette(r, r1, r2, omega1):
    """Steady circular Couette flow, outer cylinder at rest (Sec. III.B):
    u_theta = (r1^2 - beta^2 r^2) omega1 / ((1 - beta^2) r), beta = r1/r2."""
    r = np.asarray(r, dtype=np.float64)
    beta = r1 / r2
    return (r1 ** 2 - beta ** 2 * r ** 2) * omega1 / ((1.0 - beta ** 2) * r)


def couette_torque(rho0, nu, omega1, r1, r2):
    """Torque per unit length on the inner cylinder of steady circular Couette flow
    (textbook: 4 pi mu omega1 r1^2 r2^2 / (r2^2 - r1^2))."""
    return 4.0 * np.pi * rho0 * nu * omega1 * r1 ** 2 * r2 ** 2 / (r2 ** 2 - r1 ** 2)


def poiseuille_transient(s, t, W, g, nu, nterms=2001):
    """Body-force driven channel flow from rest between no-slip walls at s = 0, W
    (textbook sine-series solution of u_t = nu u_ss + g):
    u = g s (W - s)/(2 nu) - sum_{k odd} 4 g W^2/(nu pi^3 k^3) sin(k pi s/W) e^{-k^2 pi^2 nu t/W^2}."""
    s = np.asarray(s, dtype=np.float64)
    u = g * s * (W - s) / (2.0 * nu)
    for k in range(1, nterms + 1, 2):
        u = u - 4.0 * g * W ** 2 / (nu * np.pi ** 3 * k ** 3) * np.sin(k * np.pi * s / W) \
            * np.exp(-k * k * np.pi ** 2 * nu * t / W ** 2)
    return u


def rrse(u, u_th):
    """Relative root squared error (Sec. III.A, Eq. rRMSE)."""
    u = np.asarray(u, dtype=np.float64)
    u_th = np.asarray(u_th, dtype=np.float64)
    return float(np.sqrt(np.sum((u - u_th) ** 2) / np.sum(u_th ** 2)))


def jeffery_rate(theta, gamma_dot, aspect):
    """Rotation rate of a prolate ellipsoid (or elliptic cylinder) in simple shear,
    Jeffery's orbit (Sec. III.C): theta_dot = gamma_dot (r^2 cos^2 theta + sin^2 theta)
    / (r^2 + 1), theta the major axis's angle from the shear gradient direction.
    r is read as the aspect ratio r_a / r_b; the printed "equivalent radius" has the
    dimension of a length, which the rate cannot take."""
    theta = np.asarray(theta, dtype=np.float64)
    r2 = aspect * aspect
    return gamma_dot * (r2 * np.cos(theta) ** 2 + np.sin(theta) ** 2) / (r2 + 1.0)


def jeffery_angle(t, gamma_dot, aspect, theta0=0.0):
    """Closed-form integral of jeffery_rate from theta0 = 0 (major axis along the
    gradient): tan theta = r tan(gamma_dot t r / (r^2 + 1)), continued across the
    half-turns."""
    t = np.asarray(t, dtype=np.float64)
    assert theta0 == 0.0
    phase = gamma_dot * t * aspect / (aspect * aspect + 1.0)
    turns = np.floor(phase / np.pi + 0.5)
    return np.arctan(aspect * np.tan(phase - turns * np.pi)) + turns * np.pi


def torque_squared_fluctuation(t, T, order=30):
    """Torque squared fluctuation (App. D, Eq. TSF30): a least-squares polynomial of
    the given order through the torque series gives a smooth baseline T_ip; the
    squared deviation (T - T_ip)^2 is fitted again by a polynomial of the same order.
    Returns (T_ip, TSF, TSF_ip). The fits use the Chebyshev basis on the span of t,
    which spans the same polynomials as the monomials and stays well conditioned."""
    t = np.asarray(t, dtype=np.float64)
    T = np.asarray(T, dtype=np.float64)
    Cheb = np.polynomial.Chebyshev
    T_ip = Cheb.fit(t, T, order)(t)
    tsf = (T - T_ip) ** 2
    tsf_ip = Cheb.fit(t, tsf, order)(t)
    return T_ip, tsf, tsf_ip
