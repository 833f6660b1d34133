"""Closed forms the paper compares its simulations against (test infrastructure).

Each function states the equation it evaluates.  These are the physics pins of
the oracle: the coupled LB runs in tests/ are compared with them.
"""
from __future__ import annotations

import math

import numpy as np

HASIMOTO_SC = 2.8373  # leading periodic-array constant (Hasimoto 1959), cited in Sec. III.A


def eccentricity(a: float, b: float) -> float:
    """epsilon = sqrt(1 - b^2/a^2) for a prolate spheroid a >= b = c (Sec. III.A)."""
    return math.sqrt(max(0.0, 1.0 - (b * b) / (a * a)))


def oberbeck_coefficients(eps: float):
    """C_par and C_perp of Eq. settlingvel.

    The bracket cancels for small eps; below 1e-3 the expansion of the
    logarithm gives C_par = 1/(1 + 2 eps^2/5) and C_perp = 1/(1 + 3 eps^2/10) to
    O(eps^4), which tend to 1 (sphere).
    """
    if eps < 1e-3:
        return 1.0 / (1.0 + 0.4 * eps * eps), 1.0 / (1.0 + 0.3 * eps * eps)
    lg = math.log((1.0 + eps) / (1.0 - eps))
    cpar = (8.0 / 3.0) * eps ** 3 / (-2.0 * eps + (1.0 + eps * eps) * lg)
    cperp = (16.0 / 3.0) * eps ** 3 / (2.0 * eps + (3.0 * eps * eps - 1.0) * lg)
    return cpar, cperp


def settling_velocity_ratio(a: float, b: float):
    """(U_par, U_perp) / U_sphere(radius b) under the same force (Eq. settlingvel).

    U = F / (6 pi mu a C) and U_sphere(b) = F / (6 pi mu b)."""
    cpar, cperp = oberbeck_coefficients(eccentricity(a, b))
    return b / (a * cpar), b / (a * cperp)


def drift_angle(alpha: float, a: float, b: float) -> float:
    """delta from Eq. drift, tan(alpha - delta) = (C_par / C_perp) tan(alpha), radians."""
    cpar, cperp = oberbeck_coefficients(eccentricity(a, b))
    return alpha - math.atan((cpar / cperp) * math.tan(alpha))


def squirmer_speed(B1: float, a: float, b: float) -> float:
    """Eq. squirmervel: U_s = B1 eps^-1 (eps^-1 - (eps^-2 - 1) arccoth(eps^-1)).

    Sphere limit (eps -> 0): 2 B1 / 3 (Sec. III.D)."""
    eps = eccentricity(a, b)
    if eps < 1e-4:
        return 2.0 * B1 / 3.0
    ie = 1.0 / eps
    acoth = 0.5 * math.log((ie + 1.0) / (ie - 1.0))
    return B1 * ie * (ie - (ie * ie - 1.0) * acoth)


def stokes_velocity(F: float, mu: float, a: float) -> float:
    return F / (6.0 * math.pi * mu * a)


def hasimoto_velocity(F: float, mu: float, a: float, L: float) -> float:
    """Sphere of radius a in a periodic cube of side L, leading correction."""
    return F / (6.0 * math.pi * mu * a) * (1.0 - HASIMOTO_SC * a / L)


def hasimoto_series(a: float, L: float) -> float:
    """U_L / U_Stokes of a simple cubic array of spheres of radius a, cell side L,
    moving through the fluid at zero mean volume flux (Hasimoto 1959, cited in
    Sec. III.A, with the next terms of Sangani and Acrivos 1982):
    1 - 1.7601 phi^(1/3) + phi - 1.5593 phi^2, phi = (4 pi / 3)(a / L)^3.
    The first term is the shape-independent Stokeslet image sum,
    1.7601 phi^(1/3) = HASIMOTO_SC a / L."""
    phi = 4.0 * math.pi / 3.0 * (a / L) ** 3
    return 1.0 - 1.7601 * phi ** (1.0 / 3.0) + phi - 1.5593 * phi * phi


def jeffery_rhs(e: np.ndarray, G: np.ndarray, beta: float) -> np.ndarray:
    """Eq. jeffery: de/dt = Lambda e + beta (E e - e (e.E e)), G = grad u (G_ij = du_i/dx_j)."""
    E = 0.5 * (G + G.T)
    Lam = 0.5 * (G - G.T)
    Ee = E @ e
    return Lam @ e + beta * (Ee - e * (e @ Ee))


def jeffery_orbit(e0, G, beta, t_end: float, dt: float):
    """RK4 integration of Eq. jeffery; returns times and unit vectors."""
    n = int(round(t_end / dt))
    e = np.asarray(e0, dtype=np.float64).copy()
    out = [e.copy()]
    for _ in range(n):
        k1 = jeffery_rhs(e, G, beta)
        k2 = jeffery_rhs(e + 0.5 * dt * k1, G, beta)
        k3 = jeffery_rhs(e + 0.5 * dt * k2, G, beta)
        k4 = jeffery_rhs(e + dt * k3, G, beta)
        e = e + dt / 6.0 * (k1 + 2 * k2 + 2 * k3 + k4)
        e /= np.linalg.norm(e)
        out.append(e.copy())
    return np.arange(n + 1) * dt, np.array(out)


def jeffery_orbit_constant(p, r: float):
    """Orbit constant of Eq. jeffery in simple shear u_x = gamma y (flow x,
    gradient y, vorticity z): C = tan(theta) (r^2 cos^2 phi + sin^2 phi)^(1/2) / r
    with theta the angle of the axis p from the vorticity axis and phi its
    azimuth from the gradient axis, i.e. C = (r^2 p_y^2 + p_x^2)^(1/2) / (r |p_z|)
    (Jeffery 1922, cited in Sec. III.C)."""
    p = np.asarray(p, dtype=np.float64)
    return np.sqrt(r * r * p[..., 1] ** 2 + p[..., 0] ** 2) / (r * np.abs(p[..., 2]))


def jeffery_aspect_from_period(T: float, gamma_dot: float) -> float:
    """The aspect ratio r >= 1 with T = 2 pi (r + 1/r) / gamma_dot."""
    s = T * gamma_dot / (2.0 * math.pi)           # r + 1/r
    return 0.5 * (s + math.sqrt(max(0.0, s * s - 4.0)))


def jeffery_period(r: float, gamma_dot: float) -> float:
    """T = 2 pi (r + 1/r) / gamma_dot (Jeffery 1922, cited in Sec. III.C)."""
    return 2.0 * math.pi * (r + 1.0 / r) / gamma_dot
