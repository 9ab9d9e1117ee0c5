"""Closed-form potentials of the paper's test problems (Sec. 4), FP64 numpy.

TEST INFRASTRUCTURE (part of the oracle).  Newton's constant is 1, so a body
of density rho has source S = 4 pi rho and these functions return the Phi
that solves Eq. 1 with Phi -> 0 at infinity.

* ``sphere``   -- uniform sphere, Eq. 10 (Sec. 4.1).
* ``spheroid`` -- uniform oblate spheroid about the z axis, inside Eq. 14
  with the coefficients of Eqs. 15-16, outside Eq. 17 with h of Eq. 18 and
  lambda the positive root of Eq. 19 (Sec. 4.2).  Shifting the centre is the
  substitution the paper uses for the binary spheroid (Sec. 4.3).
* ``gaussian`` -- a smooth body, rho = A exp(-r^2 / (2 sigma^2)), whose
  potential is -M erf(r / (sqrt(2) sigma)) / r with M = A (2 pi sigma^2)^1.5.
  Not in the paper; it isolates the second-order error of the discrete
  Green's function from the first-order error of sampling a sharp surface.
"""
import numpy as np
from scipy.special import erf


def sphere(x, y, z, center, R, rho):
    """Eq. 10: -(2/3) pi rho (3R^2 - r^2) inside, -(4/3) pi rho R^3 / r outside."""
    r = np.sqrt((x - center[0]) ** 2 + (y - center[1]) ** 2 + (z - center[2]) ** 2)
    inside = -(2.0 / 3.0) * np.pi * rho * (3.0 * R * R - r * r)
    with np.errstate(divide="ignore", invalid="ignore"):
        outside = -(4.0 / 3.0) * np.pi * rho * R ** 3 / r
    return np.where(r <= R, inside, outside)


def spheroid_coefficients(e):
    """Eqs. 15-16: A and B of the interior potential for eccentricity e."""
    s = np.sqrt(1.0 - e * e)
    ae = np.arcsin(e)
    A = s / e ** 3 * ae - (1.0 - e * e) / (e * e)
    B = 2.0 / (e * e) - 2.0 * s / e ** 3 * ae
    return A, B


def spheroid(x, y, z, center, a, b, rho):
    """Uniform oblate spheroid (a >= b, symmetry axis z) of Sec. 4.2.

    For e below 1e-3 the spheroid is a sphere to rounding and the sphere
    form is used (Eqs. 15-17 lose all digits as e -> 0)."""
    if b > a:
        raise ValueError("the paper's closed form is for oblate spheroids (a >= b)")
    e = np.sqrt(1.0 - (b / a) ** 2)
    if e < 1e-3:
        return sphere(x, y, z, center, a, rho)
    X = x - center[0]
    Y = y - center[1]
    Z = z - center[2]
    w2 = X * X + Y * Y
    z2 = Z * Z
    A, B = spheroid_coefficients(e)
    inside = -np.pi * rho * (A * (2.0 * a * a - w2) + B * (b * b - z2))
    # Eq. 19 as a quadratic in lambda:
    #   lambda^2 + (a^2 + b^2 - w2 - z2) lambda + a^2 b^2 - w2 b^2 - z2 a^2 = 0
    p = a * a + b * b - w2 - z2
    q = a * a * b * b - w2 * b * b - z2 * a * a
    disc = np.sqrt(np.maximum(p * p - 4.0 * q, 0.0))
    lam = 0.5 * (-p + disc)
    lam = np.maximum(lam, 0.0)
    hh = a * e / np.sqrt(b * b + lam)  # Eq. 18
    at = np.arctan(hh)
    outside = -2.0 * np.pi * rho * (a * b / e) * (
        at - (w2 * (at - hh / (1.0 + hh * hh)) + 2.0 * z2 * (hh - at)) / (2.0 * a * a * e * e))
    is_in = w2 / (a * a) + z2 / (b * b) <= 1.0
    return np.where(is_in, inside, outside)


def gaussian(x, y, z, center, sigma, amp):
    """Potential of rho = amp exp(-r^2/(2 sigma^2)): -M erf(r/(sqrt2 sigma))/r."""
    r = np.sqrt((x - center[0]) ** 2 + (y - center[1]) ** 2 + (z - center[2]) ** 2)
    M = amp * (2.0 * np.pi * sigma * sigma) ** 1.5
    with np.errstate(divide="ignore", invalid="ignore"):
        out = -M * erf(r / (np.sqrt(2.0) * sigma)) / r
    at0 = -M * np.sqrt(2.0 / np.pi) / sigma
    return np.where(r > 0, out, at0)


def bodies_potential(bodies, x, y, z):
    """Sum of the closed forms of a list of bodies as produced by the source
    generators (dicts with kind 'sphere', 'spheroid' or 'gaussian')."""
    phi = np.zeros(np.broadcast(x, y, z).shape, dtype=np.float64)
    for bd in bodies:
        k = bd["kind"]
        if k == "sphere":
            phi += sphere(x, y, z, bd["center"], bd["radius"], bd["rho"])
        elif k == "spheroid":
            phi += spheroid(x, y, z, bd["center"], bd["a"], bd["b"], bd["rho"])
        elif k == "gaussian":
            phi += gaussian(x, y, z, bd["center"], bd["sigma"], bd["amp"])
        else:
            raise ValueError(k)
    return phi
