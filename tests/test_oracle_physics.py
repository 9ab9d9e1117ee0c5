"""Pins for the closed-form potentials and for the oracle's convergence to
them under refinement (Sec. 4) -- CPU only.

The closed forms are checked as solutions of Eq. 1 (finite-difference
Laplacian equals 4 pi rho inside and 0 outside), for continuity across the
surface, for the far field -M/r, and for the sphere limit of the spheroid.
The oracle is then checked to converge to them: second order on a smooth
Gaussian body, better than first order on the sharp-surfaced sphere and
spheroid (the paper's Sec. 4.1/4.2 statements).
"""
import math

import numpy as np
import pytest

from oracle import analytic
from paper_1106_0557_gb300 import sources


def laplacian(f, p, eps=1e-3):
    x, y, z = p
    c = f(x, y, z)
    acc = 0.0
    for d in np.eye(3):
        acc += f(x + eps * d[0], y + eps * d[1], z + eps * d[2]) + f(x - eps * d[0], y - eps * d[1], z - eps * d[2]) - 2 * c
    return acc / eps ** 2


def test_sphere_closed_form():
    R, rho, c = 0.6, 1.3, (0.1, -0.2, 0.3)
    f = lambda x, y, z: float(analytic.sphere(np.array(x), np.array(y), np.array(z), c, R, rho))
    assert laplacian(f, (0.2, -0.1, 0.4)) == pytest.approx(4 * math.pi * rho, rel=1e-5)
    assert abs(laplacian(f, (1.2, 0.5, 0.1))) < 1e-4
    # continuity at the surface and the far field -M/r
    for s in (R * (1 - 1e-12), R * (1 + 1e-12)):
        assert f(c[0] + s, c[1], c[2]) == pytest.approx(-(4 / 3) * math.pi * rho * R ** 2, rel=1e-9)
    Mass = (4 / 3) * math.pi * R ** 3 * rho
    assert f(c[0], c[1] + 50.0, c[2]) == pytest.approx(-Mass / 50.0, rel=1e-12)


def test_spheroid_coefficients():
    for e in (0.1, 0.5, 0.9, 0.99):
        A, B = analytic.spheroid_coefficients(e)
        assert 2 * A + B == pytest.approx(2.0, rel=1e-12)
    A, B = analytic.spheroid_coefficients(1e-2)
    assert A == pytest.approx(2 / 3, abs=1e-4) and B == pytest.approx(2 / 3, abs=1e-4)


@pytest.mark.parametrize("e", [0.28, 0.6, 0.9])
def test_spheroid_closed_form(e):
    a, rho, c = 0.5, 1.0, (0.05, -0.1, 0.2)
    b = a * math.sqrt(1 - e * e)
    f = lambda x, y, z: float(analytic.spheroid(np.array(x), np.array(y), np.array(z), c, a, b, rho))
    # Poisson's equation inside and Laplace's outside
    assert laplacian(f, (c[0] + 0.1, c[1] - 0.1, c[2] + 0.3 * b)) == pytest.approx(4 * math.pi * rho, rel=1e-4)
    assert abs(laplacian(f, (c[0] + 0.7, c[1] + 0.2, c[2] + 0.4))) < 1e-3
    # continuity across the surface, on the equator and at the pole
    for p in [(c[0] + a, c[1], c[2]), (c[0], c[1], c[2] + b), (c[0] + a * 0.6, c[1], c[2] + b * 0.8)]:
        d = np.array(p) - np.array(c)
        inner = f(*(np.array(c) + d * (1 - 1e-9)))
        outer = f(*(np.array(c) + d * (1 + 1e-9)))
        assert inner == pytest.approx(outer, rel=1e-7)
    # far field -M/r with M = 4/3 pi a^2 b rho
    Mass = (4 / 3) * math.pi * a * a * b * rho
    r = 200.0
    assert f(c[0] + r / math.sqrt(3), c[1] + r / math.sqrt(3), c[2] + r / math.sqrt(3)) == pytest.approx(-Mass / r, rel=1e-5)


def test_spheroid_sphere_limit():
    a = 0.4
    pts = [np.array(v) for v in ((0.1, 0.0, 0.0), (0.0, 0.2, 0.3), (0.7, 0.1, -0.3))]
    for p in pts:
        s = analytic.sphere(*p, (0, 0, 0), a, 1.0)
        t = analytic.spheroid(*p, (0, 0, 0), a, a * math.sqrt(1 - 0.02 ** 2), 1.0)
        assert float(t) == pytest.approx(float(s), rel=1e-3)


def test_gaussian_closed_form():
    sig, amp, c = 0.2, 1.7, (0.0, 0.1, -0.1)
    f = lambda x, y, z: float(analytic.gaussian(np.array(x), np.array(y), np.array(z), c, sig, amp))
    for p in [(0.05, 0.12, -0.05), (0.3, -0.1, 0.2)]:
        r2 = sum((pi - ci) ** 2 for pi, ci in zip(p, c))
        rho = amp * math.exp(-r2 / (2 * sig * sig))
        assert laplacian(f, p, eps=1e-3) == pytest.approx(4 * math.pi * rho, rel=1e-4)
    Mass = amp * (2 * math.pi * sig * sig) ** 1.5
    assert f(c[0] + 30.0, c[1], c[2]) == pytest.approx(-Mass / 30.0, rel=1e-12)


def order_fit(ns, errs):
    slope = np.polyfit(np.log(ns), np.log(errs), 1)[0]
    return -slope


def _errors(oracle_mod, make, ns):
    errs = []
    for n in ns:
        w = make(n)
        phi = oracle_mod.solve(w.source(), w.h)
        x, y, z = w.coords()
        ref = analytic.bodies_potential(w.bodies, x, y, z)
        errs.append(oracle_mod.l1_error(phi, ref))
    return errs


def test_gaussian_second_order(oracle_mod):
    ns = [24, 48, 96]

    def make(n):
        h = 1.0 / n
        return sources.Workload("g", (n, n, n), (h, h, h),
                                [{"kind": "gaussian", "center": (0.5, 0.5, 0.5), "sigma": 0.1, "amp": 1.0}])
    errs = _errors(oracle_mod, make, ns)
    assert errs[0] > errs[1] > errs[2]
    assert order_fit(ns, errs) > 1.8


def test_sphere_better_than_first_order(oracle_mod):
    ns = [24, 48, 96]
    errs = _errors(oracle_mod, lambda n: sources.single_sphere(n, radius=0.3), ns)
    assert errs[-1] < 1e-2
    assert order_fit(ns, errs) > 1.0


def test_anisotropic_spheroid_converges(oracle_mod):
    """e = 0.9, a = 0.25 oblate spheroid in the box [0,1]^2 x [0,2] with
    cells twice as tall as wide (h = (1,1,2)/n): exercises Eq. 6's
    anisotropic widths against the Sec. 4.2 closed form."""
    ns = [24, 48, 96]
    a = 0.25
    b = a * math.sqrt(1 - 0.81)

    def make(n):
        return sources.Workload("sp", (n, n, n), (1.0 / n, 1.0 / n, 2.0 / n),
                                [{"kind": "spheroid", "center": (0.5, 0.5, 1.0), "a": a, "b": b, "rho": 1.0}])
    errs = _errors(oracle_mod, make, ns)
    assert errs[0] > errs[1] > errs[2]
    assert order_fit(ns, errs) > 1.0
    assert errs[-1] < 2e-2
