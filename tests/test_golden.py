"""Stored fixtures under tests/golden/ (CPU).

* paper_test_problems.txt: the parameters the paper's Sec. 4 states for its
  test problems; the seeded generators must use them.
* sphere16.txt, random12x10x8_h.txt: the potential at fixed cells by the
  direct sum of the definition (oracle route 1), written by
  tests/golden/make_golden.py.  Route 2 (the paper's padded-FFT route) must
  reproduce them, and route 1 must keep reproducing itself.
"""
import math
import os

import numpy as np
import pytest

from paper_1106_0557_gb300 import sources

HERE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def paper_values():
    out = {}
    for line in open(os.path.join(HERE, "paper_test_problems.txt")):
        line = line.split("#", 1)[0].strip()
        if line:
            k, v = (s.strip() for s in line.split("=", 1))
            out[k] = [float(x) for x in v.split()]
    return out


def golden(name):
    cells, vals = [], []
    for line in open(os.path.join(HERE, name + ".txt")):
        if line.startswith("#"):
            continue
        c, v = line.split()
        cells.append(int(c))
        vals.append(float(v))
    return np.asarray(cells), np.asarray(vals)


def golden_sources():
    # the same inputs make_golden.py uses
    yield "sphere16", sources.single_sphere(16).source(), sources.single_sphere(16).h
    g = np.random.default_rng(2024)
    yield "random12x10x8_h", g.uniform(0.0, 1.0, (8, 10, 12)), (0.5, 0.25, 1.0)


def test_generators_use_the_papers_parameters():
    p = paper_values()
    w = sources.paper_sphere(48)
    (b,) = w.bodies
    assert b["radius"] == p["sphere.radius"][0] and b["rho"] == p["sphere.density"][0]
    assert b["center"] == (p["sphere.center"][0],) * 3
    assert w.lo == (p["sphere.box_lo"][0],) * 3
    assert w.lo[0] + 48 * w.h[0] == pytest.approx(p["sphere.box_hi"][0])
    w = sources.paper_spheroid(48)
    (b,) = w.bodies
    e = p["spheroid.eccentricity"][0]
    assert b["a"] == p["spheroid.semi_major"][0] and b["rho"] == p["spheroid.density"][0]
    assert b["b"] == pytest.approx(b["a"] * math.sqrt(1.0 - e * e), rel=1e-15)
    assert 48 * w.h[0] == pytest.approx(p["spheroid.box_size"][0])
    w = sources.binary_spheroid()
    assert w.N == (2 * int(p["binary.paper_n"][0]),) + (int(p["binary.paper_n"][0]),) * 2
    e = p["binary.eccentricity"][0]
    for b in w.bodies:
        assert b["a"] == p["binary.semi_major"][0]
        assert b["b"] == pytest.approx(b["a"] * math.sqrt(1.0 - e * e), rel=1e-15)
        assert abs(b["center"][0]) == p["binary.center_x"][0]
    assert w.N[0] * w.h[0] == pytest.approx(p["binary.box_x"][0])
    assert list(sources.PAPER_LADDER) == [int(v) for v in p["ladder"]]


@pytest.mark.parametrize("name,src,h", list(golden_sources()), ids=lambda x: x if isinstance(x, str) else "")
def test_oracle_routes_reproduce_the_stored_direct_sums(oracle_mod, name, src, h):
    cells, want = golden(name)
    # route 1 reproduces itself (regression)
    assert np.allclose(oracle_mod.direct_points(src, h, cells), want, rtol=1e-14, atol=0)
    # route 2, the paper's padded-FFT route, agrees with the definition
    phi = oracle_mod.solve(src, h)
    assert np.max(np.abs(phi.ravel()[cells] - want)) / np.max(np.abs(phi)) < 1e-12
