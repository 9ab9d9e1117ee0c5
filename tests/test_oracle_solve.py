"""Pins for the oracle's solve (route 2) against the definition (route 1)
and against invariants the convolution must satisfy (CPU only).

The mesh-doubling method reproduces the aperiodic discrete convolution
exactly up to rounding (Sec. 2.1), so route 2 must match direct summation to
~1e-12; the impulse response of the solve is the Green's function itself.
"""
import itertools

import numpy as np
import pytest


def rand_src(N, seed, frac=0.5):
    g = np.random.default_rng(seed)
    s = g.uniform(0.0, 1.0, (N[2], N[1], N[0]))
    s[g.uniform(size=s.shape) > frac] = 0.0
    return s


CASES = [
    ((8, 8, 8), (1.0, 1.0, 1.0)),
    ((16, 16, 16), (1.0 / 16, 1.0 / 16, 1.0 / 16)),
    ((5, 7, 9), (1.0, 1.0, 1.0)),
    ((12, 10, 6), (0.5, 0.25, 1.0)),
    ((16, 12, 8), (1.0, 1.0, 2.0)),
    ((1, 1, 1), (1.0, 1.0, 1.0)),
    ((1, 6, 3), (0.3, 0.2, 0.5)),
    ((13, 11, 3), (1.0, 2.0, 1.0)),
]


@pytest.mark.parametrize("N,h", CASES)
def test_route2_equals_direct_sum(oracle_mod, N, h):
    src = rand_src(N, seed=sum(N))
    ref = oracle_mod.direct_sum(src, h)
    phi = oracle_mod.solve(src, h)
    assert oracle_mod.max_rel_error(phi, ref) < 1e-12
    # the sampled direct sum agrees with the full one
    cells = np.arange(0, src.size, max(1, src.size // 17))
    pts = oracle_mod.direct_points(src, h, cells)
    assert np.max(np.abs(pts - ref.ravel()[cells])) <= 1e-14 * np.max(np.abs(ref))


@pytest.mark.parametrize("N,M", [((8, 8, 8), (16, 18, 20)), ((5, 7, 9), (9, 13, 17)), ((6, 6, 6), (24, 12, 16))])
def test_any_mesh_at_least_2N_minus_1(oracle_mod, N, M):
    """Offsets span [-(N-1), N-1]; any doubled mesh M >= 2N-1 holds them
    without aliasing, so the cropped result does not depend on M."""
    h = (1.0, 0.5, 2.0)
    src = rand_src(N, seed=3)
    a = oracle_mod.solve(src, h)
    b = oracle_mod.solve(src, h, M=M)
    assert oracle_mod.max_rel_error(b, a) < 1e-13


@pytest.mark.parametrize("N,h", [((8, 6, 5), (1.0, 1.0, 1.0)), ((7, 9, 4), (0.5, 0.25, 1.0))])
def test_impulse_response_is_green(oracle_mod, N, h):
    Nx, Ny, Nz = N
    for corner in [(0, 0, 0), (Nx - 1, Ny - 1, Nz - 1), (Nx // 2, 0, Nz - 1)]:
        src = np.zeros((Nz, Ny, Nx))
        src[corner[2], corner[1], corner[0]] = 1.0
        phi = oracle_mod.solve(src, h)
        want = np.empty_like(phi)
        for k, j, i in itertools.product(range(Nz), range(Ny), range(Nx)):
            want[k, j, i] = oracle_mod.green((abs(i - corner[0]), abs(j - corner[1]), abs(k - corner[2])), h)
        assert np.max(np.abs(phi - want)) < 1e-14 * np.max(np.abs(want))


def test_linearity(oracle_mod):
    N, h = (10, 8, 6), (0.5, 0.25, 1.0)
    a, b = rand_src(N, 1), rand_src(N, 2)
    pa, pb = oracle_mod.solve(a, h), oracle_mod.solve(b, h)
    pab = oracle_mod.solve(2.5 * a - 0.75 * b, h)
    assert oracle_mod.max_rel_error(pab, 2.5 * pa - 0.75 * pb) < 1e-13


def test_translation(oracle_mod):
    """A compact source shifted inside the box gives the shifted potential."""
    N, h = (12, 12, 12), (1.0, 1.0, 1.0)
    src = np.zeros((12, 12, 12))
    src[2:6, 3:5, 1:7] = rand_src((6, 2, 4), 5, frac=1.0)
    s = (3, 2, 4)  # shift in x, y, z
    moved = np.roll(src, (s[2], s[1], s[0]), axis=(0, 1, 2))
    p0, p1 = oracle_mod.solve(src, h), oracle_mod.solve(moved, h)
    # compare on the overlap region where both potentials are defined
    a = p1[s[2]:, s[1]:, s[0]:]
    b = p0[:N[2] - s[2], :N[1] - s[1], :N[0] - s[0]]
    assert np.max(np.abs(a - b)) < 1e-13 * np.max(np.abs(p0))


def test_reflection_and_axis_permutation(oracle_mod):
    N, h = (9, 9, 9), (1.0, 1.0, 1.0)
    src = rand_src(N, 11)
    p = oracle_mod.solve(src, h)
    pr = oracle_mod.solve(src[:, :, ::-1], h)
    assert np.max(np.abs(pr - p[:, :, ::-1])) < 1e-13 * np.max(np.abs(p))
    pt = oracle_mod.solve(np.ascontiguousarray(src.transpose(2, 1, 0)), h)
    assert np.max(np.abs(pt - p.transpose(2, 1, 0))) < 1e-13 * np.max(np.abs(p))
    # anisotropic widths permute with the axes
    h2 = (0.5, 1.0, 2.0)
    q = oracle_mod.solve(src, h2)
    qt = oracle_mod.solve(np.ascontiguousarray(src.transpose(2, 1, 0)), (2.0, 1.0, 0.5))
    assert np.max(np.abs(qt - q.transpose(2, 1, 0))) < 1e-13 * np.max(np.abs(q))


def test_width_scaling(oracle_mod):
    """G scales as h^3 / h = h^2, so scaling every width by s scales phi by s^2."""
    N, h = (8, 7, 6), (0.5, 0.25, 1.0)
    src = rand_src(N, 21)
    p = oracle_mod.solve(src, h)
    s = 3.0
    ps = oracle_mod.solve(src, tuple(s * v for v in h))
    assert oracle_mod.max_rel_error(ps, s * s * p) < 1e-13
