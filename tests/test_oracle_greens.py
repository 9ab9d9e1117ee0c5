"""Pins for the oracle's Green's function and doubled-mesh table (Sec. 2.1).

Checked against what the paper states about them in words rather than by
retyping the formulas: the isotropic unit-width case is the textbook
-1/(4 pi r) (Eq. 2); the Jacobian scaling of Eq. 6; the origin value equals
the largest off-origin magnitude on the mesh (Eq. 9 text); periodic
replication of the doubled table reproduces the Green's function at every
offset within +-(n-1) (Eq. 9 text); the transform of a real even table is
real, even, and its k = 0 bin is the table sum.
"""
import itertools
import math

import numpy as np
import pytest


def test_unit_width_is_textbook_green(oracle_mod):
    h = (1.0, 1.0, 1.0)
    for d in [(1, 0, 0), (0, 3, 4), (2, 2, 1), (7, 5, 3)]:
        r = math.sqrt(sum(v * v for v in d))
        assert oracle_mod.green(d, h) == pytest.approx(-1.0 / (4 * math.pi * r), rel=1e-15)


@pytest.mark.parametrize("h", [(0.1, 0.1, 0.1), (0.5, 0.25, 1.0), (1.0, 1.0, 2.0), (2.0, 0.3, 0.7)])
def test_jacobian_scaling(oracle_mod, h):
    """Eq. 6 is h_x h_y h_z times the unit Green's function at the physical
    distance: check against the unit-width values at physically equal
    distances (an offset along one axis of length L/h_axis)."""
    hx, hy, hz = h
    vol = hx * hy * hz
    for axis, hv in enumerate(h):
        for n in (1, 2, 5):
            d = [0, 0, 0]
            d[axis] = n
            r_phys = n * hv
            unit = oracle_mod.green((1, 0, 0), (1.0, 1.0, 1.0))  # -1/(4 pi)
            assert oracle_mod.green(d, h) == pytest.approx(vol * unit / r_phys, rel=1e-15)
    # sign: attractive potential, negative everywhere
    for d in itertools.product(range(3), repeat=3):
        assert oracle_mod.green(d, h) < 0


@pytest.mark.parametrize("h", [(1.0, 1.0, 1.0), (1.0, 1.0, 2.0), (0.3, 0.2, 0.5), (0.7, 0.9, 0.4)])
def test_origin_is_largest_off_origin_value(oracle_mod, h):
    vals = [abs(oracle_mod.green(d, h)) for d in itertools.product(range(-3, 4), repeat=3) if d != (0, 0, 0)]
    assert abs(oracle_mod.green((0, 0, 0), h)) == pytest.approx(max(vals), rel=1e-15)
    assert oracle_mod.green((0, 0, 0), h) < 0


@pytest.mark.parametrize("N,h", [((4, 5, 3), (1.0, 1.0, 1.0)), ((6, 4, 5), (0.5, 0.25, 1.0))])
def test_table_replicates_green(oracle_mod, N, h):
    M = tuple(2 * n for n in N)
    T = oracle_mod.green_table(M, h)
    assert T.shape == (M[2], M[1], M[0])
    for dz in range(-N[2] + 1, N[2]):
        for dy in range(-N[1] + 1, N[1]):
            for dx in range(-N[0] + 1, N[0]):
                want = oracle_mod.green((abs(dx), abs(dy), abs(dz)), h)
                assert T[dz % M[2], dy % M[1], dx % M[0]] == want
    # mirror symmetry in each axis
    assert np.array_equal(T, np.roll(T[::-1, :, :], 1, axis=0))
    assert np.array_equal(T, np.roll(T[:, ::-1, :], 1, axis=1))
    assert np.array_equal(T, np.roll(T[:, :, ::-1], 1, axis=2))


@pytest.mark.parametrize("h", [(1.0, 1.0, 1.0), (0.5, 0.25, 1.0)])
def test_green_block_is_the_table_read_in_a_box(oracle_mod, h):
    """The block evaluator equals the doubled table on its non-negative
    offsets (so a corner impulse's response can be read slab by slab), and a
    block away from the origin equals the scalar function cell by cell."""
    N = (5, 4, 6)
    M = tuple(2 * n for n in N)
    T = oracle_mod.green_table(M, h)
    B = oracle_mod.green_block((0, 0, 0), N, h)
    assert np.array_equal(B, T[:N[2], :N[1], :N[0]])
    lo = (3, 7, 2)
    B = oracle_mod.green_block(lo, (3, 2, 4), h)
    for k, j, i in itertools.product(range(4), range(2), range(3)):
        assert B[k, j, i] == oracle_mod.green((lo[0] + i, lo[1] + j, lo[2] + k), h)


@pytest.mark.parametrize("M,h", [((8, 8, 8), (1.0, 1.0, 1.0)), ((12, 8, 10), (0.5, 0.25, 1.0))])
def test_spectrum_real_even(oracle_mod, M, h):
    Gt = oracle_mod.green_spectrum(M, h)
    T = oracle_mod.green_table(M, h)
    scale = np.max(np.abs(Gt))
    assert np.max(np.abs(Gt.imag)) < 1e-15 * scale * 10
    assert Gt[0, 0, 0].real == pytest.approx(T.sum() / T.size, rel=1e-13)
    R = Gt.real
    for ax in range(3):
        flipped = np.roll(np.flip(R, axis=ax), 1, axis=ax)
        assert np.max(np.abs(flipped - R)) < 1e-14 * scale
