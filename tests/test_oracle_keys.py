"""Pins of the oracle's key generation (Sec. 3) against closed forms, exact arithmetic and brute force.

Nothing here re-types the oracle's formulas: the Morton checks use single-bit closed forms and
superposition, the grid checks use exact rational arithmetic, and the Hilbert checks are
exhaustive properties of a Hilbert curve (bijection, unit steps, octree nesting).
"""
import itertools
from fractions import Fraction

import numpy as np
import pytest

L = 21


# ------------------------------------------------------------------ bounding cube + grid (Sec. 3)
def test_bounding_cube_closed_form(oracle):
    x = np.array([0.5, -1.0, 2.0])
    y = np.array([0.0, 0.25, 0.125])
    z = np.array([3.0, 3.0, 7.0])
    box = oracle.bounding_cube(x, y, z)
    # lo = per-axis minimum; side = largest per-axis extent (x: 3.0, y: 0.25, z: 4.0)
    assert list(box) == [-1.0, 0.0, 3.0, 4.0]


def test_bounding_cube_degenerate(oracle):
    box = oracle.bounding_cube([2.0, 2.0], [2.0, 2.0], [2.0, 2.0])
    assert list(box) == [2.0, 2.0, 2.0, 1.0]
    assert list(oracle.bounding_cube([], [], [])) == [0.0, 0.0, 0.0, 1.0]


def test_grid_coord_faces(oracle):
    # the left face maps to 0, the right face to the last cell, outside points are clamped
    for lo, side in [(0.0, 1.0), (-1.5, 3.0), (0.1, 0.7), (-20.0, 40.0)]:
        assert oracle.grid_coord(lo, lo, side) == 0
        assert oracle.grid_coord(lo + side, lo, side) == 2 ** L - 1
        assert oracle.grid_coord(lo - 1.0, lo, side) == 0
        assert oracle.grid_coord(lo + 2 * side, lo, side) == 2 ** L - 1


def test_grid_coord_exact_grid_points(oracle):
    # x = k / 2^21 in the unit cube is exactly representable and lands in cell k
    rng = np.random.default_rng(1)
    for k in list(rng.integers(0, 2 ** L, 200)) + [0, 1, 2 ** L - 1]:
        assert oracle.grid_coord(float(k) / 2 ** L, 0.0, 1.0) == k
        # the point just below the cell boundary belongs to the previous cell
        if k > 0:
            below = np.nextafter(float(k) / 2 ** L, 0.0)
            assert oracle.grid_coord(below, 0.0, 1.0) == k - 1


def test_grid_coord_exact_rational(oracle):
    # away from cell boundaries the cell is floor of the exact rational (x - lo) * 2^21 / side
    rng = np.random.default_rng(2)
    for _ in range(2000):
        lo = float(rng.uniform(-10, 10))
        side = float(rng.uniform(0.01, 30))
        x = lo + float(rng.uniform(0, side))
        exact = (Fraction(x) - Fraction(lo)) * 2 ** L / Fraction(side)
        g = oracle.grid_coord(x, lo, side)
        frac = exact - (exact.numerator // exact.denominator)
        if Fraction(1, 10 ** 6) < frac < 1 - Fraction(1, 10 ** 6):
            assert g == min(int(exact), 2 ** L - 1)
        else:
            assert abs(g - int(exact)) <= 1


# ------------------------------------------------------------------ Morton (Sec. 3)
def test_morton_single_bits(oracle):
    # bit b of x lands at key bit 3b+2, of y at 3b+1, of z at 3b (x is the high bit of a digit)
    for b in range(L):
        assert oracle.morton_key(1 << b, 0, 0) == 1 << (3 * b + 2)
        assert oracle.morton_key(0, 1 << b, 0) == 1 << (3 * b + 1)
        assert oracle.morton_key(0, 0, 1 << b) == 1 << (3 * b)


def test_morton_superposition_and_range(oracle):
    rng = np.random.default_rng(3)
    for _ in range(500):
        ix, iy, iz = (int(v) for v in rng.integers(0, 2 ** L, 3))
        k = oracle.morton_key(ix, iy, iz)
        assert k == oracle.morton_key(ix, 0, 0) | oracle.morton_key(0, iy, 0) | oracle.morton_key(0, 0, iz)
        assert 0 <= k < 2 ** 63
        assert oracle.morton_decode(k) == (ix, iy, iz)
    m = 2 ** L - 1
    assert oracle.morton_key(m, m, m) == 2 ** 63 - 1


def test_morton_octree_prefix(oracle):
    # Sec. 3: the first i octal digits identify the level-i octree node containing the point
    rng = np.random.default_rng(4)
    for _ in range(300):
        ix, iy, iz = (int(v) for v in rng.integers(0, 2 ** L, 3))
        k = oracle.morton_key(ix, iy, iz)
        for i in range(L + 1):
            s = L - i
            assert k >> (3 * s) == oracle.morton_key(ix >> s, iy >> s, iz >> s)


# ------------------------------------------------------------------ Hilbert (Sec. 1, Sec. 3)
@pytest.mark.parametrize("order", [1, 2, 3, 4])
def test_hilbert_bijection_and_unit_steps(oracle, order):
    side = 1 << order
    cells = {}
    for p in itertools.product(range(side), repeat=3):
        k = oracle.hilbert_key(*p, order=order)
        assert 0 <= k < side ** 3
        assert k not in cells
        cells[k] = p
    assert len(cells) == side ** 3
    assert cells[0] == (0, 0, 0)
    for k in range(side ** 3 - 1):  # consecutive keys are face neighbours: a continuous curve
        a, b = cells[k], cells[k + 1]
        assert sum(abs(u - v) for u, v in zip(a, b)) == 1
    last = cells[side ** 3 - 1]  # a Hilbert curve ends on a corner of the cube
    assert all(c in (0, side - 1) for c in last)


@pytest.mark.parametrize("order", [2, 3, 4])
def test_hilbert_octree_prefix(oracle, order):
    # Sec. 3: the curve traverses the cube octant by octant, so every level-i node is one aligned
    # key range: cells sharing the top i coordinate bits share the top i octal digits.
    side = 1 << order
    for i in range(1, order + 1):
        groups = {}
        for p in itertools.product(range(side), repeat=3):
            node = tuple(c >> (order - i) for c in p)
            groups.setdefault(node, set()).add(oracle.hilbert_key(*p, order=order) >> (3 * (order - i)))
        assert all(len(v) == 1 for v in groups.values())
        assert len({next(iter(v)) for v in groups.values()}) == 8 ** i


@pytest.mark.parametrize("order", [2, 3, 4, 5])
def test_hilbert_nesting_across_orders(oracle, order):
    # refining the grid keeps the coarse key as prefix
    side = 1 << order
    rng = np.random.default_rng(order)
    pts = rng.integers(0, side, (400, 3))
    for p in pts:
        p = tuple(int(c) for c in p)
        assert oracle.hilbert_key(*p, order=order) >> 3 == oracle.hilbert_key(*(c >> 1 for c in p),
                                                                              order=order - 1)


def test_hilbert_full_order_properties(oracle):
    rng = np.random.default_rng(5)
    for _ in range(500):
        p = tuple(int(v) for v in rng.integers(0, 2 ** L, 3))
        k = oracle.hilbert_key(*p)
        assert 0 <= k < 2 ** 63
        assert oracle.hilbert_decode(k) == p
        for i in (1, 5, 13, 20):
            s = L - i
            assert k >> (3 * s) == oracle.hilbert_key(*(c >> s for c in p), order=i)
    for _ in range(500):  # random unit steps along the order-21 curve
        k = int(rng.integers(0, 2 ** 63 - 1))
        a, b = oracle.hilbert_decode(k), oracle.hilbert_decode(k + 1)
        assert sum(abs(u - v) for u, v in zip(a, b)) == 1


def test_keys_array_entry(oracle):
    x = np.array([0.0, 0.999999, 0.5, 0.25])
    y = np.array([0.0, 0.999999, 0.5, 0.75])
    z = np.array([0.0, 0.999999, 0.5, 0.125])
    box = [0.0, 0.0, 0.0, 1.0]
    km = oracle.keys(x, y, z, box, oracle.MORTON)
    kh = oracle.keys(x, y, z, box, oracle.HILBERT)
    for i in range(4):
        g = [oracle.grid_coord(c[i], 0.0, 1.0) for c in (x, y, z)]
        assert km[i] == oracle.morton_key(*g)
        assert kh[i] == oracle.hilbert_key(*g)
    # the centre point (0.5, 0.5, 0.5) is cell 2^20 on every axis: Morton digit 7 then zeros
    assert int(km[2]) == 7 << 60
