"""Pins of the oracle's Sec. 6 helpers: the cube from per-axis bounds reduced over processes, and
the SFC domain decomposition into bins of consecutive leaves with about N_tot / n_ranks particles.

The cube must equal the bounding cube of the union computed from the raw coordinates; the cuts are
checked against their definition by brute force (each cut is the first leaf whose preceding leaves
hold at least r N_tot / n_ranks particles), against hand-worked cases, and for the balance the
paper asks for (every bin within one leaf's count of N_tot / n_ranks)."""
from fractions import Fraction

import numpy as np
import pytest


def test_cube_from_bounds_equals_bounding_cube_of_the_union(oracle):
    rng = np.random.default_rng(5)
    parts = [rng.normal(size=(3, k)) * s + c for k, s, c in ((100, 1.0, 0.0), (7, 3.0, 2.0), (50, 0.1, -4.0))]
    allp = np.concatenate(parts, axis=1)
    lo = np.min([p.min(axis=1) for p in parts], axis=0)
    hi = np.max([p.max(axis=1) for p in parts], axis=0)
    box = oracle.cube_from_bounds(np.concatenate([lo, hi]))
    assert np.array_equal(box, oracle.bounding_cube(allp[0], allp[1], allp[2]))


def test_cube_from_bounds_degenerate_cases(oracle):
    inf = np.inf
    assert np.array_equal(oracle.cube_from_bounds([inf, inf, inf, -inf, -inf, -inf]), [0.0, 0.0, 0.0, 1.0])
    # a single point: zero extent gives side 1 at the point
    assert np.array_equal(oracle.cube_from_bounds([2.0, -1.0, 0.5, 2.0, -1.0, 0.5]), [2.0, -1.0, 0.5, 1.0])
    # the side is the largest extent, lo the per-axis minima
    assert np.array_equal(oracle.cube_from_bounds([0.0, 1.0, 2.0, 4.0, 2.0, 9.0]), [0.0, 1.0, 2.0, 7.0])


def test_decompose_hand_cases(oracle):
    assert oracle.decompose(np.ones(100, np.uint32), 4).tolist() == [0, 25, 50, 75, 100]
    assert oracle.decompose(np.ones(10, np.uint32), 1).tolist() == [0, 10]
    # counts 5, 0, 5, 0, 10 (total 20), two ranks: the first leaf with 10 particles before it is leaf 3
    assert oracle.decompose(np.array([5, 0, 5, 0, 10], np.uint32), 2).tolist() == [0, 3, 5]
    # no particles: every inner cut at 0
    assert oracle.decompose(np.zeros(6, np.uint32), 3).tolist() == [0, 0, 0, 6]
    # more ranks than leaves with particles: later bins are empty and end at n_l
    assert oracle.decompose(np.array([7, 0, 0], np.uint32), 4).tolist() == [0, 1, 1, 1, 3]


@pytest.mark.parametrize("seed", range(6))
def test_decompose_matches_definition_and_balance(oracle, seed):
    rng = np.random.default_rng(seed)
    nl = int(rng.integers(1, 3000))
    N = rng.integers(0, 80, nl).astype(np.uint32)
    N[rng.random(nl) < 0.3] = 0
    world = int(rng.integers(1, 40))
    cuts = oracle.decompose(N, world)
    prefix = np.concatenate([[0], np.cumsum(N.astype(np.int64))])
    total = int(prefix[-1])
    assert cuts[0] == 0 and cuts[-1] == nl and np.all(np.diff(cuts) >= 0)
    for r in range(1, world):
        want = next((i for i in range(nl) if Fraction(int(prefix[i])) >= Fraction(total * r, world)), nl)
        assert cuts[r] == want
    # balance: a bin's count differs from N_tot / n_ranks by less than the largest leaf count
    # (bins are cut at the leaves, which are never divided)
    if total > 0:
        bins = prefix[cuts[1:]] - prefix[cuts[:-1]]
        assert np.all(np.abs(bins - total / world) <= int(N.max()) + 1e-9)
