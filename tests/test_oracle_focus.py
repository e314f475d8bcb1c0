"""Pins of the oracle's locally essential (focused) octree (Sec. 7) on one process.

* the tiling of the focus range: exact cover by aligned octree nodes, checked cell by cell;
* the minimum-distance MAC: brute force over every grid cell of a small focus (L = 10 build);
* limits that reduce to the balanced tree of Sec. 4: a focus covering every key, or theta so
  small that no node passes the MAC; an empty focus accepts every node (the root stays a leaf);
* the literal f / g1^LE / g2 / g3 iteration equals the top-down definition, also from a warm start;
* the three conditions of the definition, checked node by node with the brute-force MAC.
"""
import numpy as np
import pytest

END10 = 1 << 30


def _decoder(oracle, curve):
    if curve == 0:
        return lambda k: oracle.morton_decode(int(k), levels=10)
    return lambda k: oracle.hilbert_decode(int(k), order=10)


def _brute_mac(oracle, cells, start, level, theta, curve):
    """r_min^2 > (l / theta)^2 with r_min over every cell of the focus, by enumeration."""
    l = 1 << (10 - level)
    c = np.array(_decoder(oracle, curve)(start)) // l * l
    gap = np.maximum(0, np.maximum(cells - (c + l), c - (cells + 1)))
    r2 = (gap * gap).sum(1).min()
    q = l / theta
    return float(r2) > q * q


@pytest.mark.parametrize("f", [(0, 1), (5, 1000), (8 ** 5 * 3 + 17, 8 ** 6 * 5 + 3), (0, END10), (END10 - 9, END10)])
def test_focus_tiles_cover_the_range(oracle, f):
    tiles = oracle.focus_tiles(*f, levels=10)
    s = f[0]
    for start, level in tiles:
        size = 8 ** (10 - level)
        assert start == s and start % size == 0
        s += size
    assert s == f[1]
    assert len(tiles) <= 2 * 7 * 10


@pytest.mark.parametrize("curve", [0, 1])
@pytest.mark.parametrize("seed", range(3))
def test_mac_brute_force(oracle, curve, seed):
    rng = np.random.default_rng(70 + seed + 10 * curve)
    f_start = int(rng.integers(0, END10 - 5000))
    f_end = f_start + int(rng.integers(1, 3000))
    dec = _decoder(oracle, curve)
    cells = np.array([dec(k) for k in range(f_start, f_end)], np.int64)
    for _ in range(60):
        level = int(rng.integers(1, 8))
        size = 8 ** (10 - level)
        start = int(rng.integers(0, END10 // size)) * size
        theta = float(rng.choice([0.2, 0.5, 0.75, 1.0]))
        assert oracle.mac_passes(start, level, f_start, f_end, theta, curve, levels=10) == \
            _brute_mac(oracle, cells, start, level, theta, curve)


def _keys(rng, n, levels=21):
    end = 1 << (3 * levels)
    centres = rng.integers(0, end, 4, dtype=np.uint64)
    off = rng.integers(0, end // 64, n, dtype=np.uint64)
    k = np.minimum(centres[rng.integers(0, 4, n)] + off, np.uint64(end - 1))
    return np.sort(np.concatenate([k, rng.integers(0, end, n // 4, dtype=np.uint64)]))


@pytest.mark.parametrize("curve", [0, 1])
def test_limits_reduce_to_the_balanced_tree(oracle, curve):
    rng = np.random.default_rng(80 + curve)
    P = _keys(rng, 4000)
    full = oracle.canonical_leaves(P, 16)
    K, _, _ = oracle.build_focus_leaves(P, 16, 0, 1 << 63, 0.5, curve)  # focus = every key
    assert np.array_equal(K, full)
    f = (int(P[1000]), int(P[1200]))
    K, _, _ = oracle.build_focus_leaves(P, 16, *f, 1e-30, curve)  # no node passes the MAC
    assert np.array_equal(K, full)
    K, _, _ = oracle.build_focus_leaves(P, 16, 7, 7, 0.5, curve)  # empty focus
    assert list(K) == [0, 1 << 63]


def _check_definition(oracle, P, K, ncrit, f, theta, curve, levels=21):
    end = 1 << (3 * levels)

    def count(s, size):
        return int(np.searchsorted(P, np.uint64(s + size))) - int(np.searchsorted(P, np.uint64(s)))

    def outside(s, size):
        return f[1] <= f[0] or s + size <= f[0] or s >= f[1]

    Ki = [int(k) for k in K]
    for i in range(len(Ki) - 1):  # leaves
        s, size = Ki[i], Ki[i + 1] - Ki[i]
        level = levels - (size.bit_length() - 1) // 3
        c = count(s, size)
        if size > 1 and c > ncrit:  # an over-full leaf is only allowed outside F when it passes the MAC
            assert outside(s, size) and oracle.mac_passes(s, level, *f, theta, curve, levels=levels)
    internal = set()
    for i in range(len(Ki) - 1):  # proper ancestors of the leaves are the internal nodes
        size = (Ki[i + 1] - Ki[i]) * 8
        while size <= end:
            internal.add(((Ki[i] // size) * size, size))
            size *= 8
    for s, size in internal:
        level = levels - (size.bit_length() - 1) // 3
        assert count(s, size) > ncrit
        if outside(s, size):
            assert not oracle.mac_passes(s, level, *f, theta, curve, levels=levels)


@pytest.mark.parametrize("curve", [0, 1])
@pytest.mark.parametrize("seed", range(6))
def test_iteration_equals_definition(oracle, curve, seed):
    rng = np.random.default_rng(90 + seed + 20 * curve)
    P = _keys(rng, 3000)
    ncrit = (2, 8, 32)[seed % 3]
    theta = (0.3, 0.6, 1.0)[seed % 3]
    a, b = sorted(rng.integers(0, P.size, 2))
    f = (int(P[a]), int(P[b]) + 1)
    K, N, iters = oracle.build_focus_leaves(P, ncrit, *f, theta, curve)
    assert oracle.check_cornerstone(K)
    assert np.array_equal(K, oracle.canonical_focus_leaves(P, ncrit, *f, theta, curve))
    assert iters <= 22
    _check_definition(oracle, P, K, ncrit, f, theta, curve)
    # warm start from the balanced tree of all particles reaches the same focused tree
    Kg = oracle.canonical_leaves(P, ncrit)
    Kw, _, _ = oracle.build_focus_leaves(P, ncrit, *f, theta, curve, K_init=Kg)
    assert np.array_equal(Kw, K)
    # a focused tree is coarser than the balanced tree away from F
    assert len(K) <= len(Kg)
