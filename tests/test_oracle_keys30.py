"""Pins of the oracle built for L = 10 (30-bit keys, the other natural key length of Sec. 3).

The L = 10 build is the same C source compiled with ORACLE_L=10. What pins it to something other
than itself:
* grid cells: faces, exact grid points, and the identity cell_10 = floor(cell_21 / 2^11), which
  holds because 2^21 / side = 2^11 (2^10 / side) exactly in IEEE arithmetic;
* keys: a Morton or Hilbert key of 10 levels is the top 30 bits of the 21-level key of any cell
  inside it (octree prefix and nesting of the curves);
* leaves: the literal f/g iteration equals the top-down definition, every leaf holds at most
  N_crit particles unless it is a single level-10 cell, and warm starts reach the cold tree;
* tree: the breadth-first walk written here, brute-force node counts, and, for data that never
  needs more than 10 levels, the 21-level tree with its keys shifted by 33 bits.
"""
import numpy as np
import pytest

L10 = 10
END10 = 1 << 30


def rand_coords(rng, n, kind):
    if kind == "uniform":
        return rng.random(n), rng.random(n), rng.random(n)
    c = rng.random((3, 3))
    s = 10.0 ** rng.uniform(-4, -2, 3)
    w = rng.integers(0, 3, n)
    return tuple(c[d][w] + s[w] * rng.standard_normal(n) for d in range(3))


def test_grid_faces_and_exact_points(oracle):
    assert oracle.grid_coord(0.25, 0.25, 2.0, levels=10) == 0
    assert oracle.grid_coord(2.25, 0.25, 2.0, levels=10) == 1023  # the right face clamps
    assert oracle.grid_coord(-5.0, 0.25, 2.0, levels=10) == 0
    for k in (0, 1, 2, 511, 512, 1000, 1023):  # lo + k side / 2^10 is exactly representable
        assert oracle.grid_coord(-1.0 + k * (4.0 / 1024), -1.0, 4.0, levels=10) == k


@pytest.mark.parametrize("seed", range(4))
def test_grid_cells_nest_in_the_21_level_grid(oracle, seed):
    rng = np.random.default_rng(900 + seed)
    lo, side = rng.uniform(-10, 10), 10.0 ** rng.uniform(-3, 3)
    xs = lo + side * rng.uniform(-0.1, 1.1, 2000)
    # include points on and next to level-10 cell boundaries
    k = rng.integers(0, 1024, 500)
    edge = lo + k * (side / 1024)
    xs = np.concatenate([xs, edge, np.nextafter(edge, -np.inf), np.nextafter(edge, np.inf)])
    for x in xs:
        g21 = oracle.grid_coord(float(x), lo, side)
        assert oracle.grid_coord(float(x), lo, side, levels=10) == g21 >> 11


@pytest.mark.parametrize("curve", [0, 1])
@pytest.mark.parametrize("kind", ["uniform", "clustered"])
def test_keys_are_the_top_30_bits(oracle, curve, kind):
    rng = np.random.default_rng(910 + curve)
    x, y, z = rand_coords(rng, 5000, kind)
    box = oracle.bounding_cube(x, y, z)
    k21 = oracle.keys(x, y, z, box, curve)
    k10 = oracle.keys(x, y, z, box, curve, levels=10)
    assert k10.max() < END10
    assert np.array_equal(k10, k21 >> np.uint64(33))


def test_morton_round_trip_and_bits(oracle):
    for ix, iy, iz in [(1, 0, 0), (0, 1, 0), (0, 0, 1), (1023, 0, 0), (5, 1000, 77), (1023, 1023, 1023)]:
        key = oracle.morton_key(ix, iy, iz, levels=10)
        assert key < END10
        assert oracle.morton_decode(key, levels=10) == (ix, iy, iz)
    assert oracle.morton_key(512, 0, 0, levels=10) == 4 << 27  # top bit of x leads the first digit


def _keys10(rng, n, kind):
    if kind == "uniform":
        return rng.integers(0, END10, n, dtype=np.uint64)
    if kind == "clustered":  # dense spots that reach level 10
        centres = rng.integers(0, END10, 3, dtype=np.uint64)
        off = rng.integers(0, 1 << int(rng.integers(0, 7)), n, dtype=np.uint64)
        return np.minimum(centres[rng.integers(0, 3, n)] + off, np.uint64(END10 - 1))
    vals = rng.integers(0, END10, 4, dtype=np.uint64)
    return vals[rng.integers(0, 4, n)]


@pytest.mark.parametrize("kind", ["uniform", "clustered", "duplicates"])
@pytest.mark.parametrize("ncrit", [1, 4, 32])
def test_leaves_definition_and_balance(oracle, kind, ncrit):
    rng = np.random.default_rng(hash((kind, ncrit)) % 2 ** 32)
    P = np.sort(_keys10(rng, 2500, kind))
    K, N, iters = oracle.build_leaves(P, ncrit, levels=10)
    assert K[0] == 0 and K[-1] == END10 and oracle.check_cornerstone(K, levels=10)
    assert iters <= L10 + 1
    assert np.array_equal(K, oracle.canonical_leaves(P, ncrit, levels=10))
    sizes = np.diff(K.astype(np.int64))
    assert all(N[i] <= ncrit or sizes[i] == 1 for i in range(len(N)))
    # every leaf is a node of the 10-level octree: a power-of-8 size aligned to itself
    for k, s in zip(K[:-1].astype(np.int64), sizes):
        assert s & (s - 1) == 0 and (int(s).bit_length() - 1) % 3 == 0 and k % s == 0
    if kind != "uniform":
        assert (sizes == 1).any()  # the dense spots reach the deepest level
    P1 = np.sort(_keys10(rng, 2000, kind))
    warm, _, _ = oracle.build_leaves(P1, ncrit, K_init=K, levels=10)
    cold, _, _ = oracle.build_leaves(P1, ncrit, levels=10)
    assert np.array_equal(warm, cold)


def _bfs10(K):
    import bisect
    Kset = [int(k) for k in K]
    inner = set(Kset[1:-1])
    keys, child, q = [], [], [(0, 0)]
    head = 0
    while head < len(q):
        start, lev = q[head]
        head += 1
        size = 8 ** (L10 - lev)
        keys.append((1 << (3 * lev)) | (start >> (3 * (L10 - lev))))
        j = bisect.bisect_right(Kset, start)
        if size > 1 and j < len(Kset) and Kset[j] < start + size and Kset[j] in inner:
            child.append(len(q))
            for c in range(8):
                q.append((start + c * size // 8, lev + 1))
        else:
            child.append(0)
    return keys, child


@pytest.mark.parametrize("seed", range(6))
def test_link_and_counts(oracle, seed):
    rng = np.random.default_rng(950 + seed)
    P = np.sort(_keys10(rng, int(rng.integers(1, 3000)), ("uniform", "clustered", "duplicates")[seed % 3]))
    K, N, _ = oracle.build_leaves(P, (1, 4, 16)[seed % 3], levels=10)
    t = oracle.link(K, levels=10)
    nl = len(K) - 1
    assert t["NK"].size == nl + (nl - 1) // 7 and t["LO"].size == L10 + 2
    keys, child = _bfs10(K)
    assert [int(k) for k in t["NK"]] == keys and [int(c) for c in t["CO"]] == child
    c = oracle.node_counts(P, t["NK"], levels=10)
    for v, nk in enumerate(t["NK"]):
        lev = (int(nk).bit_length() - 1) // 3
        start = (int(nk) ^ (1 << (3 * lev))) << (3 * (L10 - lev))
        assert c[v] == np.count_nonzero((P >= np.uint64(start)) & (P < np.uint64(start + 8 ** (L10 - lev))))
    assert np.array_equal(c[t["leaf_to_node"]], N)


def test_shallow_tree_equals_the_21_level_tree(oracle):
    # uniform data with few particles never needs 10 levels: both key lengths give the same tree
    rng = np.random.default_rng(977)
    x, y, z = rng.random(20_000), rng.random(20_000), rng.random(20_000)
    box = np.array([0.0, 0.0, 0.0, 1.0])
    for curve in (0, 1):
        a = oracle.full_build(x, y, z, curve, 16, box=box)
        b = oracle.full_build(x, y, z, curve, 16, box=box, levels=10)
        assert int(np.diff(a["K"].astype(object)).min()) >= 1 << 33  # no leaf below level 10
        assert np.array_equal(b["K"], a["K"] >> np.uint64(33))
        assert np.array_equal(b["perm"], a["perm"]) and np.array_equal(b["counts"], a["counts"])
        # placeholder keys of levels <= 10 do not depend on the key length
        assert np.array_equal(b["NK"], a["NK"])
        assert np.array_equal(b["CO"], a["CO"]) and np.array_equal(b["LO"][:11], a["LO"][:11])
