"""Pins of the oracle's linked octree (Sec. 5) and node properties (count + multipole upsweep)
against the paper's worked example (Fig. 2), a breadth-first walk written independently here,
brute-force counts, closed forms and exact rational arithmetic."""
import collections
from fractions import Fraction

import numpy as np
import pytest

from test_oracle_leaves import golden, random_keys

L = 21
KEY_END = 1 << 63


def bfs_tree(K):
    """Breadth-first walk from the root: a node is internal iff some key of K lies strictly inside it.
    Returns (node keys in placeholder format, first-child indices)."""
    Kset = [int(k) for k in K]
    inner = set(Kset[1:-1])

    def is_internal(start, size):
        if size == 1:
            return False
        # any cornerstone key strictly inside (start, start + size) means the node is subdivided
        import bisect
        j = bisect.bisect_right(Kset, start)
        return j < len(Kset) and Kset[j] < start + size and Kset[j] in inner

    keys, child = [], []
    q = collections.deque([(0, 0)])  # (start, level)
    while q:
        start, lev = q.popleft()
        size = 8 ** (L - lev)
        keys.append((1 << (3 * lev)) | (start >> (3 * (L - lev))))
        if is_internal(start, size):
            child.append(len(keys) + len(q))
            for c in range(8):
                q.append((start + c * size // 8, lev + 1))
        else:
            child.append(0)
    return keys, child


def test_worked_example_fig2(oracle):
    g = golden()
    t = oracle.link(np.array(g["K_refined"], np.uint64))
    assert list(t["NK"]) == g["NK"]
    assert list(t["LO"]) == g["LO"]
    assert list(t["CO"]) == g["CO"]
    assert (len(g["K_refined"]) - 1 - 1) // 7 == 2  # n_i = (n_l - 1) / 7 internal nodes
    assert list(t["parent"]) == [0, 3]
    assert list(t["leaf_to_node"]) == [1, 2] + list(range(9, 17)) + [4, 5, 6, 7, 8]


def test_root_only_tree(oracle):
    t = oracle.link(np.array([0, KEY_END], np.uint64))
    assert list(t["NK"]) == [1] and list(t["CO"]) == [0]
    assert list(t["LO"]) == [0] + [1] * (L + 1)
    assert list(t["leaf_to_node"]) == [0]


@pytest.mark.parametrize("seed", range(10))
def test_link_matches_breadth_first_walk(oracle, seed):
    rng = np.random.default_rng(200 + seed)
    kind = ("uniform", "clustered", "duplicates")[seed % 3]
    P = np.sort(random_keys(rng, int(rng.integers(1, 3000)), kind))
    K = oracle.canonical_leaves(P, int((1, 2, 8, 16, 64)[seed % 5]))
    t = oracle.link(K)
    nl = len(K) - 1
    n = nl + (nl - 1) // 7
    assert t["NK"].size == n
    keys, child = bfs_tree(K)
    assert [int(k) for k in t["NK"]] == keys
    assert [int(c) for c in t["CO"]] == child
    # level offsets: first node of each level, L + 1 entries plus the end marker
    levels = [(int(k).bit_length() - 1) // 3 for k in keys]
    for lev in range(L + 1):
        assert t["LO"][lev] == next((i for i, x in enumerate(levels) if x >= lev), n)
    assert t["LO"][L + 1] == n
    # leaves map to nodes with the same key range
    for i in range(nl):
        v = t["leaf_to_node"][i]
        size = int(K[i + 1]) - int(K[i])
        lev = L - (size.bit_length() - 1) // 3
        assert int(t["NK"][v]) == (1 << (3 * lev)) | (int(K[i]) >> (3 * (L - lev)))
        assert t["CO"][v] == 0
    for g_idx, p in enumerate(t["parent"]):
        assert t["CO"][p] == 1 + 8 * g_idx
    # the internal nodes of level l are the g-th in that order for g in [(LO[l+1]-1)/8, (LO[l+2]-1)/8)
    # (the upsweeps take each level's internal nodes this way)
    internal = [i for i in range(n) if t["CO"][i] != 0]
    assert sorted(internal) == sorted(int(p) for p in t["parent"])
    for lev in range(L):
        lo, hi = t["LO"][lev + 1], t["LO"][lev + 2]
        assert (lo - 1) % 8 == 0 and (hi - 1) % 8 == 0
        want = [i for i in internal if t["LO"][lev] <= i < t["LO"][lev + 1]]
        assert sorted(int(p) for p in t["parent"][(lo - 1) // 8:(hi - 1) // 8]) == want


def brute_node_counts(P, NK):
    out = []
    for nk in NK:
        lev = (int(nk).bit_length() - 1) // 3
        start = (int(nk) ^ (1 << (3 * lev))) << (3 * (L - lev))
        end = start + 8 ** (L - lev)
        out.append(sum(1 for p in P if start <= int(p) < end))
    return np.array(out)


@pytest.mark.parametrize("seed", range(6))
def test_node_counts_brute_force(oracle, seed):
    rng = np.random.default_rng(300 + seed)
    P = np.sort(random_keys(rng, 700, ("uniform", "clustered", "duplicates")[seed % 3]))
    K, N, _ = oracle.build_leaves(P, 8)
    t = oracle.link(K)
    c = oracle.node_counts(P, t["NK"])
    assert np.array_equal(c, brute_node_counts(P, t["NK"]))
    assert c[0] == P.size
    assert np.array_equal(c[t["leaf_to_node"]], N)
    internal = np.nonzero(t["CO"])[0]
    for v in internal:  # the upsweep relation: a node holds the sum of its 8 children
        assert c[v] == c[t["CO"][v]: t["CO"][v] + 8].sum()


# ------------------------------------------------------------------ multipoles (Sec. 5, Sec. 8)
def _tree_for(oracle, x, y, z, ncrit=2):
    box = oracle.bounding_cube(x, y, z)
    k = oracle.keys(x, y, z, box, oracle.HILBERT)
    P, perm = oracle.sort(k)
    K, _, _ = oracle.build_leaves(P, ncrit)
    return P, perm, oracle.link(K)


def test_multipole_single_particle(oracle):
    x, y, z = np.array([0.3]), np.array([-2.0]), np.array([5.5])
    m = np.array([2.5], np.float32)
    P, perm, t = _tree_for(oracle, x, y, z)
    M, com, q = oracle.multipoles(x, y, z, m, P, perm, t["NK"])
    assert M[0] == 2.5 and list(com[0]) == [0.3, -2.0, 5.5] and not q[0].any()


def test_multipole_symmetric_pair(oracle):
    # two equal masses at c +- a e_x: centre c, Q_xx = 2 m a^2, all other components 0
    c, a, mass = np.array([1.0, 2.0, 3.0]), 0.25, 3.0
    x = np.array([c[0] - a, c[0] + a])
    y = np.array([c[1], c[1]])
    z = np.array([c[2], c[2]])
    m = np.full(2, mass, np.float32)
    P, perm, t = _tree_for(oracle, x, y, z, ncrit=4)
    M, com, q = oracle.multipoles(x, y, z, m, P, perm, t["NK"], nodes=[0])
    assert M[0] == 6.0 and np.allclose(com[0], c, rtol=0, atol=1e-15)
    assert q[0][0] == pytest.approx(2 * mass * a * a, rel=1e-15)
    assert np.all(q[0][1:] == 0.0)


def test_multipole_exact_rational(oracle):
    # every node of a small random set against exact rational arithmetic
    rng = np.random.default_rng(7)
    n = 60
    x, y, z = rng.random(n), rng.random(n), rng.random(n)
    m = rng.lognormal(0, 1, n).astype(np.float32)
    P, perm, t = _tree_for(oracle, x, y, z, ncrit=4)
    M, com, q = oracle.multipoles(x, y, z, m, P, perm, t["NK"])
    for v in range(t["NK"].size):
        lev = (int(t["NK"][v]).bit_length() - 1) // 3
        start = (int(t["NK"][v]) ^ (1 << (3 * lev))) << (3 * (L - lev))
        end = start + 8 ** (L - lev)
        idx = [int(perm[j]) for j in range(n) if start <= int(P[j]) < end]
        if not idx:
            assert M[v] == 0 and not com[v].any() and not q[v].any()
            continue
        ms = [Fraction(float(m[i])) for i in idx]
        pos = [[Fraction(float(c[i])) for c in (x, y, z)] for i in idx]
        Mt = sum(ms)
        ct = [sum(mi * p[d] for mi, p in zip(ms, pos)) / Mt for d in range(3)]
        pairs = [(0, 0), (0, 1), (0, 2), (1, 1), (1, 2), (2, 2)]
        qt = [sum(mi * (p[a] - ct[a]) * (p[b] - ct[b]) for mi, p in zip(ms, pos)) for a, b in pairs]
        assert abs(M[v] - float(Mt)) <= 1e-14 * float(Mt)
        assert max(abs(com[v][d] - float(ct[d])) for d in range(3)) <= 1e-14
        scale = max(abs(float(val)) for val in qt) or 1.0
        assert max(abs(q[v][c] - float(qt[c])) for c in range(6)) <= 1e-12 * scale


def test_multipole_translation(oracle):
    # shifting every particle by a vector shifts the centre and leaves the second moments unchanged
    rng = np.random.default_rng(8)
    n = 200
    x, y, z = rng.random(n), rng.random(n), rng.random(n)
    m = rng.lognormal(0, 1, n).astype(np.float32)
    P, perm, t = _tree_for(oracle, x, y, z, ncrit=8)
    M0, c0, q0 = oracle.multipoles(x, y, z, m, P, perm, t["NK"])
    s = np.array([0.5, -0.25, 2.0])  # exact binary fractions keep the particle-to-node assignment
    M1, c1, q1 = oracle.multipoles(x + s[0], y + s[1], z + s[2], m, P, perm, t["NK"])
    assert np.array_equal(M0, M1)
    nz = M0 > 0
    assert np.allclose(c1[nz] - c0[nz], s, atol=1e-12)
    assert np.allclose(q1, q0, rtol=1e-9, atol=1e-12)
