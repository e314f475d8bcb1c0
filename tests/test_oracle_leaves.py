"""Pins of the oracle's sort and cornerstone leaf construction (Sec. 4) against brute force, the
paper's invariants (Eq. cstone, the balance definition), its worked example (Fig. 1) and the
uniqueness of the balanced tree."""
import os

import numpy as np
import pytest

L = 21
KEY_END = 1 << 63
GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "fig1_fig2_example.txt")


def golden():
    out = {}
    for line in open(GOLDEN):
        if line.startswith("#") or not line.strip():
            continue
        name, *vals = line.split()
        base = 8 if name.startswith(("K_", "NK")) else 10
        out[name] = [int(v, base) for v in vals]
    return out


def random_keys(rng, n, kind):
    if kind == "uniform":
        return rng.integers(0, KEY_END, n, dtype=np.uint64)
    if kind == "clustered":  # a few dense spots: deep trees
        centres = rng.integers(0, KEY_END, 4, dtype=np.uint64)
        spread = np.uint64(1) << np.uint64(int(rng.integers(3, 40)))
        off = rng.integers(0, int(spread), n, dtype=np.uint64)
        return np.minimum(centres[rng.integers(0, 4, n)] + off, np.uint64(KEY_END - 1))
    if kind == "duplicates":
        vals = rng.integers(0, KEY_END, 5, dtype=np.uint64)
        return vals[rng.integers(0, 5, n)]
    raise ValueError(kind)


def brute_counts(P, K):
    P = np.asarray(P, np.uint64)
    return np.array([np.count_nonzero((P >= np.uint64(K[i])) & (P < np.uint64(K[i + 1]))) for i in range(len(K) - 1)])


def ancestors(K):
    """All internal nodes (start, size) implied by a cornerstone array."""
    out = set()
    for i in range(len(K) - 1):
        size = int(K[i + 1]) - int(K[i])
        s = size * 8
        while s <= KEY_END:
            out.add(((int(K[i]) // s) * s, s))
            s *= 8
    return out


# ------------------------------------------------------------------ sort (Sec. 4, Table 1)
def test_sort_matches_library_stable_sort(oracle):
    rng = np.random.default_rng(10)
    for kind in ("uniform", "clustered", "duplicates"):
        k = random_keys(rng, 3000, kind)
        s, p = oracle.sort(k)
        ref = np.argsort(k, kind="stable")
        assert np.array_equal(p, ref.astype(np.uint32))
        assert np.array_equal(s, k[ref])


def test_sort_ties_keep_input_order(oracle):
    k = np.array([5, 3, 5, 3, 5, 1], np.uint64)
    s, p = oracle.sort(k)
    assert list(s) == [1, 3, 3, 5, 5, 5]
    assert list(p) == [5, 1, 3, 0, 2, 4]
    s, p = oracle.sort(np.array([], np.uint64))
    assert s.size == 0 and p.size == 0


# ------------------------------------------------------------------ f, g1, g2, g3 (Eqs. histogram, g1-g3)
def test_histogram_matches_brute_force(oracle):
    rng = np.random.default_rng(11)
    for kind in ("uniform", "clustered", "duplicates"):
        P = np.sort(random_keys(rng, 2000, kind))
        K = oracle.canonical_leaves(P, 16)
        assert np.array_equal(oracle.histogram(P, K), brute_counts(P, K))


def test_single_split_step(oracle):
    # root with Ncrit + 1 particles: O = {8, 0}, O' = {0, 8}, K' = the 8 root octants (Eq. rebalancesplit)
    K = np.array([0, KEY_END], np.uint64)
    O = oracle.rebalance_decision(K, np.array([5], np.uint32), 4)
    assert list(O) == [8, 0]
    Op = oracle.exclusive_scan(O)
    assert list(Op) == [0, 8]
    assert list(oracle.rebalance(K, O, Op)) == [c * 8 ** 20 for c in range(8)] + [KEY_END]


def test_merge_step_and_first_octant_kept(oracle):
    # 8 sibling leaves with a combined count <= Ncrit: octants 1..7 are removed (O = 0), the first
    # octant stays (O = 1) and becomes the parent's key (Eq. g1 conditions, Eq. rebalancecopy)
    K = np.array([c * 8 ** 20 for c in range(8)] + [KEY_END], np.uint64)
    N = np.array([1, 0, 2, 0, 0, 1, 0, 0], np.uint32)
    O = oracle.rebalance_decision(K, N, 4)
    assert list(O) == [1, 0, 0, 0, 0, 0, 0, 0, 0]
    assert list(oracle.rebalance(K, O, oracle.exclusive_scan(O))) == [0, KEY_END]
    # one more particle: the group no longer merges
    N[3] = 1
    assert list(oracle.rebalance_decision(K, N, 4)) == [1] * 8 + [0]


def test_merge_needs_all_siblings_as_leaves(oracle):
    # octant 0 of the root is split, so octants 1..7 are not 8 consecutive sibling leaves
    K = np.array([c * 8 ** 19 for c in range(8)] + [c * 8 ** 20 for c in range(1, 8)] + [KEY_END], np.uint64)
    N = np.zeros(len(K) - 1, np.uint32)
    O = oracle.rebalance_decision(K, N, 4)
    # the children of octant 0 merge (first kept), the level-1 octants stay
    assert list(O[:8]) == [1, 0, 0, 0, 0, 0, 0, 0]
    assert list(O[8:15]) == [1] * 7


def test_merge_rule_reading_is_less_or_equal(oracle):
    # A group whose combined count equals Ncrit merges: with it, a warm start reaches the same tree
    # as a cold start (the root holds exactly Ncrit particles and is therefore a leaf).
    P = np.sort(np.array([c * 8 ** 20 + 5 for c in range(8)], np.uint64))
    cold, _, _ = oracle.build_leaves(P, 8)
    assert list(cold) == [0, KEY_END]
    K_top = np.array([c * 8 ** 20 for c in range(8)] + [KEY_END], np.uint64)
    warm, _, _ = oracle.build_leaves(P, 8, K_init=K_top)
    assert list(warm) == [0, KEY_END]


def test_full_depth_leaf_is_not_split(oracle):
    # more than Ncrit identical keys: the tree descends to level L and stops there
    P = np.full(5, 12345, np.uint64)
    K, N, iters = oracle.build_leaves(P, 1)
    i = int(np.searchsorted(K, 12345, side="right")) - 1
    assert int(K[i + 1]) - int(K[i]) == 1 and N[i] == 5
    assert iters == L + 1  # L splitting passes plus the pass that finds nothing to change (Sec. 4)


# ------------------------------------------------------------------ worked example (Fig. 1)
def test_worked_example_fig1(oracle):
    g = golden()
    # particles: 2 in each level-1 octant except the third, 2 in each child of the third octant
    pts = [c * 8 ** 20 + 3 for c in range(8) if c != 2 for _ in range(2)]
    pts += [2 * 8 ** 20 + c * 8 ** 19 + 7 for c in range(8) for _ in range(2)]
    P = np.sort(np.array(pts, np.uint64))
    K_top = np.array(g["K_top"], np.uint64)
    # one f/g step on the top panel gives the lower panel
    N = oracle.histogram(P, K_top)
    O = oracle.rebalance_decision(K_top, N, 4)
    assert list(O) == [1, 1, 8, 1, 1, 1, 1, 1, 0]
    assert list(oracle.rebalance(K_top, O, oracle.exclusive_scan(O))) == g["K_refined"]
    # from the root the iteration needs 3 passes: split root, split third octant, confirm
    K, N, iters = oracle.build_leaves(P, 4)
    assert list(K) == g["K_refined"] and iters == 3
    assert list(N) == [2, 2] + [2] * 8 + [2] * 5


# ------------------------------------------------------------------ invariants, balance, uniqueness
CASES = [(kind, n, ncrit) for kind in ("uniform", "clustered", "duplicates")
         for n in (0, 1, 7, 64, 513, 3000) for ncrit in (1, 3, 16, 64)]


@pytest.mark.parametrize("kind,n,ncrit", CASES)
def test_iteration_reaches_balanced_unique_tree(oracle, kind, n, ncrit):
    rng = np.random.default_rng(hash((kind, n, ncrit)) % 2 ** 32)
    P = np.sort(random_keys(rng, n, kind)) if n else np.zeros(0, np.uint64)
    K, N, iters = oracle.build_leaves(P, ncrit)
    assert oracle.check_cornerstone(K)  # Eq. cstone
    assert iters <= L + 1
    assert np.array_equal(N, brute_counts(P, K))
    sizes = np.diff(K.astype(object))
    for i in range(len(N)):  # leaves hold <= Ncrit unless they are single keys at depth L
        assert N[i] <= ncrit or sizes[i] == 1
    for start, size in ancestors(K):  # internal nodes hold more than Ncrit
        cnt = np.count_nonzero((P >= np.uint64(start)) & (P < np.uint64(min(start + size, KEY_END))))
        if start + size >= KEY_END:
            cnt = np.count_nonzero(P >= np.uint64(start))
        assert cnt > ncrit
    assert np.array_equal(K, oracle.canonical_leaves(P, ncrit))


@pytest.mark.parametrize("seed", range(12))
def test_warm_start_converges_to_cold_tree(oracle, seed):
    # Sec. 4: rebuilding from the previous step's array reaches the same balanced tree
    rng = np.random.default_rng(100 + seed)
    kind = ("uniform", "clustered", "duplicates")[seed % 3]
    ncrit = (1, 4, 16, 32)[seed % 4]
    P0 = np.sort(random_keys(rng, 2000, kind))
    P1 = np.sort(random_keys(rng, 1500, kind))
    K0, _, _ = oracle.build_leaves(P0, ncrit)
    warm, _, it_w = oracle.build_leaves(P1, ncrit, K_init=K0)
    cold, _, it_c = oracle.build_leaves(P1, ncrit)
    assert np.array_equal(warm, cold)
    assert it_w <= L + 2 and it_c <= L + 1
    # an array that is already balanced needs exactly one confirming pass
    again, _, it = oracle.build_leaves(P1, ncrit, K_init=cold)
    assert np.array_equal(again, cold) and it == 1


def test_cornerstone_checker_rejects_bad_arrays(oracle):
    good = np.array([0, 8 ** 20, 2 * 8 ** 20] + [c * 8 ** 20 for c in range(3, 8)] + [KEY_END], np.uint64)
    assert oracle.check_cornerstone(good)
    assert not oracle.check_cornerstone(np.array([0, 3, KEY_END], np.uint64))  # gap not a power of 8
    assert not oracle.check_cornerstone(np.array([1, KEY_END], np.uint64))  # K_0 != 0
    bad = good.copy()
    bad[1], bad[2] = bad[2], bad[1]
    assert not oracle.check_cornerstone(bad)  # not increasing
