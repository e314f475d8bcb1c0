"""The oracle's parallel loops and chunked sorts give the sequential program's results.

Each parallel loop iteration does the sequential iteration's operations in the same order, and the
chunked sort merges qsorted chunks under a total order, so every output must be bit-identical for
any thread count. Pinned here against the single-threaded run and, for the sort, against numpy's
stable lexicographic sort (an independent implementation), at sizes that span several chunks."""
import numpy as np
import pytest


@pytest.fixture
def threads(oracle):
    yield oracle
    oracle.set_threads(0)


def test_sort_matches_numpy_lexsort_for_every_thread_count(threads):
    o = threads
    rng = np.random.default_rng(3)
    n = 100_003
    k = rng.integers(0, 1 << 63, n, dtype=np.uint64)
    k[rng.integers(0, n, n // 3)] = k[17]  # many ties: the index decides their order
    want = np.lexsort((np.arange(n), k))
    for t in (1, 2, 3, 8):
        o.set_threads(t)
        P, perm = o.sort(k)
        assert np.array_equal(perm, want.astype(np.uint32)), t
        assert np.array_equal(P, k[want]), t


def test_full_build_and_multipoles_independent_of_threads(threads):
    from paper_2307_06345_gb300 import workloads as w
    o = threads
    n = 1 << 17
    x, y, z = w.clumps(n, 77)
    m = w.lognormal_masses(n, 78)
    res = []
    for t in (1, 5):
        o.set_threads(t)
        r = o.full_build(x, y, z, o.HILBERT, 16)
        r["M"], r["com"], r["quad"] = o.multipoles(x, y, z, m, r["P"], r["perm"], r["NK"])
        r["canon"] = o.canonical_leaves(r["P"], 16)
        res.append(r)
    for key, v in res[0].items():
        if isinstance(v, np.ndarray):
            assert np.array_equal(v, res[1][key]), key
    assert np.array_equal(res[0]["canon"], res[0]["K"])
