"""GPU parity of the locally essential (focused) tree of Sec. 7 on one process: one g1^LE-g3
pass (cstone_rebalance_focus) against the oracle's decision, scan and rebalance, and the whole
focused build (f and g^LE until nothing changes) against the oracle's literal iteration, for both
curves and both key lengths."""
import numpy as np
import pytest
import torch

from _gpu_util import dev, u32, u64

pytestmark = pytest.mark.gpu


def _tree_and_keys(oracle, rng, n, ncrit, curve, levels):
    from paper_2307_06345_gb300 import workloads as w
    x, y, z = w.clumps(n, int(rng.integers(0, 1 << 30)), n_clumps=25)
    box = oracle.bounding_cube(x, y, z)
    P, _ = oracle.sort(oracle.keys(x, y, z, box, curve, levels=levels))
    K = oracle.canonical_leaves(P, ncrit, levels=levels)
    return P, K


def _dev_keys(a, levels):
    return dev(np.asarray(a, np.uint64).astype(np.uint64 if levels == 21 else np.uint32))


def _host_keys(t, levels):
    return u64(t) if levels == 21 else u32(t).astype(np.uint64)


@pytest.mark.parametrize("levels", [21, 10])
@pytest.mark.parametrize("curve", [0, 1])
def test_one_focused_pass_matches_the_oracle(lib, oracle, levels, curve):
    rng = np.random.default_rng(100 + levels + curve)
    for trial in range(6):
        P, K = _tree_and_keys(oracle, rng, 20_000, (4, 16, 64)[trial % 3], curve, levels)
        nl = K.size - 1
        N = oracle.histogram(P, K)
        a, b = sorted(rng.integers(0, nl + 1, 2))
        f = (int(K[a]), int(K[b]))  # focus on a run of leaves (empty when a == b)
        theta = float((0.35, 0.7, 1.2)[trial % 3])
        ncrit = (8, 32, 2)[trial % 3]
        out = torch.empty(8 * nl + 2, dtype=torch.int64 if levels == 21 else torch.int32, device="cuda")
        nl2, changed = lib.cstone_rebalance_focus(_dev_keys(K, levels), dev(N), nl, ncrit, *f, theta, curve, out,
                                                  lib.Workspace(), levels=levels)
        O = oracle.focus_decision(K, N, ncrit, *f, theta, curve, levels=levels)
        K2 = oracle.rebalance(K, O, oracle.exclusive_scan(O), levels=levels)
        assert nl2 == K2.size - 1 and changed == bool((O[:nl] != 1).any())
        assert np.array_equal(_host_keys(out, levels)[: nl2 + 1], K2)


@pytest.mark.parametrize("levels", [21, 10])
@pytest.mark.parametrize("curve", [0, 1])
def test_focused_build_matches_the_oracle(lib, oracle, levels, curve):
    rng = np.random.default_rng(200 + levels + curve)
    P, Kg = _tree_and_keys(oracle, rng, 200_000, 32, curve, levels)
    Pd = _dev_keys(P, levels)
    for trial in range(3):
        a, b = sorted(rng.integers(0, P.size, 2))
        f = (int(P[a]), int(P[b]) + 1)
        theta = (0.4, 0.8, 1.5)[trial]
        K, N, passes = lib.build_focus_leaves(Pd, 32, *f, theta, curve, levels=levels)
        Kr, Nr, it = oracle.build_focus_leaves(P, 32, *f, theta, curve, levels=levels)
        assert np.array_equal(_host_keys(K, levels), Kr) and np.array_equal(u32(N), Nr) and passes == it
        # warm start from the balanced tree of all particles
        Kw, _, _ = lib.build_focus_leaves(Pd, 32, *f, theta, curve, warm_leaves=_dev_keys(Kg, levels),
                                          levels=levels)
        assert np.array_equal(_host_keys(Kw, levels), Kr)
    # a focus covering every key gives the balanced tree of the single-process build
    end = 1 << (3 * levels)
    K, _, _ = lib.build_focus_leaves(Pd, 32, 0, end, 0.5, curve, levels=levels)
    assert np.array_equal(_host_keys(K, levels), Kg)
