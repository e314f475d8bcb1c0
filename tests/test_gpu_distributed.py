"""GPU parity of the separate f and g steps (cstone_leaf_counts, cstone_rebalance), the per-axis
bounds, and the global-tree protocol driven by them (Sec. 6). Several ranks are emulated on the one
GPU by summing the counts of disjoint particle subsets between f and g, with no collective and no
kernel waiting on another; the result must equal the oracle's build of the union."""
import numpy as np
import pytest
import torch

from _gpu_util import dev, u32, u64

pytestmark = pytest.mark.gpu


def _random_cornerstone(oracle, rng, n, ncrit, levels=21):
    keys = rng.integers(0, 1 << (3 * levels), n, dtype=np.uint64)
    P = np.sort(keys)
    K, _, _ = oracle.build_leaves(P, ncrit, levels=levels)
    return P, K


@pytest.mark.parametrize("levels", [21, 10])
def test_leaf_counts_and_rebalance_match_the_oracle(lib, oracle, levels):
    rng = np.random.default_rng(60 + levels)
    kdt = np.uint64 if levels == 21 else np.uint32
    for n, ncrit_tree, ncrit in [(5000, 64, 8), (20_000, 4, 64), (1, 1, 1), (3000, 16, 16)]:
        P, K = _random_cornerstone(oracle, rng, n, ncrit_tree, levels)
        nl = K.size - 1
        N = torch.empty(nl, dtype=torch.int32, device="cuda")
        lib.cstone_leaf_counts(dev(P.astype(kdt)), dev(K.astype(kdt)), nl, N, levels=levels)
        N_ref = oracle.histogram(P, K)
        assert np.array_equal(u32(N), N_ref)
        # g on these counts with another ncrit: splits and merges both occur
        out = torch.empty(8 * nl + 2, dtype=torch.int64 if levels == 21 else torch.int32, device="cuda")
        nl2, changed = lib.cstone_rebalance(dev(K.astype(kdt)), N, nl, ncrit, out, lib.Workspace(), levels=levels)
        O = oracle.rebalance_decision(K, N_ref, ncrit, levels=levels)
        K2 = oracle.rebalance(K, O, oracle.exclusive_scan(O), levels=levels)
        assert nl2 == K2.size - 1 and changed == bool((O[:nl] != 1).any())
        got = (u64(out) if levels == 21 else u32(out).astype(np.uint64))[: nl2 + 1]
        assert np.array_equal(got, K2)


def test_rebalance_capacity_error(lib, oracle):
    rng = np.random.default_rng(3)
    P, K = _random_cornerstone(oracle, rng, 4000, 64)
    nl = K.size - 1
    N = torch.full((nl,), 10_000, dtype=torch.int32, device="cuda")  # every leaf splits
    out = torch.empty(nl + 2, dtype=torch.int64, device="cuda")  # room for nl + 1 leaves only
    with pytest.raises(lib.CstoneError) as e:
        lib.cstone_rebalance(dev(K), N, nl, 16, out, lib.Workspace())
    assert e.value.status == lib.ERR_CAPACITY and e.value.required == 8 * nl


def test_bounds(lib, oracle):
    from paper_2307_06345_gb300 import workloads as w
    x, y, z = w.plummer(100_001, 5)
    b = torch.empty(6, dtype=torch.float64, device="cuda")
    lib.cstone_bounds(dev(x), dev(y), dev(z), b, lib.Workspace())
    assert b.cpu().tolist() == [x.min(), y.min(), z.min(), x.max(), y.max(), z.max()]
    e = torch.empty(0, dtype=torch.float64, device="cuda")
    lib.cstone_bounds(e, e, e, b, lib.Workspace())
    assert b.cpu().tolist() == [np.inf] * 3 + [-np.inf] * 3


@pytest.mark.parametrize("levels,curve,ncrit", [(21, 1, 64), (21, 0, 8), (10, 1, 16)])
def test_emulated_ranks_build_the_union_tree(lib, oracle, levels, curve, ncrit):
    from paper_2307_06345_gb300 import distributed as D
    from paper_2307_06345_gb300 import workloads as w
    x, y, z = w.clumps(200_000, 17, n_clumps=40)
    ranks = 3
    owner = np.random.default_rng(18).integers(0, ranks, x.size)
    ops = D.DeviceOps("cuda", levels)
    parts = [tuple(dev(np.ascontiguousarray(a[owner == r])) for a in (x, y, z)) for r in range(ranks)]
    # global box: min / max of the parts' bounds (what the allreduce does)
    bs = torch.stack([ops.bounds(*p) for p in parts])
    lo, hi = bs[:, :3].min(0).values.cpu().tolist(), bs[:, 3:].max(0).values.cpu().tolist()
    box = torch.tensor(lo + [max(h - l for l, h in zip(lo, hi))], dtype=torch.float64, device="cuda")
    ref_box = oracle.bounding_cube(x, y, z)
    assert np.array_equal(box.cpu().numpy(), ref_box)
    sorted_parts = [ops.sort(ops.keys(*p, box, curve))[0] for p in parts]
    K, nl, passes = ops.root(), 1, 0
    while True:  # f on every part, counts summed, the same g once
        passes += 1
        N = sum(ops.leaf_counts(P, K, nl) for P in sorted_parts)
        K2, nl2, changed = ops.rebalance(K, N, nl, ncrit)
        if not changed:
            break
        K, nl = K2, nl2
    ref = oracle.full_build(x, y, z, curve, ncrit, box=ref_box, levels=levels)
    got = u64(K) if levels == 21 else u32(K).astype(np.uint64)
    assert np.array_equal(got, ref["K"]) and np.array_equal(u32(N), ref["N"]) and passes == ref["iters"]
    # the single-rank driver (no process group) gives the same array
    t = D.build_global_tree(dev(x), dev(y), dev(z), curve=curve, ncrit=ncrit, levels=levels)
    got1 = u64(t["K"]) if levels == 21 else u32(t["K"]).astype(np.uint64)
    assert np.array_equal(got1, ref["K"]) and t["passes"] == ref["iters"]
    cuts = D.decompose(t["N_global"], 4)
    rx, ry, rz = D.exchange(ops, dev(x), dev(y), dev(z), t["P"], t["perm"], t["K"], cuts)
    assert np.array_equal(rx.cpu().numpy(), x[ref["perm"]])  # one rank: the particles in key order
