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
    cuts = D.decompose(ops, t["N_global"], 4)
    rx, ry, rz = D.exchange(ops, dev(x), dev(y), dev(z), t["P"], t["perm"], t["K"], cuts)
    assert np.array_equal(rx.cpu().numpy(), x[ref["perm"]])  # one rank: the particles in key order


@pytest.mark.parametrize("world", [1, 2, 3, 8, 97])
def test_decompose_kernel_matches_oracle(lib, oracle, world):
    """cstone_decompose through the C ABI against the oracle's cuts (Sec. 6), on leaf counts of the
    clump workload's balanced tree and on counts with long runs of empty leaves."""
    import ctypes
    from paper_2307_06345_gb300 import workloads as w
    x, y, z = w.clumps(400_000, w.BASE_SEED + 90, n_clumps=30)
    ref = oracle.full_build(x, y, z, oracle.HILBERT, 16)
    rng = np.random.default_rng(world)
    sparse = rng.integers(0, 50, 200_003).astype(np.uint32)
    sparse[rng.random(sparse.size) < 0.9] = 0
    clib = lib.load()
    for N in (ref["N"], sparse, np.zeros(5000, np.uint32), np.zeros(0, np.uint32)):
        cuts = torch.full((world + 1,), -7, dtype=torch.int64, device="cuda")
        Nd = dev(N) if N.size else torch.zeros(1, dtype=torch.int32, device="cuda")
        sz = ctypes.c_size_t()
        assert clib.cstone_decompose_workspace_size(N.size, world, ctypes.byref(sz)) == lib.OK
        ws = torch.empty(sz.value, dtype=torch.uint8, device="cuda")
        rc = clib.cstone_decompose(ctypes.c_void_p(Nd.data_ptr()), N.size, world, ctypes.c_void_p(cuts.data_ptr()),
                                   ctypes.c_void_p(ws.data_ptr()), sz.value,
                                   ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
        assert rc == lib.OK
        torch.cuda.synchronize()
        assert cuts.cpu().tolist() == oracle.decompose(N, world).tolist()


def test_cube_from_bounds_kernel_matches_oracle(lib, oracle):
    """cstone_cube_from_bounds on bounds reduced over three parts equals the oracle's cube of the
    same bounds and the bounding cube of the union; no points give the unit cube at the origin."""
    from paper_2307_06345_gb300 import workloads as w
    parts = [w.plummer(20_000 + 5000 * k, w.BASE_SEED + 91 + k) for k in range(3)]
    ws = lib.Workspace()
    lo, hi = [], []
    for p in parts:
        b = torch.empty(6, dtype=torch.float64, device="cuda")
        lib.cstone_bounds(dev(p[0]), dev(p[1]), dev(p[2]), b, ws)
        lo.append(b[:3])
        hi.append(b[3:])
    bounds = torch.cat([torch.stack(lo).min(0).values, torch.stack(hi).max(0).values])
    box = torch.empty(4, dtype=torch.float64, device="cuda")
    lib.cstone_cube_from_bounds(bounds, box)
    torch.cuda.synchronize()
    union = [np.concatenate([p[d] for p in parts]) for d in range(3)]
    assert np.array_equal(box.cpu().numpy(), oracle.cube_from_bounds(bounds.cpu().numpy()))
    assert np.array_equal(box.cpu().numpy(), oracle.bounding_cube(*union))
    empty = torch.tensor([np.inf] * 3 + [-np.inf] * 3, dtype=torch.float64, device="cuda")
    lib.cstone_cube_from_bounds(empty, box)
    assert box.cpu().tolist() == [0.0, 0.0, 0.0, 1.0]
