"""GPU parity of the batched builds: many independent sets stored back to back, one launch per
phase for all sets. Every set's result must equal the oracle's single-set build of that set."""
import numpy as np
import pytest
import torch

from _gpu_util import dev, i32, u32, u64

pytestmark = pytest.mark.gpu

KEY_END = 1 << 63


def _sets(sizes, seed):
    from paper_2307_06345_gb300 import workloads as w
    xs, ys, zs, kinds = [], [], [], []
    for i, n in enumerate(sizes):
        if i % 2 == 0:
            x, y, z = w.uniform(int(n), seed + i)
            kinds.append("uniform")
        else:
            x, y, z = w.plummer(int(n), seed + i)
            kinds.append("plummer")
        xs.append(x), ys.append(y), zs.append(z)
    off = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
    return np.concatenate(xs), np.concatenate(ys), np.concatenate(zs), off, kinds


def test_segmented_sort_bit_exact(lib, oracle):
    rng = np.random.default_rng(1)
    sizes = [0, 1, 4095, 4096, 4097, 10_000, 0, 3, 70_001, 1]
    keys = [rng.integers(0, 1 << 63, n, dtype=np.uint64) for n in sizes]
    keys[5][: 5000] = keys[5][0]  # many equal keys inside one segment
    k = np.concatenate(keys)
    off = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
    kin = dev(k)
    kout = torch.empty_like(kin)
    perm = torch.empty(k.size, dtype=torch.int32, device="cuda")
    ws = lib.Workspace()
    lib.cstone_sort_segmented(kin, kout, perm, dev(off), ws)
    assert ws.status() == 0
    ko, po = u64(kout), u32(perm)
    for s in range(len(sizes)):
        a, b = off[s], off[s + 1]
        ref_k, ref_p = oracle.sort(k[a:b])
        assert np.array_equal(ko[a:b], ref_k)
        assert np.array_equal(po[a:b].astype(np.int64) - a, ref_p.astype(np.int64))


def test_batched_bbox_and_keys(lib, oracle):
    sizes = [1000, 1, 5003, 0, 777, 20_000]
    x, y, z, off, kinds = _sets(sizes, 40)
    boxes = torch.empty((len(sizes), 4), dtype=torch.float64, device="cuda")
    lib.cstone_bbox_batched(dev(x), dev(y), dev(z), dev(off), boxes)
    bx = boxes.cpu().numpy()
    for s in range(len(sizes)):
        a, b = off[s], off[s + 1]
        assert np.array_equal(bx[s], oracle.bounding_cube(x[a:b], y[a:b], z[a:b]))
    for curve in (0, 1):
        keys = torch.empty(x.size, dtype=torch.int64, device="cuda")
        lib.cstone_keys_batched(dev(x), dev(y), dev(z), dev(off), boxes, curve, keys, lib.Workspace())
        kk = u64(keys)
        for s in range(len(sizes)):
            a, b = off[s], off[s + 1]
            assert np.array_equal(kk[a:b], oracle.keys(x[a:b], y[a:b], z[a:b], bx[s], curve))


def _check_batched_against_oracle(out, x, y, z, off, curve, ncrit, oracle, sets=None, boxes=None):
    eo = out["element_offsets_host"]
    no = out["node_offsets_host"]
    E = u64(out["elements"])
    N = u32(out["leaf_counts"])
    NK, CO, LO = u64(out["NK"]), i32(out["CO"]), i32(out["LO"])
    l2n = i32(out["leaf_to_node"])
    counts = u32(out["node_counts"])
    P, perm = u64(out["sorted_keys"]), u32(out["perm"])
    bx = out["boxes"].cpu().numpy() if boxes is None else boxes
    iters = []
    for s in (range(len(off) - 1) if sets is None else sets):
        a, b = off[s], off[s + 1]
        ref = oracle.full_build(x[a:b], y[a:b], z[a:b], curve, ncrit, box=bx[s])
        iters.append(ref["iters"])
        assert np.array_equal(P[a:b], ref["P"])
        assert np.array_equal(perm[a:b].astype(np.int64) - a, ref["perm"].astype(np.int64))
        assert np.array_equal(E[eo[s]: eo[s + 1]], ref["K"])
        assert np.array_equal(N[eo[s]: eo[s + 1] - 1], ref["N"])
        base = no[s]
        assert np.array_equal(NK[base: no[s + 1]], ref["NK"])
        co = CO[base: no[s + 1]]
        assert np.array_equal(np.where(co > 0, co - base, 0), ref["CO"])
        assert np.array_equal(LO[s] - base, ref["LO"])
        assert np.array_equal(l2n[eo[s]: eo[s + 1] - 1] - base, ref["leaf_to_node"])
        assert l2n[eo[s + 1] - 1] == -1
        assert np.array_equal(counts[base: no[s + 1]], ref["counts"])
    return iters


@pytest.mark.parametrize("curve", [0, 1])
def test_batched_build_small_sets(lib, oracle, curve):
    rng = np.random.default_rng(7 + curve)
    sizes = np.floor(2.0 ** rng.uniform(4, 14, 40)).astype(np.int64)
    sizes[3] = 0  # an empty set has a single empty leaf
    x, y, z, off, kinds = _sets(sizes, 500)
    out = lib.build_octrees_batched(dev(x), dev(y), dev(z), dev(off), curve=curve, ncrit=16)
    torch.cuda.synchronize()
    assert out["ws"].status() == 0
    iters = _check_batched_against_oracle(out, x, y, z, off, curve, 16, oracle)
    assert out["iters"] == max(iters)


def test_batched_warm_start(lib, oracle):
    from paper_2307_06345_gb300 import workloads as w
    rng = np.random.default_rng(3)
    sizes = np.floor(2.0 ** rng.uniform(8, 14, 12)).astype(np.int64)
    x, y, z, off, kinds = _sets(sizes, 900)
    first = lib.build_octrees_batched(dev(x), dev(y), dev(z), dev(off), curve=1, ncrit=8)
    boxes = first["boxes"]
    # move the particles and rebuild from the previous leaves with the same boxes
    dx, dy, dz = w.displacement(x.size, 901, 0.05)
    x2, y2, z2 = x + dx, y + dy, z + dz
    warm = lib.build_octrees_batched(dev(x2), dev(y2), dev(z2), dev(off), curve=1, ncrit=8, boxes=boxes, warm=first)
    torch.cuda.synchronize()
    _check_batched_against_oracle(warm, x2, y2, z2, off, 1, 8, oracle, boxes=boxes.cpu().numpy())


def test_batched_512_sets_sampled(lib, oracle):
    # the batched workload: 512 sets, sizes log-uniform in [2^10, 2^20), uniform (unit cube) or
    # Plummer (bounding cube), Morton keys, Ncrit 32; a sample of sets against the oracle
    from paper_2307_06345_gb300 import workloads as w
    sets = w.batched_sets(512, w.BASE_SEED + 3)
    sizes = np.array([len(s[0]) for s in sets], np.int64)
    off = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
    x = np.concatenate([s[0] for s in sets])
    y = np.concatenate([s[1] for s in sets])
    z = np.concatenate([s[2] for s in sets])
    boxes = torch.empty((512, 4), dtype=torch.float64, device="cuda")
    X, Y, Z, OFF = dev(x), dev(y), dev(z), dev(off)
    lib.cstone_bbox_batched(X, Y, Z, OFF, boxes)
    unit = torch.tensor([0.0, 0.0, 0.0, 1.0], dtype=torch.float64, device="cuda")
    for i, s in enumerate(sets):
        if s[3] == "uniform":
            boxes[i] = unit
    out = lib.build_octrees_batched(X, Y, Z, OFF, curve=0, ncrit=32, boxes=boxes)
    torch.cuda.synchronize()
    assert out["ws"].status() == 0
    rng = np.random.default_rng(5)
    pick = sorted(set(rng.choice(512, 10, replace=False).tolist()) | {int(np.argmax(sizes)), int(np.argmin(sizes))})
    _check_batched_against_oracle(out, x, y, z, off, 0, 32, oracle, sets=pick, boxes=boxes.cpu().numpy())


def test_one_call_batched_build_through_the_c_abi(lib, oracle):
    """cstone_build_batched called directly through ctypes (one C call for the whole batched build,
    then cstone_build_batched_result): cold from the roots with bounding cubes computed on the
    device, then warm-started in place after the particles moved; every set against the oracle."""
    import ctypes
    sizes = [5000, 0, 1, 12_345, 777, 40_000]
    x, y, z, off, kinds = _sets(sizes, 70)
    s, n = len(sizes), x.size
    X, Y, Z, OFF = dev(x), dev(y), dev(z), dev(off)
    cap = lib.batched_capacity(n, s, 16)
    bufs = lib.BatchBuffers.allocate(n, s, cap, "cuda")
    clib = lib.load()
    sz = ctypes.c_size_t()
    assert clib.cstone_build_batched_workspace_size(n, s, cap, 64, ctypes.byref(sz)) == lib.OK
    ws = torch.empty(sz.value, dtype=torch.uint8, device="cuda")
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    for step, warm in enumerate((0, 1)):
        if warm:  # small moves: the warm start needs few passes and reaches the same tree
            rng = np.random.default_rng(5)
            x, y, z = (c + 1e-4 * rng.standard_normal(c.size) for c in (x, y, z))
            X.copy_(dev(x)), Y.copy_(dev(y)), Z.copy_(dev(z))
        inp = lib._BatchInput(X.data_ptr(), Y.data_ptr(), Z.data_ptr(), n, OFF.data_ptr(), s, None)
        prm = lib._BatchParams(lib.MORTON, 16, 64, warm)
        out = bufs.c_struct()
        rc = clib.cstone_build_batched(ctypes.byref(inp), ctypes.byref(prm), ctypes.byref(out),
                                       ctypes.c_void_p(ws.data_ptr()), sz.value, stream)
        assert rc == lib.OK
        ne, nn, it = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int32()
        rc = clib.cstone_build_batched_result(ctypes.c_void_p(ws.data_ptr()), n, s, cap, 64,
                                              ctypes.c_void_p(bufs.t["LO"].data_ptr()), stream, ctypes.byref(ne),
                                              ctypes.byref(nn), ctypes.byref(it))
        assert rc == lib.OK
        res = lib._batched_result(bufs, ne.value, nn.value, it.value, None)
        bx = res["boxes"].cpu().numpy()
        if warm == 0:
            for q in range(s):
                a, b = off[q], off[q + 1]
                assert np.array_equal(bx[q], oracle.bounding_cube(x[a:b], y[a:b], z[a:b]))
        _check_batched_against_oracle(res, x, y, z, off, 0, 16, oracle, boxes=bx)
