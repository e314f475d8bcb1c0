"""GPU parity of the time-step driver: several runs moved by small Gaussian displacements, every
step rebuilt from the previous step's leaves (warm start, Sec. 4) in a box fixed at step 0.

Every warm rebuild equals a cold rebuild of the same step (the balanced tree is unique), and
sampled runs and steps equal the oracle's build from the raw coordinates."""
import numpy as np
import pytest
import torch

from _gpu_util import dev, i32, u32, u64

pytestmark = pytest.mark.gpu

KEY_END = 1 << 63


def _equal(a, b, keys):
    for k in keys:
        assert torch.equal(a[k], b[k]), k


def test_time_steps_warm_equals_cold_and_oracle(lib, oracle):
    from paper_2307_06345_gb300 import workloads as w
    runs, n, steps = 8, 1 << 18, 6
    parts = [w.plummer(n, w.BASE_SEED + 4 + r) for r in range(runs)]
    x = np.concatenate([p[0] for p in parts])
    y = np.concatenate([p[1] for p in parts])
    z = np.concatenate([p[2] for p in parts])
    off = (np.arange(runs + 1) * n).astype(np.int64)
    X, Y, Z, OFF = dev(x), dev(y), dev(z), dev(off)
    st = lib.TimeStepper(X, Y, Z, OFF, curve=lib.HILBERT, ncrit=64)
    boxes = st.boxes.cpu().numpy()
    side0 = float(boxes[0, 3]) / 1.2
    for step in range(steps):
        if step > 0:
            dx, dy, dz = w.displacement(x.size, w.BASE_SEED + 100 + step, 1e-3 * side0)
            x, y, z = x + dx, y + dy, z + dz
            X.copy_(dev(x)), Y.copy_(dev(y)), Z.copy_(dev(z))
        warm = st.rebuild(warm=step > 0)
        cold = lib.build_octrees_batched(X, Y, Z, OFF, curve=lib.HILBERT, ncrit=64, boxes=st.boxes)
        torch.cuda.synchronize()
        _equal(warm, cold, ["elements", "element_offsets", "leaf_counts", "NK", "CO", "LO", "node_counts"])
        if step > 0:
            assert warm["iters"] <= 4  # a slowly moving distribution needs few passes
        check = range(runs) if step in (0, steps - 1) else [0]
        eo, no = warm["element_offsets_host"], warm["node_offsets_host"]
        E, NK, counts = u64(warm["elements"]), u64(warm["NK"]), u32(warm["node_counts"])
        for r in check:
            a, b = off[r], off[r + 1]
            lo = boxes[r, :3]
            inside = np.all((np.stack([x[a:b], y[a:b], z[a:b]]) >= lo[:, None]) &
                            (np.stack([x[a:b], y[a:b], z[a:b]]) < lo[:, None] + boxes[r, 3]))
            assert inside  # the padded box still holds every particle: nothing is clamped
            ref = oracle.full_build(x[a:b], y[a:b], z[a:b], oracle.HILBERT, 64, box=boxes[r])
            assert np.array_equal(E[eo[r]: eo[r + 1]], ref["K"])
            assert np.array_equal(NK[no[r]: no[r + 1]], ref["NK"])
            assert np.array_equal(counts[no[r]: no[r + 1]], ref["counts"])


def test_graph_time_steps_equal_eager_and_oracle(lib, oracle):
    # the whole rebuild replayed as one CUDA graph per step gives the eager driver's trees
    from paper_2307_06345_gb300 import workloads as w
    runs, n, steps = 4, 1 << 16, 5
    parts = [w.plummer(n, w.BASE_SEED + 40 + r) for r in range(runs)]
    x = np.concatenate([p[0] for p in parts])
    y = np.concatenate([p[1] for p in parts])
    z = np.concatenate([p[2] for p in parts])
    off = (np.arange(runs + 1) * n).astype(np.int64)
    X, Y, Z, OFF = dev(x), dev(y), dev(z), dev(off)
    g = lib.GraphTimeStepper(X, Y, Z, OFF, curve=lib.HILBERT, ncrit=32)
    e = lib.TimeStepper(X, Y, Z, OFF, curve=lib.HILBERT, ncrit=32)
    assert torch.equal(g.boxes, e.boxes)
    boxes = g.boxes.cpu().numpy()
    side0 = float(boxes[0, 3]) / 1.2
    for step in range(steps):
        if step > 0:
            dx, dy, dz = w.displacement(x.size, w.BASE_SEED + 140 + step, 2e-3 * side0)
            x, y, z = x + dx, y + dy, z + dz
            X.copy_(dev(x)), Y.copy_(dev(y)), Z.copy_(dev(z))
        a = g.rebuild(warm=step > 0)
        b = e.rebuild(warm=step > 0)
        torch.cuda.synchronize()
        _equal(a, b, ["sorted_keys", "perm", "elements", "element_offsets", "leaf_counts", "NK", "CO", "LO",
                      "leaf_to_node", "node_counts"])
        assert a["node_offsets_host"] == b["node_offsets_host"]
        if step == steps - 1:
            assert g.graph is not None  # warm steps were replayed from the graph
            eo, no = a["element_offsets_host"], a["node_offsets_host"]
            E, NK, counts = u64(a["elements"]), u64(a["NK"]), u32(a["node_counts"])
            for r in range(runs):
                ra, rb = off[r], off[r + 1]
                ref = oracle.full_build(x[ra:rb], y[ra:rb], z[ra:rb], oracle.HILBERT, 32, box=boxes[r])
                assert np.array_equal(E[eo[r]: eo[r + 1]], ref["K"])
                assert np.array_equal(NK[no[r]: no[r + 1]], ref["NK"])
                assert np.array_equal(counts[no[r]: no[r + 1]], ref["counts"])


@pytest.mark.parametrize("failure", ["capacity", "not_converged"])
def test_async_leaves_failure_leaves_root_arrays(lib, failure):
    # a failed asynchronous leaf loop reports its status afterwards and leaves every set's root
    # array, so that the phases queued after it run within their buffers
    from paper_2307_06345_gb300 import workloads as w
    sizes = [5000, 3000, 0, 7000]
    xs = [w.uniform(k, w.BASE_SEED + 60 + i) for i, k in enumerate(sizes)]
    x, y, z = (np.concatenate([p[d] for p in xs]) for d in range(3))
    off = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
    X, Y, Z, OFF = dev(x), dev(y), dev(z), dev(off)
    s = len(sizes)
    boxes = torch.tensor([[0.0, 0.0, 0.0, 1.0]] * s, dtype=torch.float64, device="cuda")
    ws = lib.Workspace()
    keys = torch.empty(x.size, dtype=torch.int64, device="cuda")
    lib.cstone_keys_batched(X, Y, Z, OFF, boxes, lib.MORTON, keys, ws)
    sk, perm = torch.empty_like(keys), torch.empty(x.size, dtype=torch.int32, device="cuda")
    lib.cstone_sort_segmented(keys, sk, perm, OFF, ws)
    cap, iters = (2 * s + 8, 64) if failure == "capacity" else (4096, 2)
    elements = torch.empty(cap, dtype=torch.int64, device="cuda")
    eo = torch.empty(s + 1, dtype=torch.int64, device="cuda")
    counts = torch.empty(cap, dtype=torch.int32, device="cuda")
    lws = lib.Workspace()
    lib.cstone_build_leaves_batched_async(sk, OFF, 8, elements, eo, counts, None, False, iters, lws)
    node_cap = cap + cap // 7 + s
    NK = torch.empty(node_cap, dtype=torch.int64, device="cuda")
    CO = torch.empty(node_cap, dtype=torch.int32, device="cuda")
    LO = torch.empty((s, 23), dtype=torch.int32, device="cuda")
    l2n = torch.empty(cap, dtype=torch.int32, device="cuda")
    nc = torch.empty(node_cap, dtype=torch.int32, device="cuda")
    kws, cws = lib.Workspace(), lib.Workspace()
    lib.cstone_link_tree_batched(elements, cap, eo, node_cap, NK, CO, LO, l2n, kws)
    lib.cstone_upsweep_counts_batched(counts, cap, l2n, CO, LO, s, nc, cws)
    with pytest.raises(lib.CstoneError) as ei:
        lib.cstone_leaves_result(lws, cap, iters)
    assert ei.value.status == (lib.ERR_CAPACITY if failure == "capacity" else lib.ERR_NOT_CONVERGED)
    if failure == "capacity":
        assert ei.value.required > cap
    assert kws.status() == 0 and cws.status() == 0
    assert u64(eo).tolist() == [2 * q for q in range(s + 1)]
    E = u64(elements[: 2 * s])
    assert E[0::2].tolist() == [0] * s and E[1::2].tolist() == [KEY_END] * s
    assert u32(counts[: 2 * s])[0::2].tolist() == sizes
    assert u32(nc[:s]).tolist() == sizes  # one root node per set, holding the whole set


def test_async_leaves_equal_sync(lib, oracle):
    from paper_2307_06345_gb300 import workloads as w
    sizes = [20_000, 1, 0, 33_333, 4096]
    xs = [w.plummer(k, w.BASE_SEED + 70 + i) for i, k in enumerate(sizes)]
    x, y, z = (np.concatenate([p[d] for p in xs]) for d in range(3))
    off = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
    X, Y, Z, OFF = dev(x), dev(y), dev(z), dev(off)
    ref = lib.build_octrees_batched(X, Y, Z, OFF, curve=lib.HILBERT, ncrit=16)
    cap = 1 << 16  # room for the intermediate arrays of the loop, not only the result
    elements = torch.empty(cap, dtype=torch.int64, device="cuda")
    eo = torch.empty(len(sizes) + 1, dtype=torch.int64, device="cuda")
    counts = torch.empty(cap, dtype=torch.int32, device="cuda")
    ws = lib.Workspace()
    for warm in (False, True):  # cold, then warm from its own (converged) output
        lib.cstone_build_leaves_batched_async(ref["sorted_keys"], OFF, 16, elements, eo, counts, None, warm, 64, ws)
        ne, iters = lib.cstone_leaves_result(ws, cap, 64)
        assert ne == ref["n_elements"]
        assert torch.equal(elements[:ne], ref["elements"]) and torch.equal(eo, ref["element_offsets"])
        assert torch.equal(counts[:ne], ref["leaf_counts"])
        if warm:
            assert iters == 1


def test_graph_time_stepper_capacity_floor(lib):
    # a requested capacity below the batched builder's estimate is raised to it, so the cold build
    # fits; later steps replay the graph at that capacity
    from paper_2307_06345_gb300 import workloads as w
    runs, n = 3, 20_000
    parts = [w.uniform(n, w.BASE_SEED + 80 + r) for r in range(runs)]
    X, Y, Z = (dev(np.concatenate([p[d] for p in parts])) for d in range(3))
    OFF = dev((np.arange(runs + 1) * n).astype(np.int64))
    g = lib.GraphTimeStepper(X, Y, Z, OFF, curve=lib.MORTON, ncrit=16, elem_cap=2 * runs + 8)
    assert g.elem_cap == g.min_cap > 2 * runs + 8
    e = lib.TimeStepper(X, Y, Z, OFF, curve=lib.MORTON, ncrit=16)
    for warm in (False, True, True):
        a, b = g.rebuild(warm=warm), e.rebuild(warm=warm)
        torch.cuda.synchronize()
        _equal(a, b, ["elements", "element_offsets", "leaf_counts", "NK", "CO", "LO", "node_counts"])
    assert g.elem_cap == g.min_cap and g.graph is not None


def _oracle_box(oracle, x, y, z, pad=0.1):
    """The step-0 bounding cube of a run grown by `pad` of its side on every side, from the
    oracle's bounding cube (the same two IEEE operations per component as the stepper's)."""
    b = oracle.bounding_cube(x, y, z)
    out = b.copy()
    out[:3] = b[:3] - pad * b[3]
    out[3] = b[3] * (1.0 + 2.0 * pad)
    return out


def test_time_steps_8x2p26_full_size_spot_checks(lib, oracle):
    """The time-step workload at its full size, in the launch configuration bench.py times: 8 runs of
    2^26 Plummer particles, 100 steps of Gaussian displacements of 1e-3 of the box (drawn on the
    device), Hilbert keys, Ncrit 64, every rebuild one CUDA graph replay warm-started from the
    previous step's leaves. Every step's warm rebuild equals a cold rebuild of the same
    coordinates (the balanced tree is unique, Sec. 4); run 0 at steps 0, 1, 50 and 99 and every run
    at step 99 equal the oracle's build from the raw coordinates (sorted keys, permutation, leaves,
    leaf counts, NK, CO, LO, node counts)."""
    from paper_2307_06345_gb300 import workloads as w
    runs, n, steps = 8, 1 << 26, 100
    oracle.set_threads(0)
    d = torch.device("cuda")
    parts = [w.plummer_device(n, w.BASE_SEED + 5 + r, d) for r in range(runs)]
    X, Y, Z = (torch.cat([p[k] for p in parts]) for k in range(3))
    del parts
    OFF = torch.arange(runs + 1, dtype=torch.int64, device=d) * n
    st = lib.GraphTimeStepper(X, Y, Z, OFF, curve=lib.HILBERT, ncrit=64)
    boxes = st.boxes.cpu().numpy()
    for r in range(runs):
        sl = slice(r * n, (r + 1) * n)
        assert np.array_equal(boxes[r], _oracle_box(oracle, X[sl].cpu().numpy(), Y[sl].cpu().numpy(),
                                                    Z[sl].cpu().numpy()))
    sigma = 1e-3 * float(boxes[0, 3]) / 1.2
    g = torch.Generator(device=d)
    g.manual_seed(w.BASE_SEED + 6)
    ws = lib.Workspace()
    keys = ["elements", "element_offsets", "leaf_counts", "NK", "CO", "LO", "node_counts"]
    for step in range(steps):
        if step > 0:
            for c in (X, Y, Z):
                c.add_(torch.randn(c.shape, dtype=torch.float64, device=d, generator=g), alpha=sigma)
        warm = st.rebuild(warm=step > 0)
        cold = lib.build_octrees_batched(X, Y, Z, OFF, curve=lib.HILBERT, ncrit=64, boxes=st.boxes, ws=ws)
        torch.cuda.synchronize()
        _equal(warm, cold, keys)
        if step > 1:
            assert warm["iters"] <= 4  # a slowly moving distribution needs few passes
        check = range(runs) if step == steps - 1 else ([0] if step in (0, 1, 50) else [])
        if not check:
            continue
        eo, no = warm["element_offsets_host"], warm["node_offsets_host"]
        E, NK, CO, counts = u64(warm["elements"]), u64(warm["NK"]), i32(warm["CO"]), u32(warm["node_counts"])
        LC, SK, PERM = u32(warm["leaf_counts"]), u64(warm["sorted_keys"]), u32(warm["perm"])
        LO = i32(warm["LO"])
        for r in check:
            sl = slice(r * n, (r + 1) * n)
            x, y, z = X[sl].cpu().numpy(), Y[sl].cpu().numpy(), Z[sl].cpu().numpy()
            lo, side = boxes[r, :3], boxes[r, 3]
            assert all(((c >= lo[k]) & (c < lo[k] + side)).all() for k, c in enumerate((x, y, z)))  # no clamping
            ref = oracle.full_build(x, y, z, oracle.HILBERT, 64, box=boxes[r])
            assert np.array_equal(SK[sl], ref["P"])
            assert np.array_equal(PERM[sl].astype(np.int64) - r * n, ref["perm"].astype(np.int64))
            assert np.array_equal(E[eo[r]: eo[r + 1]], ref["K"])
            assert np.array_equal(LC[eo[r]: eo[r + 1] - 1], ref["N"])
            assert np.array_equal(NK[no[r]: no[r + 1]], ref["NK"])
            assert np.array_equal(CO[no[r]: no[r + 1]] - np.where(CO[no[r]: no[r + 1]] > 0, no[r], 0), ref["CO"])
            assert np.array_equal(LO[r] - no[r], ref["LO"])
            assert np.array_equal(counts[no[r]: no[r + 1]], ref["counts"])
        del E, NK, CO, counts, LC, SK, PERM
