"""GPU tests of StreamedBuilder: full builds of host-resident sets with the transfers overlapped
with the builds must equal build_octree on device copies of the same sets, bit for bit, for every
set of the sequence (the two slots alternate, so sets k and k+2 share buffers)."""
import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu


def _sets(n, count):
    from paper_2307_06345_gb300 import workloads as w
    out = []
    for k in range(count):
        x, y, z = (w.clumps(n, 500 + k, n_clumps=20) if k % 2 else w.plummer(n, 600 + k))
        m = w.lognormal_masses(n, 700 + k)
        out.append(tuple(torch.from_numpy(np.ascontiguousarray(a)).pin_memory() for a in (x, y, z, m)))
    return out


@pytest.mark.parametrize("curve", [0, 1])
def test_streamed_equals_build_octree(lib, curve):
    n = 150_001
    sets = _sets(n, 5)
    sb = lib.StreamedBuilder(n, "cuda", curve=curve, ncrit=32)
    got = {}

    def keep(k, r):  # copy: the pinned result buffers are reused two sets later
        got[k] = {name: (v.clone() if torch.is_tensor(v) else v) for name, v in r.items()}

    h2d, d2h = sb.run(sets, on_result=keep)
    assert sorted(got) == list(range(len(sets)))
    assert h2d == len(sets) * n * 28
    for k, (x, y, z, m) in enumerate(sets):
        ref = lib.build_octree(x.cuda(), y.cuda(), z.cuda(), curve=curve, ncrit=32, masses=m.cuda())
        torch.cuda.synchronize()
        r = got[k]
        assert r["n_leaves"] == ref["n_leaves"]
        for name in sb.OUT:
            assert torch.equal(r[name], ref[name].reshape(-1).cpu()), (k, name)
    assert d2h == sum(sum(got[k][name].numel() * got[k][name].element_size() for name in sb.OUT) for k in got)


def test_streamed_rejects_wrong_sets(lib):
    sb = lib.StreamedBuilder(1000, "cuda")
    x = torch.zeros(999, dtype=torch.float64)
    with pytest.raises(ValueError):
        sb.run([(x, x, x, torch.zeros(999, dtype=torch.float32))])
    with pytest.raises(ValueError):
        sb.run([(torch.zeros(1000, dtype=torch.float64, device="cuda"),) * 3 + (torch.zeros(1000),)])


@pytest.mark.parametrize("count", [1, 2])
def test_streamed_short_sequences(lib, count):
    n = 10_000
    sets = _sets(n, count)
    sb = lib.StreamedBuilder(n, "cuda", curve=1, ncrit=16)
    got = {}
    sb.run(sets, on_result=lambda k, r: got.setdefault(k, r["NK"].clone()))
    assert sorted(got) == list(range(count))
    for k, (x, y, z, m) in enumerate(sets):
        ref = lib.build_octree(x.cuda(), y.cuda(), z.cuda(), curve=1, ncrit=16, masses=m.cuda())
        assert torch.equal(got[k], ref["NK"].cpu())


def test_host_build_through_c_abi(lib):
    # one set through cstone_host_stage and cstone_host_build directly: the host tree equals
    # build_octree on a device copy; then a leaf capacity too small is reported with a count above it
    import ctypes
    n = 70_001
    (x, y, z, m), = _sets(n, 1)
    L = lib.load()
    ref = lib.build_octree(x.cuda(), y.cuda(), z.cuda(), curve=1, ncrit=24, masses=m.cuda())
    torch.cuda.synchronize()
    for cap, ok in ((lib.leaf_capacity(n, 24), True), (ref["n_leaves"] - 7, False)):
        nbytes = ctypes.c_size_t()
        assert L.cstone_host_workspace_size(n, cap, 1, ctypes.byref(nbytes)) == 0
        ws = torch.empty(nbytes.value, dtype=torch.uint8, device="cuda")
        evs = [torch.cuda.Event() for _ in range(4)]
        for e in evs:
            e.record()
        slot = lib._HostSlot(ws.data_ptr(), nbytes.value, *(e.cuda_event for e in evs))
        nc = cap + (cap - 1) // 7
        host = [torch.empty(k, dtype=dt, pin_memory=True) for k, dt in
                ((cap + 1, torch.int64), (cap, torch.int32), (nc, torch.int64), (nc, torch.int32), (23, torch.int32),
                 (nc, torch.int32), (nc, torch.float32), (3 * nc, torch.float64), (6 * nc, torch.float32))]
        tree = lib._HostTree(*(t.data_ptr() for t in host), 0, 0, 0)
        s_in, s_c, s_o = torch.cuda.Stream(), torch.cuda.Stream(), torch.cuda.Stream()
        P = ctypes.c_void_p
        assert L.cstone_host_stage(P(x.data_ptr()), P(y.data_ptr()), P(z.data_ptr()), P(m.data_ptr()), n, cap,
                                   ctypes.byref(slot), P(s_in.cuda_stream)) == 0
        rc = L.cstone_host_build(n, cap, 1, 1, 24, 64, ctypes.byref(slot), ctypes.byref(tree), P(s_c.cuda_stream),
                                 P(s_o.cuda_stream))
        if not ok:
            assert rc == lib.ERR_CAPACITY and tree.n_leaves > cap
            continue
        assert rc == 0
        evs[3].synchronize()
        assert L.cstone_host_status(n, cap, 1, ctypes.byref(slot), P(s_c.cuda_stream)) == 0
        nl, nn = tree.n_leaves, tree.n_nodes
        assert nl == ref["n_leaves"] and nn == ref["NK"].numel() and tree.iters == ref["iters"]
        got = dict(zip(lib.StreamedBuilder.OUT, (host[0][: nl + 1], host[1][:nl], host[2][:nn], host[3][:nn],
                                                 host[4], host[5][:nn], host[6][:nn], host[7][: 3 * nn],
                                                 host[8][: 6 * nn])))
        for name, t in got.items():
            assert torch.equal(t, ref[name].reshape(-1).cpu()), name
