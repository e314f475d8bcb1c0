"""GPU parity of the 30-bit key path (L = 10, entry points cstone30_*): keys, sort, leaves,
linked octree, node counts and multipoles against the oracle built for L = 10, bit for bit
(multipoles within the tolerance of the 63-bit path)."""
import numpy as np
import pytest
import torch

from _gpu_util import dev, i32, multipole_errors, node_level, u32, u64

pytestmark = pytest.mark.gpu

L10 = 10
END10 = 1 << 30
TOL = 1e-6


def _workload(kind, n, seed):
    from paper_2307_06345_gb300 import workloads as w
    if kind == "uniform":
        return w.uniform(n, seed)
    if kind == "plummer":
        return w.plummer(n, seed)
    return w.clumps(n, seed, n_clumps=50)


@pytest.mark.parametrize("curve", [0, 1])
@pytest.mark.parametrize("kind", ["uniform", "plummer", "clumps"])
def test_keys30_bit_exact_and_nested(lib, oracle, curve, kind):
    x, y, z = _workload(kind, 200_001, 31 + curve)
    box = oracle.bounding_cube(x, y, z)
    X, Y, Z, B = dev(x), dev(y), dev(z), dev(box)
    k30 = torch.empty(x.size, dtype=torch.int32, device="cuda")
    lib.cstone_keys(X, Y, Z, B, curve, k30, levels=10)
    k63 = torch.empty(x.size, dtype=torch.int64, device="cuda")
    lib.cstone_keys(X, Y, Z, B, curve, k63)
    got = u32(k30).astype(np.uint64)
    assert np.array_equal(got, oracle.keys(x, y, z, box, curve, levels=10))
    assert np.array_equal(got, u64(k63) >> np.uint64(33))


@pytest.mark.parametrize("n", [0, 1, 2, 4095, 4096, 4097, 100_003, 1 << 20])
def test_sort30_bit_exact(lib, oracle, n):
    rng = np.random.default_rng(n + 7)
    for kind in ("uniform", "few"):
        if kind == "uniform":
            k = rng.integers(0, END10, n, dtype=np.uint64)
        else:
            k = rng.integers(0, 8, n, dtype=np.uint64) << np.uint64(27)
        kin = dev(k.astype(np.uint32))
        kout = torch.empty_like(kin)
        perm = torch.empty(n, dtype=torch.int32, device="cuda")
        ws = lib.Workspace()
        lib.cstone_sort(kin, kout, perm, ws, levels=10)
        s, p = oracle.sort(k)
        assert np.array_equal(u32(kout).astype(np.uint64), s)
        assert np.array_equal(u32(perm), p)
        if n:
            assert ws.status() == 0


def test_sort30_in_place(lib, oracle):
    k = np.random.default_rng(3).integers(0, END10, 77_777, dtype=np.uint64)
    t = dev(k.astype(np.uint32))
    perm = torch.empty(k.size, dtype=torch.int32, device="cuda")
    lib.cstone_sort(t, t, perm, lib.Workspace(), levels=10)
    s, p = oracle.sort(k)
    assert np.array_equal(u32(t).astype(np.uint64), s) and np.array_equal(u32(perm), p)


def _check_tree(out, ref):
    assert np.array_equal(u32(out["keys"]).astype(np.uint64), ref["keys"])
    assert np.array_equal(u32(out["sorted_keys"]).astype(np.uint64), ref["P"])
    assert np.array_equal(u32(out["perm"]), ref["perm"])
    assert np.array_equal(u32(out["leaves"]).astype(np.uint64), ref["K"])
    assert np.array_equal(u32(out["leaf_counts"]), ref["N"])
    assert out["iters"] == ref["iters"]
    assert np.array_equal(u32(out["NK"]).astype(np.uint64), ref["NK"])
    assert np.array_equal(i32(out["CO"]), ref["CO"])
    assert np.array_equal(i32(out["LO"]), ref["LO"])
    assert np.array_equal(i32(out["leaf_to_node"]), ref["leaf_to_node"])
    assert np.array_equal(u32(out["node_counts"]), ref["counts"])


@pytest.mark.parametrize("kind,n,curve,ncrit", [("uniform", 65_536, 0, 64), ("plummer", 1 << 21, 1, 64),
                                                ("clumps", 1 << 20, 1, 16), ("clumps", 300_000, 0, 1)])
def test_full_build30(lib, oracle, kind, n, curve, ncrit):
    x, y, z = _workload(kind, n, 55)
    box = np.array([0.0, 0.0, 0.0, 1.0]) if kind == "uniform" else oracle.bounding_cube(x, y, z)
    ref = oracle.full_build(x, y, z, curve, ncrit, box=box, levels=10)
    out = lib.build_octree(dev(x), dev(y), dev(z), curve=curve, ncrit=ncrit, box=dev(box), levels=10)
    torch.cuda.synchronize()
    _check_tree(out, ref)
    sizes = np.diff(ref["K"].astype(np.int64))
    if kind == "clumps":  # dense clumps end in over-full level-10 cells, which are not split
        assert ((sizes == 1) & (ref["N"] > ncrit)).any()
    assert ref["LO"].size == L10 + 2


def test_warm_start30(lib, oracle):
    from paper_2307_06345_gb300 import workloads as w
    x, y, z = w.plummer(1 << 18, 77)
    box = oracle.bounding_cube(x, y, z)
    first = lib.build_octree(dev(x), dev(y), dev(z), curve=1, ncrit=32, box=dev(box), levels=10)
    dx, dy, dz = w.displacement(x.size, 78, 0.02)
    x2, y2, z2 = x + dx, y + dy, z + dz
    warm = lib.build_octree(dev(x2), dev(y2), dev(z2), curve=1, ncrit=32, box=dev(box), levels=10,
                            warm_leaves=first["leaves"].clone())
    torch.cuda.synchronize()
    ref = oracle.full_build(x2, y2, z2, 1, 32, box=box, levels=10)
    assert np.array_equal(u32(warm["leaves"]).astype(np.uint64), ref["K"])
    assert np.array_equal(u32(warm["node_counts"]), ref["counts"])


@pytest.mark.parametrize("kind", ["plummer", "clumps"])
def test_multipoles30(lib, oracle, kind):
    from paper_2307_06345_gb300 import workloads as w
    n = 60_000
    x, y, z = _workload(kind, n, 91)
    m = w.lognormal_masses(n, 92)
    box = oracle.bounding_cube(x, y, z)
    ref = oracle.full_build(x, y, z, 1, 16, box=box, levels=10)
    M_ref, c_ref, q_ref = oracle.multipoles(x, y, z, m, ref["P"], ref["perm"], ref["NK"], levels=10)
    out = lib.build_octree(dev(x), dev(y), dev(z), curve=1, ncrit=16, box=dev(box), masses=dev(m), levels=10)
    torch.cuda.synchronize()
    assert np.array_equal(u32(out["NK"]).astype(np.uint64), ref["NK"])
    side = box[3] * 2.0 ** (-node_level(ref["NK"]).astype(np.float64))
    err = multipole_errors(M_ref, c_ref, q_ref, out["mass"].cpu().numpy().astype(np.float64),
                           out["com"].cpu().numpy().T.copy(), out["quad"].cpu().numpy().T.astype(np.float64), side)
    assert err["mass"] <= TOL and err["com"] <= TOL and err["quad"] <= TOL, err
