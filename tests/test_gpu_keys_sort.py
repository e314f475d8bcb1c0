"""GPU parity: bounding cube, SFC keys (Sec. 3) and the stable radix sort (Sec. 4) against the
oracle, bit for bit, including ragged tails, several tiles, duplicates and edge coordinates."""
import numpy as np
import pytest
import torch

from _gpu_util import dev, u32, u64

pytestmark = pytest.mark.gpu


def _inputs(kind, n, seed):
    from paper_2307_06345_gb300 import workloads as w
    if kind == "uniform":
        return w.uniform(n, seed)
    if kind == "plummer":
        return w.plummer(n, seed)
    if kind == "clumps":
        return w.clumps(n, seed, n_clumps=20)
    raise ValueError(kind)


@pytest.mark.parametrize("kind", ["uniform", "plummer", "clumps"])
@pytest.mark.parametrize("n", [1, 2, 1000, 100003])
def test_bbox_matches_oracle(lib, oracle, kind, n):
    x, y, z = _inputs(kind, n, 7 + n)
    box = torch.empty(4, dtype=torch.float64, device="cuda")
    ws = lib.Workspace()
    lib.cstone_bbox(dev(x), dev(y), dev(z), box, ws)
    assert np.array_equal(box.cpu().numpy(), oracle.bounding_cube(x, y, z))


def test_bbox_empty(lib, oracle):
    box = torch.empty(4, dtype=torch.float64, device="cuda")
    e = torch.empty(0, dtype=torch.float64, device="cuda")
    lib.cstone_bbox(e, e, e, box, lib.Workspace())
    assert list(box.cpu().numpy()) == [0.0, 0.0, 0.0, 1.0]


@pytest.mark.parametrize("curve", [0, 1])
@pytest.mark.parametrize("kind", ["uniform", "plummer", "clumps"])
def test_keys_bit_exact(lib, oracle, curve, kind):
    n = 200_003
    x, y, z = _inputs(kind, n, 11)
    box = np.array([0.0, 0.0, 0.0, 1.0]) if kind == "uniform" else oracle.bounding_cube(x, y, z)
    keys = torch.empty(n, dtype=torch.int64, device="cuda")
    lib.cstone_keys(dev(x), dev(y), dev(z), dev(box), curve, keys)
    assert np.array_equal(u64(keys), oracle.keys(x, y, z, box, curve))


@pytest.mark.parametrize("curve", [0, 1])
def test_keys_edge_coordinates(lib, oracle, curve):
    lo, side = -1.25, 2.5
    box = np.array([lo, lo, lo, side])
    hi = lo + side
    special = [lo, hi, lo - 1.0, hi + 1.0, np.nextafter(lo, -np.inf), np.nextafter(lo, np.inf),
               np.nextafter(hi, -np.inf), np.nextafter(hi, np.inf), -0.0, 0.0, 1e-300, -1e-300, 1e300, -1e300,
               lo + side / 2 ** 21, lo + side / 2]
    g = np.random.default_rng(3)
    pts = np.array(special)
    x = np.concatenate([pts, g.choice(pts, 997)])
    y = np.concatenate([pts[::-1], g.choice(pts, 997)])
    z = np.concatenate([np.roll(pts, 3), g.choice(pts, 997)])
    keys = torch.empty(x.size, dtype=torch.int64, device="cuda")
    lib.cstone_keys(dev(x), dev(y), dev(z), dev(box), curve, keys)
    assert np.array_equal(u64(keys), oracle.keys(x, y, z, box, curve))


@pytest.mark.parametrize("curve", [0, 1])
def test_keys_unaligned_views(lib, oracle, curve):
    # arrays that start one element into an allocation take the scalar path
    n = 5001
    x, y, z = _inputs("plummer", n + 1, 5)
    box = oracle.bounding_cube(x, y, z)
    X, Y, Z = dev(x)[1:], dev(y)[1:], dev(z)[1:]
    keys_buf = torch.empty(n + 1, dtype=torch.int64, device="cuda")
    keys = keys_buf[1:]
    lib.cstone_keys(X, Y, Z, dev(box), curve, keys)
    assert np.array_equal(u64(keys), oracle.keys(x[1:], y[1:], z[1:], box, curve))


def _key_sets(rng, n):
    yield "uniform", rng.integers(0, 1 << 63, n, dtype=np.uint64)
    c = rng.integers(0, 1 << 63, 7, dtype=np.uint64)
    yield "clustered", (c[rng.integers(0, 7, n)] + rng.integers(0, 1 << 20, n, dtype=np.uint64)) & np.uint64((1 << 63) - 1)
    yield "few_distinct", rng.integers(0, 1 << 63, 5, dtype=np.uint64)[rng.integers(0, 5, n)]
    yield "all_equal", np.full(n, 123456789, np.uint64)
    yield "sorted", np.sort(rng.integers(0, 1 << 63, n, dtype=np.uint64))
    yield "reversed", np.sort(rng.integers(0, 1 << 63, n, dtype=np.uint64))[::-1].copy()


@pytest.mark.parametrize("n", [0, 1, 2, 4095, 4096, 4097, 3 * 4096 + 17, 100_003, (1 << 20) + 7])
def test_sort_bit_exact(lib, oracle, n):
    rng = np.random.default_rng(n + 1)
    ws = lib.Workspace()
    for name, k in _key_sets(rng, n):
        kin = dev(k)
        kout = torch.empty_like(kin)
        perm = torch.empty(n, dtype=torch.int32, device="cuda")
        lib.cstone_sort(kin, kout, perm, ws)
        s, p = oracle.sort(k)
        assert np.array_equal(u64(kout), s), name
        assert np.array_equal(u32(perm), p), name
        assert ws.status() == 0


def test_sort_in_place(lib, oracle):
    rng = np.random.default_rng(9)
    k = rng.integers(0, 1 << 63, 50_000, dtype=np.uint64)
    t = dev(k)
    perm = torch.empty(k.size, dtype=torch.int32, device="cuda")
    lib.cstone_sort(t, t, perm, lib.Workspace())
    s, p = oracle.sort(k)
    assert np.array_equal(u64(t), s) and np.array_equal(u32(perm), p)


def test_kernel_launch_counter(lib):
    k = dev(np.arange(1000, dtype=np.uint64)[::-1].copy())
    kout = torch.empty_like(k)
    perm = torch.empty(1000, dtype=torch.int32, device="cuda")
    ws = lib.Workspace()
    before = lib.cstone_kernel_launches()
    lib.cstone_sort(k, kout, perm, ws)
    torch.cuda.synchronize()
    # per 8-bit digit pass: tile counts, chunk sums, chunk scan (which also totals the digits),
    # tile offsets and the pass itself
    assert lib.cstone_kernel_launches() - before == 8 * 5


def test_sort_repeated_calls_reuse_workspace(lib, oracle):
    # the per-tile count and offset regions are reused across calls of different sizes
    ws = lib.Workspace()
    rng = np.random.default_rng(10)
    for n in (300_000, 4097, 1 << 18, 17):
        k = rng.integers(0, 1 << 63, n, dtype=np.uint64)
        kin = dev(k)
        kout = torch.empty_like(kin)
        perm = torch.empty(n, dtype=torch.int32, device="cuda")
        lib.cstone_sort(kin, kout, perm, ws)
        s, p = oracle.sort(k)
        assert np.array_equal(u64(kout), s) and np.array_equal(u32(perm), p)


@pytest.mark.parametrize("curve", [0, 1])
@pytest.mark.parametrize("box", [(0.0, 0.0, 0.0, 1.0), (-20.0, -19.5, -21.0, 40.0), (0.1, -0.3, 7.0, 0.7),
                                 (1e6, 1e6, 1e6, 1e-3)])
def test_keys_at_cell_boundaries(lib, oracle, curve, box):
    # coordinates on and next to cell boundaries, where the integer fast path must defer to the
    # IEEE evaluation; the last box is too thin for the fast path altogether
    box = np.array(box)
    rng = np.random.default_rng(int(box[3] * 1000) + curve)
    n = 30_000
    cells = rng.integers(0, 1 << 21, (3, n))
    pts = []
    for d in range(3):
        b = box[d] + cells[d] * (box[3] / 2.0 ** 21)
        shift = rng.integers(-2, 3, n)
        for s in range(2):
            b = np.where(shift > 0, np.nextafter(b, np.inf), np.where(shift < 0, np.nextafter(b, -np.inf), b))
            shift = shift - np.sign(shift)
        pts.append(b)
    keys = torch.empty(n, dtype=torch.int64, device="cuda")
    lib.cstone_keys(dev(pts[0]), dev(pts[1]), dev(pts[2]), dev(box), curve, keys)
    assert np.array_equal(u64(keys), oracle.keys(pts[0], pts[1], pts[2], box, curve))
