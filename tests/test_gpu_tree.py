"""GPU parity: cornerstone leaves (Sec. 4), linked octree (Sec. 5), count and multipole upsweeps
against the oracle. Integer outputs bit for bit; multipoles within 1e-6 per moment."""
import numpy as np
import pytest
import torch

from _gpu_util import dev, i32, multipole_errors, node_level, u32, u64

pytestmark = pytest.mark.gpu

KEY_END = 1 << 63
TOL = 1e-6


def _sorted_keys(rng, n, kind):
    if kind == "uniform":
        k = rng.integers(0, KEY_END, n, dtype=np.uint64)
    elif kind == "clustered":
        c = rng.integers(0, KEY_END, 6, dtype=np.uint64)
        k = np.minimum(c[rng.integers(0, 6, n)] + rng.integers(0, 1 << 24, n, dtype=np.uint64), np.uint64(KEY_END - 1))
    elif kind == "duplicates":
        k = rng.integers(0, KEY_END, 4, dtype=np.uint64)[rng.integers(0, 4, n)]
    else:
        raise ValueError(kind)
    return np.sort(k)


def _gpu_leaves(lib, P, ncrit, K_init=None, cap=None, max_iters=64):
    n = P.size
    cap = cap or max(64, lib.leaf_capacity(n, ncrit))
    leaves = torch.zeros(cap + 1, dtype=torch.int64, device="cuda")
    counts = torch.empty(cap, dtype=torch.int32, device="cuda")
    offsets = torch.empty(cap + 1, dtype=torch.int32, device="cuda")
    nl0 = 0
    if K_init is not None:
        nl0 = K_init.size - 1
        leaves[: nl0 + 1] = dev(K_init)
    nl, it = lib.cstone_build_leaves(dev(P) if n else torch.empty(0, dtype=torch.int64, device="cuda"), ncrit,
                                     leaves, counts, offsets, nl0, max_iters)
    return u64(leaves[: nl + 1]), u32(counts[:nl]), u32(offsets[: nl + 1]), it


CASES = [(kind, n, ncrit) for kind in ("uniform", "clustered", "duplicates")
         for n in (0, 1, 100, 5000, 70_001) for ncrit in (1, 8, 64)]


@pytest.mark.parametrize("kind,n,ncrit", CASES)
def test_leaves_cold_bit_exact(lib, oracle, kind, n, ncrit):
    rng = np.random.default_rng(n * 7 + ncrit)
    P = _sorted_keys(rng, n, kind) if n else np.zeros(0, np.uint64)
    K, N, off, it = _gpu_leaves(lib, P, ncrit)
    K_ref, N_ref, it_ref = oracle.build_leaves(P, ncrit)
    assert np.array_equal(K, K_ref)
    assert np.array_equal(N, N_ref)
    assert it == it_ref
    assert np.array_equal(off, np.concatenate([[0], np.cumsum(N_ref)]).astype(np.uint32))


@pytest.mark.parametrize("seed", range(6))
def test_leaves_warm_start_bit_exact(lib, oracle, seed):
    rng = np.random.default_rng(50 + seed)
    kind = ("uniform", "clustered", "duplicates")[seed % 3]
    ncrit = (4, 16, 64)[seed % 3]
    P0 = _sorted_keys(rng, 40_000, kind)
    P1 = _sorted_keys(rng, 30_000, kind)
    K0, _, _ = oracle.build_leaves(P0, ncrit)
    K, N, _, it = _gpu_leaves(lib, P1, ncrit, K_init=K0)
    K_ref, N_ref, it_ref = oracle.build_leaves(P1, ncrit, K_init=K0)
    assert np.array_equal(K, K_ref) and np.array_equal(N, N_ref) and it == it_ref


def test_leaves_many_tiles(lib, oracle):
    # enough leaves for many 2048-leaf tiles in every pass, with a ragged last tile
    rng = np.random.default_rng(77)
    P = _sorted_keys(rng, 2_000_003, "uniform")
    K, N, _, it = _gpu_leaves(lib, P, 4)
    K_ref, N_ref, it_ref = oracle.build_leaves(P, 4)
    assert K.size > 100_000
    assert np.array_equal(K, K_ref) and np.array_equal(N, N_ref) and it == it_ref


def test_leaves_capacity_error(lib):
    rng = np.random.default_rng(3)
    P = _sorted_keys(rng, 10_000, "uniform")
    with pytest.raises(lib.CstoneError) as e:
        _gpu_leaves(lib, P, 4, cap=100)
    assert e.value.status == lib.ERR_CAPACITY and e.value.required > 100


def test_leaves_not_converged(lib):
    P = np.full(100, 5, np.uint64)  # needs 22 passes
    with pytest.raises(lib.CstoneError) as e:
        _gpu_leaves(lib, P, 1, max_iters=5)
    assert e.value.status == lib.ERR_NOT_CONVERGED


def _gpu_link(lib, K, check=True):
    nl = K.size - 1
    nn = nl + (nl - 1) // 7
    NK = torch.empty(nn, dtype=torch.int64, device="cuda")
    CO = torch.empty(nn, dtype=torch.int32, device="cuda")
    LO = torch.empty(23, dtype=torch.int32, device="cuda")
    l2n = torch.empty(nl, dtype=torch.int32, device="cuda")
    parent = torch.empty(max((nn - 1) // 8, 1), dtype=torch.int32, device="cuda")
    ws = lib.Workspace()
    lib.cstone_link_tree(dev(K), nl, NK, CO, LO, l2n, parent, ws)
    if not check:
        return NK, CO, LO, l2n, parent, ws
    assert ws.status() == 0
    return NK, CO, LO, l2n, parent


@pytest.mark.parametrize("kind,n,ncrit", [(k, n, c) for k in ("uniform", "clustered", "duplicates")
                                          for n in (0, 1, 3000, 400_000) for c in (1, 16)])
def test_link_and_counts_bit_exact(lib, oracle, kind, n, ncrit):
    rng = np.random.default_rng(n + ncrit)
    P = _sorted_keys(rng, n, kind) if n else np.zeros(0, np.uint64)
    K, N, _ = oracle.build_leaves(P, ncrit)
    ref = oracle.link(K)
    NK, CO, LO, l2n, parent = _gpu_link(lib, K)
    assert np.array_equal(u64(NK), ref["NK"])
    assert np.array_equal(i32(CO), ref["CO"])
    assert np.array_equal(i32(LO), ref["LO"])
    assert np.array_equal(i32(l2n), ref["leaf_to_node"])
    nn = ref["NK"].size
    assert np.array_equal(i32(parent)[: (nn - 1) // 8], ref["parent"])
    counts = torch.empty(nn, dtype=torch.int32, device="cuda")
    lib.cstone_upsweep_counts(dev(N.astype(np.uint32)), K.size - 1, l2n, CO, LO, counts)
    assert np.array_equal(u32(counts), oracle.node_counts(P, ref["NK"]))


def test_link_reports_non_cornerstone_input(lib):
    # 15 "leaves" whose gaps are not powers of 8 and imply 19 nodes instead of
    # n_l + (n_l - 1) / 7 = 17: the device error word reports it, and writes stay inside the arrays
    K = np.array([2 * i for i in range(15)] + [KEY_END], np.uint64)
    _, _, _, _, _, ws = _gpu_link(lib, K, check=False)
    assert ws.status() == lib.ERR_INVALID_ARG
    with pytest.raises(lib.CstoneError):
        _gpu_link(lib, np.array(list(range(9)) + [KEY_END], np.uint64))  # 9 leaves is not 1 + 7k: host check


def _multipole_case(lib, oracle, x, y, z, m, curve, ncrit, box=None):
    if box is None:
        box = oracle.bounding_cube(x, y, z)
    ref = oracle.full_build(x, y, z, curve, ncrit, box=box)
    M_ref, c_ref, q_ref = oracle.multipoles(x, y, z, m, ref["P"], ref["perm"], ref["NK"])
    out = lib.build_octree(dev(x), dev(y), dev(z), curve=curve, ncrit=ncrit, box=dev(np.asarray(box)),
                           masses=dev(m))
    torch.cuda.synchronize()
    assert np.array_equal(u64(out["NK"]), ref["NK"])
    M = out["mass"].cpu().numpy().astype(np.float64)
    com = out["com"].cpu().numpy().T.copy()
    q = out["quad"].cpu().numpy().T.astype(np.float64)
    side = box[3] * 2.0 ** (-node_level(ref["NK"]).astype(np.float64))
    return multipole_errors(M_ref, c_ref, q_ref, M, com, q, side)


@pytest.mark.parametrize("kind", ["uniform", "plummer", "clumps"])
def test_multipoles_within_tolerance(lib, oracle, kind):
    from paper_2307_06345_gb300 import workloads as w
    n = 60_000
    x, y, z = {"uniform": w.uniform, "plummer": w.plummer}.get(kind, lambda n, s: w.clumps(n, s, n_clumps=30))(n, 21)
    m = w.lognormal_masses(n, 22)
    err = _multipole_case(lib, oracle, x, y, z, m, 1, 16)
    assert err["mass"] <= TOL and err["com"] <= TOL and err["quad"] <= TOL, err


def test_multipoles_of_leaves_larger_than_a_group(lib, oracle):
    # full-depth leaves of thousands of coincident particles are summed by a whole block
    rng = np.random.default_rng(5)
    base = rng.random((30, 3))
    pts = np.concatenate([np.repeat(base[:6], 3000, axis=0) + 1e-9 * rng.standard_normal((18000, 3)),
                          rng.random((5000, 3))])
    m = rng.lognormal(0, 1, len(pts)).astype(np.float32)
    err = _multipole_case(lib, oracle, pts[:, 0].copy(), pts[:, 1].copy(), pts[:, 2].copy(), m, 1, 16)
    assert err["mass"] <= TOL and err["com"] <= TOL and err["quad"] <= TOL, err


def test_multipoles_duplicates_and_single_particles(lib, oracle):
    rng = np.random.default_rng(4)
    base = rng.random((50, 3))
    pts = np.concatenate([np.repeat(base[:10], 40, axis=0), base[10:]])  # heavy duplicates + singles
    m = rng.lognormal(0, 1, len(pts)).astype(np.float32)
    err = _multipole_case(lib, oracle, pts[:, 0].copy(), pts[:, 1].copy(), pts[:, 2].copy(), m, 0, 8)
    assert err["mass"] <= TOL and err["com"] <= TOL and err["quad"] <= TOL, err


@pytest.mark.parametrize("ncrit,lo,hi", [(16, 0, 8), (48, 8, 12), (128, 12, 1e9)])
def test_multipoles_each_leaf_group_width(lib, oracle, ncrit, lo, hi):
    # the leaf sums take 2, 4 or 8 lanes per leaf by the mean leaf size (below 8, below 12, above):
    # one case in each range
    from paper_2307_06345_gb300 import workloads as w
    n = 60_000
    x, y, z = w.clumps(n, 21, n_clumps=30)
    m = w.lognormal_masses(n, 22)
    box = oracle.bounding_cube(x, y, z)
    mean = n / (oracle.full_build(x, y, z, 1, ncrit, box=box)["K"].size - 1)
    assert lo <= mean < hi, mean
    err = _multipole_case(lib, oracle, x, y, z, m, 1, ncrit, box=box)
    assert err["mass"] <= TOL and err["com"] <= TOL and err["quad"] <= TOL, err
