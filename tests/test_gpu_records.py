"""GPU tests of the record-writing key pass (cstone_keys_records) and of the multipole upsweep
from its records: the keys equal cstone_keys, the multipoles equal the packing upsweep bit for
bit, for both key lengths, and a coordinate outside the box's fixed-point range is reported in
the pass's error word."""
import numpy as np
import pytest
import torch

from _gpu_util import dev

pytestmark = pytest.mark.gpu


def _workload(kind, n, seed):
    from paper_2307_06345_gb300 import workloads as w
    if kind == "plummer":
        return w.plummer(n, seed)
    return w.clumps(n, seed, n_clumps=30)


@pytest.mark.parametrize("levels", [21, 10])
@pytest.mark.parametrize("curve", [0, 1])
@pytest.mark.parametrize("kind,n", [("plummer", 100_003), ("clumps", 1 << 18)])
def test_keys_records_and_multipoles(lib, oracle, levels, curve, kind, n):
    from paper_2307_06345_gb300 import workloads as w
    x, y, z = _workload(kind, n, 41 + curve)
    m = w.lognormal_masses(n, 43)
    box = oracle.bounding_cube(x, y, z)
    X, Y, Z, M, B = dev(x), dev(y), dev(z), dev(m), dev(box)
    kdt = torch.int64 if levels == 21 else torch.int32
    k_plain = torch.empty(n, dtype=kdt, device="cuda")
    lib.cstone_keys(X, Y, Z, B, curve, k_plain, levels=levels)
    k_rec = torch.empty(n, dtype=kdt, device="cuda")
    records = torch.empty(lib.records_size(n), dtype=torch.uint8, device="cuda")
    rws = lib.Workspace()
    lib.cstone_keys_records(X, Y, Z, M, B, curve, k_rec, records, rws, levels=levels)
    torch.cuda.synchronize()
    assert torch.equal(k_rec, k_plain)
    assert rws.status() == 0

    t = lib.build_octree(X, Y, Z, curve=curve, ncrit=16, box=B, levels=levels)
    nl = t["n_leaves"]
    nn = lib.n_nodes(nl)
    outs = []
    for use_records in (False, True):
        mass = torch.empty(nn, dtype=torch.float32, device="cuda")
        com = torch.empty(3 * nn, dtype=torch.float64, device="cuda")
        quad = torch.empty(6 * nn, dtype=torch.float32, device="cuda")
        ws = lib.Workspace()
        if use_records:
            lib.cstone_upsweep_multipoles_records(records, t["perm"], n, t["leaf_offsets"], nl, t["leaf_to_node"],
                                                  t["CO"], t["LO"], B, mass, com, quad, ws, levels=levels)
        else:
            lib.cstone_upsweep_multipoles(X, Y, Z, M, t["perm"], t["leaf_offsets"], nl, t["leaf_to_node"], t["CO"],
                                          t["LO"], B, mass, com, quad, ws, levels=levels)
        torch.cuda.synchronize()
        assert ws.status() == 0
        outs.append((mass, com, quad))
    for a, b in zip(*outs):
        assert torch.equal(a, b)
    # build_octree with masses goes through the record pass: the same multipoles
    full = lib.build_octree(X, Y, Z, curve=curve, ncrit=16, box=B, masses=M, levels=levels)
    torch.cuda.synchronize()
    assert torch.equal(full["mass"], outs[0][0])
    assert torch.equal(full["com"].reshape(-1), outs[0][1]) and torch.equal(full["quad"].reshape(-1), outs[0][2])


def test_keys_records_reports_out_of_range(lib):
    # box [0, 1]^3: the fixed-point frame covers |x| < 4; a particle at x = 100 is outside it
    n = 1000
    rng = np.random.default_rng(5)
    x, y, z = rng.random(n), rng.random(n), rng.random(n)
    x[17] = 100.0
    keys = torch.empty(n, dtype=torch.int64, device="cuda")
    records = torch.empty(lib.records_size(n), dtype=torch.uint8, device="cuda")
    rws = lib.Workspace()
    lib.cstone_keys_records(dev(x), dev(y), dev(z), dev(np.ones(n, np.float32)), dev(np.array([0.0, 0.0, 0.0, 1.0])),
                            1, keys, records, rws)
    assert rws.status() == lib.ERR_INVALID_ARG


def test_keys_records_argument_checks(lib):
    n = 64
    X = torch.zeros(n, dtype=torch.float64, device="cuda")
    keys = torch.empty(n, dtype=torch.int64, device="cuda")
    with pytest.raises(ValueError):  # records too small
        lib.cstone_keys_records(X, X, X, torch.zeros(n, dtype=torch.float32, device="cuda"),
                                torch.tensor([0.0, 0, 0, 1], dtype=torch.float64, device="cuda"), 1, keys,
                                torch.empty(16, dtype=torch.uint8, device="cuda"), lib.Workspace())


@pytest.mark.parametrize("n", [0, 1, 31, 63, 64, 65, 129, 1000, 4097])
def test_keys_records_sizes(lib, oracle, n):
    # the record pass takes 64 particles per warp (lanes l and l + 32): sizes around that window
    from paper_2307_06345_gb300 import workloads as w
    rng = np.random.default_rng(n + 3)
    x, y, z = rng.random(n), rng.random(n), rng.random(n)
    m = w.lognormal_masses(n, n + 4)
    box = np.array([0.0, 0.0, 0.0, 1.0])
    X, Y, Z, M, B = dev(x), dev(y), dev(z), dev(m), dev(box)
    for curve in (0, 1):
        keys = torch.empty(n, dtype=torch.int64, device="cuda")
        records = torch.empty(lib.records_size(n), dtype=torch.uint8, device="cuda")
        rws = lib.Workspace()
        lib.cstone_keys_records(X, Y, Z, M, B, curve, keys, records, rws)
        torch.cuda.synchronize()
        assert rws.status() == 0
        assert np.array_equal(keys.cpu().numpy().view(np.uint64), oracle.keys(x, y, z, box, curve))
        if n:  # the records hold the masses in order (last 8 bytes of each 32-byte record)
            rec = records[: 32 * n].cpu().numpy().view(np.uint32).reshape(n, 8)
            assert np.array_equal(rec[:, 6].view(np.float32), m) and not rec[:, 7].any()
