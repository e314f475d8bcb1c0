"""Host protocol of the global tree of a particle set spread over several processes (Sec. 6):
two and three gloo ranks on the CPU. The per-rank steps (bounds, keys, sort, f, g) are the oracle's, so the
test exercises the protocol (allreduce of the counts after every f, identical g on every rank, the
decomposition and the particle exchange) without a GPU; the kernels behind the same steps are
checked against the oracle by the GPU tests. The result must equal the oracle's single-process
build of the union of the ranks' particles."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


class OracleOps:
    """The per-rank steps of paper_2307_06345_gb300.distributed, computed by the oracle on CPU
    tensors (int64 keys)."""

    def __init__(self, oracle):
        self.o = oracle

    def bounds(self, x, y, z):
        if x.numel() == 0:
            return torch.tensor([np.inf] * 3 + [-np.inf] * 3, dtype=torch.float64)
        c = [t.numpy() for t in (x, y, z)]
        return torch.tensor([a.min() for a in c] + [a.max() for a in c], dtype=torch.float64)

    def cube(self, bounds):
        return torch.from_numpy(self.o.cube_from_bounds(bounds.numpy()))

    def decompose(self, N, world):
        return torch.from_numpy(self.o.decompose(N.numpy().view(np.uint32), world))

    def keys(self, x, y, z, box, curve):
        k = self.o.keys(x.numpy(), y.numpy(), z.numpy(), box.numpy(), curve)
        return torch.from_numpy(k.view(np.int64).copy())

    def sort(self, keys):
        s, p = self.o.sort(keys.numpy().view(np.uint64))
        return torch.from_numpy(s.view(np.int64).copy()), torch.from_numpy(p.view(np.int32).copy())

    def root(self):
        return torch.tensor([0, -(1 << 63)], dtype=torch.int64)

    def leaf_counts(self, P, K, n_leaves):
        N = self.o.histogram(P.numpy().view(np.uint64), K[: n_leaves + 1].numpy().view(np.uint64))
        return torch.from_numpy(N.view(np.int32).copy())

    def rebalance(self, K, N, n_leaves, ncrit):
        Ku = K[: n_leaves + 1].numpy().view(np.uint64)
        O = self.o.rebalance_decision(Ku, N.numpy().view(np.uint32), ncrit)
        Kn = self.o.rebalance(Ku, O, self.o.exclusive_scan(O))
        changed = bool((O[:n_leaves] != 1).any())
        return torch.from_numpy(Kn.view(np.int64).copy()), Kn.size - 1, changed


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _parts(world, seed):
    from paper_2307_06345_gb300 import workloads as w
    x, y, z = w.clumps(30_000, seed, n_clumps=20)
    owner = np.random.default_rng(seed).integers(0, world, x.size)  # particles dealt to ranks at random
    return x, y, z, owner


def _worker(rank, world, port, q, ncrit):
    import sys

    import torch.distributed as dist

    sys.path.insert(0, ROOT)
    import oracle
    from paper_2307_06345_gb300 import distributed as D

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        x, y, z, owner = _parts(world, 41)
        mine = owner == rank
        X, Y, Z = (torch.from_numpy(np.ascontiguousarray(a[mine])) for a in (x, y, z))
        ids = torch.from_numpy(np.nonzero(mine)[0].astype(np.float64))  # global particle ids ride along
        ops = OracleOps(oracle)
        t = D.build_global_tree(X, Y, Z, curve=1, ncrit=ncrit, group=None, ops=ops)
        cuts = D.decompose(ops, t["N_global"], world)
        rx, ry, rz, rid = D.exchange(ops, X, Y, Z, t["P"], t["perm"], t["K"], cuts, extra=(ids,))
        q.put((rank, t["box"].numpy(), t["K"].numpy().view(np.uint64), t["N_global"].numpy().view(np.uint32),
               t["passes"], cuts.tolist(), rx.numpy(), ry.numpy(), rz.numpy(), rid.numpy().astype(np.int64)))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world,ncrit", [(2, 16), (2, 64), (3, 16)])
def test_ranks_build_the_single_process_tree(oracle, world, ncrit):
    port = _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q, ncrit)) for r in range(world)]
    for p in procs:
        p.start()
    res = {}
    for _ in range(world):
        r = q.get(timeout=240)
        res[r[0]] = r
    for p in procs:
        p.join(timeout=60)
    assert all(p.exitcode == 0 for p in procs)

    x, y, z, owner = _parts(world, 41)
    box = oracle.bounding_cube(x, y, z)
    ref = oracle.full_build(x, y, z, 1, ncrit, box=box)
    for r in range(world):  # every rank holds the global box, leaves and counts of the union
        assert np.array_equal(res[r][1], box)
        assert np.array_equal(res[r][2], ref["K"])
        assert np.array_equal(res[r][3], ref["N"])
        assert res[r][4] == ref["iters"]
    # decomposition: contiguous leaf ranges in curve order, about half of the particles each
    cuts = res[0][5]
    assert cuts == res[1][5] and cuts[0] == 0 and cuts[-1] == len(ref["N"])
    K = ref["K"]
    got_ids = []
    for r in range(world):
        lo, hi = K[cuts[r]], K[cuts[r + 1]]
        k = oracle.keys(res[r][6], res[r][7], res[r][8], box, 1)
        assert np.all((k >= lo) & (k < hi))  # every particle landed on the rank owning its key
        assert abs(len(k) - x.size / world) <= ref["N"].max() + 1
        got_ids.append(res[r][9])
        assert np.array_equal(res[r][6], x[res[r][9]])  # coordinates travelled with their ids
    assert np.array_equal(np.sort(np.concatenate(got_ids)), np.arange(x.size))


def test_decompose_goes_through_the_ops(oracle):
    """The protocol's decomposition is the ops' (the device call on a GPU rank); with the oracle's
    ops it gives the oracle's cuts, which the oracle's own tests pin to the definition."""
    from paper_2307_06345_gb300 import distributed as D
    N = torch.tensor([5, 0, 7, 3, 3, 9, 1, 0, 4, 8], dtype=torch.int32)
    ops = OracleOps(oracle)
    for world in (1, 2, 3, 4, 10, 16):
        cuts = D.decompose(ops, N, world)
        assert cuts.tolist() == oracle.decompose(N.numpy().view(np.uint32), world).tolist()
    assert D.decompose(ops, torch.zeros(4, dtype=torch.int32), 3).tolist() == [0, 0, 0, 4]
