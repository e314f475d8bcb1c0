"""The global octree of a particle set spread over several processes, and its SFC domain
decomposition (Sec. 6).

Every rank holds some of the particles. The bounding cube is that of the union (per-axis minima and
maxima reduced over the ranks), keys and the sort stay local, and the cornerstone array is the same
on every rank: each f/g step counts the rank's own particles per leaf (f), sums the counts over the
ranks with one allreduce of n_l integers (f_glob = f_r o f), and applies g to the summed counts,
which every rank does identically, so the arrays never diverge. The decomposition then cuts the
array into one contiguous range of leaves per rank holding about the same number of particles, and
the exchange sends every particle to the rank that owns its key.

The per-rank steps run in the library's kernels (``DeviceOps``); ``torch.distributed`` carries the
counts and the particles (NCCL between GPUs, gloo between CPU processes). The ops object is a
parameter so that the protocol can be exercised by processes without a GPU.
"""
from __future__ import annotations

import torch

from . import (HILBERT, LEVELS, Workspace, cstone_bounds, cstone_cube_from_bounds, cstone_decompose, cstone_keys,
               cstone_leaf_counts, cstone_rebalance, cstone_sort)


class DeviceOps:
    """The per-rank steps through the CUDA library (keys, sort, f, g) on one device."""

    def __init__(self, device, levels: int = LEVELS):
        self.device = torch.device(device)
        self.levels = levels
        self.key_dtype = torch.int64 if levels == LEVELS else torch.int32
        self.ws = Workspace(self.device)

    def bounds(self, x, y, z):
        out = torch.empty(6, dtype=torch.float64, device=self.device)
        cstone_bounds(x, y, z, out, self.ws)
        return out

    def cube(self, bounds):
        """Bounding cube {lo, side} of per-axis bounds reduced over the ranks."""
        box = torch.empty(4, dtype=torch.float64, device=self.device)
        cstone_cube_from_bounds(bounds.contiguous(), box)
        return box

    def decompose(self, N, world: int):
        """The world + 1 leaf cuts of the decomposition of the global counts N (int64 tensor)."""
        cuts = torch.empty(world + 1, dtype=torch.int64, device=self.device)
        cstone_decompose(N, N.numel(), world, cuts, self.ws)
        return cuts

    def keys(self, x, y, z, box, curve):
        k = torch.empty(x.numel(), dtype=self.key_dtype, device=self.device)
        cstone_keys(x, y, z, box, curve, k, levels=self.levels)
        return k

    def sort(self, keys):
        s = torch.empty_like(keys)
        perm = torch.empty(keys.numel(), dtype=torch.int32, device=self.device)
        cstone_sort(keys, s, perm, self.ws, levels=self.levels)
        return s, perm

    def root(self):
        end = 1 << (3 * self.levels)  # 8^L, stored as the bit pattern of the key word
        if end >= 1 << 63:
            end -= 1 << 64
        return torch.tensor([0, end], dtype=self.key_dtype, device=self.device)

    def leaf_counts(self, P, K, n_leaves: int):
        N = torch.empty(n_leaves, dtype=torch.int32, device=self.device)
        cstone_leaf_counts(P, K, n_leaves, N, levels=self.levels)
        return N

    def rebalance(self, K, N, n_leaves: int, ncrit: int):
        """(new array, its n_l, changed)."""
        cap = 8 * n_leaves + 1
        out = torch.empty(cap + 1, dtype=self.key_dtype, device=self.device)
        nl, changed = cstone_rebalance(K, N, n_leaves, ncrit, out, self.ws, levels=self.levels)
        return out[: nl + 1], nl, changed


def _allreduce(t, op, group):
    import torch.distributed as dist

    if group is not False and dist.is_available() and dist.is_initialized():
        dist.all_reduce(t, op=op, group=group)
    return t


def global_box(ops, x, y, z, group=None):
    """Bounding cube of the union of all ranks' particles: {lo_x, lo_y, lo_z, side} (float64). The
    per-axis minima and maxima are reduced over the ranks; the cube is formed from them by
    ``ops.cube`` (cstone_cube_from_bounds on the device)."""
    import torch.distributed as dist

    b = ops.bounds(x, y, z)
    lo, hi = b[:3].clone(), b[3:].clone()
    _allreduce(lo, dist.ReduceOp.MIN, group)
    _allreduce(hi, dist.ReduceOp.MAX, group)
    return ops.cube(torch.cat([lo, hi]))


def global_leaves(ops, P, ncrit: int, group=None, max_iters: int = 64):
    """The cornerstone array of all ranks' particles from each rank's sorted keys P: repeated f,
    allreduce of the counts, g, until g changes nothing. Returns (K, n_leaves, N_global, passes);
    K and N_global are identical on every rank."""
    import torch.distributed as dist

    K = ops.root()
    nl = 1
    for it in range(1, max_iters + 1):
        N = ops.leaf_counts(P, K, nl)
        _allreduce(N, dist.ReduceOp.SUM, group)
        K_new, nl_new, changed = ops.rebalance(K, N, nl, ncrit)
        if not changed:
            return K, nl, N, it
        K, nl = K_new, nl_new
    raise RuntimeError(f"global leaf array not converged after {max_iters} passes")


def decompose(ops, N_global, world: int):
    """Leaf ranges per rank along the curve (Sec. 6): rank r owns leaves [cuts[r], cuts[r + 1]), cut
    at the first leaf whose preceding leaves hold r / world of the total (``ops.decompose``,
    cstone_decompose on the device). Returns the world + 1 cuts as an int64 tensor."""
    return ops.decompose(N_global, world)


def exchange(ops, x, y, z, P, perm, K, cuts, group=None, extra=()):
    """Send every particle to the rank whose key range holds its key. P / perm are this rank's sorted
    keys and permutation; the particles of one destination are a contiguous run of the sorted
    order, whose lengths are f applied to the ranks' key ranges. Returns the received (x, y, z,
    *extra) in key order of the senders."""
    import torch.distributed as dist

    world = cuts.numel() - 1
    bounds = K[cuts.to(K.device)].contiguous()  # range starts + the end key
    send = ops.leaf_counts(P, bounds, world).to(torch.int64)
    cols = [c.index_select(0, perm.to(torch.int64)) for c in (x, y, z) + tuple(extra)]
    if group is False or not (dist.is_available() and dist.is_initialized()) or dist.get_world_size(group) == 1:
        return cols
    recv = torch.empty_like(send)
    dist.all_to_all_single(recv, send, group=group)
    s_list, r_list = send.cpu().tolist(), recv.cpu().tolist()
    out = []
    for c in cols:
        r = torch.empty(sum(r_list), dtype=c.dtype, device=c.device)
        dist.all_to_all_single(r, c, r_list, s_list, group=group)
        out.append(r)
    return out


def build_global_tree(x, y, z, curve: int = HILBERT, ncrit: int = 64, group=None, ops=None, levels: int = LEVELS):
    """Global box, keys, local sort and the global cornerstone array of all ranks' particles.
    Returns a dict with box, keys, sorted keys P, perm, K, n_leaves, N_global, passes."""
    ops = ops or DeviceOps(x.device, levels)
    box = global_box(ops, x, y, z, group)
    keys = ops.keys(x, y, z, box, curve)
    P, perm = ops.sort(keys)
    K, nl, N, passes = global_leaves(ops, P, ncrit, group)
    return {"box": box, "keys": keys, "P": P, "perm": perm, "K": K, "n_leaves": nl, "N_global": N,
            "passes": passes}
