"""Autotuner for the tile shapes of the radix sort and of the leaf loop.

Run on the target GPU (``python -m paper_2307_06345_gb300.autotune``). Every candidate shape is
compiled into its own copy of the library (only the affected translation unit is rebuilt), timed
with CUDA events on the two workloads the shapes matter for, checked bit for bit against the
library's current output, and the fastest shape per knob group is written to ``tuning.json``,
which the in-tree build turns into compile definitions.

Workloads: the single-set build of 2^27 clump particles (Hilbert keys, Ncrit 64; the leaf loop also
at Ncrit 16) and the batched build of 512 sets of log-uniform size in [2^10, 2^20) (Morton keys,
Ncrit 32). A candidate's score is the sum of its median times on all of them.
"""
from __future__ import annotations

import argparse
import concurrent.futures
import ctypes
import json
import os
import tempfile
import time

import numpy as np
import torch

from . import _build

SORT_CANDIDATES = [{"threads": 256, "items": i, "min_blocks": b}
                   for i, b in ((8, 5), (8, 6), (10, 4), (10, 5), (12, 4), (14, 3), (14, 4), (16, 3), (16, 4))]
# the leaf loop stages a tile of elements in shared memory: more than 8 per thread exceeds 48 KB
LEAVES_CANDIDATES = [{"items": i} for i in (4, 6, 8)]

P = ctypes.c_void_p
i64, i32, u32, sz = ctypes.c_int64, ctypes.c_int32, ctypes.c_uint32, ctypes.c_size_t


def _open(path: str):
    L = ctypes.CDLL(path)
    sigs = {
        "cstone_sort_workspace_size": [i64, ctypes.POINTER(sz)],
        "cstone_sort": [P, P, P, i64, P, sz, P],
        "cstone_sort_segmented_workspace_size": [i64, i32, ctypes.POINTER(sz)],
        "cstone_sort_segmented": [P, P, P, i64, P, i32, P, sz, P],
        "cstone_leaves_workspace_size": [i64, i64, i32, ctypes.POINTER(sz)],
        "cstone_build_leaves": [P, i64, u32, P, i64, ctypes.POINTER(i64), P, P, i32, ctypes.POINTER(i32), P, sz, P],
        "cstone_leaves_batched_workspace_size": [i64, i32, ctypes.POINTER(sz)],
        "cstone_build_leaves_batched": [P, i64, P, i32, u32, P, i64, P, ctypes.POINTER(i64), P, P, i32,
                                        ctypes.POINTER(i32), P, sz, P],
        "cstone_workspace_status": [P, P, ctypes.POINTER(ctypes.c_int)],
    }
    for name, args in sigs.items():
        f = getattr(L, name)
        f.argtypes = args
        f.restype = ctypes.c_int
    return L


def _ptr(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _stream():
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


def _median_ms(fn, reps: int) -> float:
    fn()
    torch.cuda.synchronize()
    ts = []
    for _ in range(reps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        fn()
        e1.record()
        torch.cuda.synchronize()
        ts.append(e0.elapsed_time(e1))
    return sorted(ts)[len(ts) // 2]


class Inputs:
    """Keys and sorted keys of both workloads, made with the library as built now."""

    def __init__(self, dev, n_single: int):
        import paper_2307_06345_gb300 as cs
        from . import workloads as w

        x, y, z = w.clumps(n_single, w.BASE_SEED + 2)
        X, Y, Z = (torch.from_numpy(a).to(dev) for a in (x, y, z))
        ws = cs.Workspace(dev)
        box = torch.empty(4, dtype=torch.float64, device=dev)
        cs.cstone_bbox(X, Y, Z, box, ws)
        self.keys = torch.empty(n_single, dtype=torch.int64, device=dev)
        cs.cstone_keys(X, Y, Z, box, cs.HILBERT, self.keys)
        del X, Y, Z
        self.sorted = torch.empty_like(self.keys)
        self.perm = torch.empty(n_single, dtype=torch.int32, device=dev)
        cs.cstone_sort(self.keys, self.sorted, self.perm, ws)
        cap = cs.leaf_capacity(n_single, 64)
        self.leaves = torch.empty(cap + 1, dtype=torch.int64, device=dev)
        self.counts = torch.empty(cap, dtype=torch.int32, device=dev)
        self.n_leaves, _ = cs.cstone_build_leaves(self.sorted, 64, self.leaves, self.counts, None, 0, 64, ws)
        self.ref_leaves = self.leaves[: self.n_leaves + 1].clone()
        cap16 = cs.leaf_capacity(n_single, 16)  # the same keys at Ncrit 16 (the benchmark's other Ncrit)
        self.leaves16 = torch.empty(cap16 + 1, dtype=torch.int64, device=dev)
        self.counts16 = torch.empty(cap16, dtype=torch.int32, device=dev)
        self.n_leaves16, _ = cs.cstone_build_leaves(self.sorted, 16, self.leaves16, self.counts16, None, 0, 64, ws)
        self.ref_leaves16 = self.leaves16[: self.n_leaves16 + 1].clone()

        sets = w.batched_sets(512, w.BASE_SEED + 3)
        sizes = np.array([len(s[0]) for s in sets], np.int64)
        off = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
        BX, BY, BZ = (torch.from_numpy(np.concatenate([s[k] for s in sets])).to(dev) for k in range(3))
        self.set_offsets = torch.from_numpy(off).to(dev)
        boxes = torch.empty((512, 4), dtype=torch.float64, device=dev)
        cs.cstone_bbox_batched(BX, BY, BZ, self.set_offsets, boxes)
        unit = torch.tensor([0.0, 0.0, 0.0, 1.0], dtype=torch.float64, device=dev)
        for i, s in enumerate(sets):
            if s[3] == "uniform":
                boxes[i] = unit
        self.bkeys = torch.empty(BX.numel(), dtype=torch.int64, device=dev)
        cs.cstone_keys_batched(BX, BY, BZ, self.set_offsets, boxes, cs.MORTON, self.bkeys, ws)
        del BX, BY, BZ
        self.bsorted = torch.empty_like(self.bkeys)
        self.bperm = torch.empty(self.bkeys.numel(), dtype=torch.int32, device=dev)
        cs.cstone_sort_segmented(self.bkeys, self.bsorted, self.bperm, self.set_offsets, ws)
        self.belem_cap = max(4 * 512, 16 * (self.bkeys.numel() // 33) + 2 * 512 + 4096)
        self.belements = torch.empty(self.belem_cap, dtype=torch.int64, device=dev)
        self.beo = torch.empty(513, dtype=torch.int64, device=dev)
        self.bcounts = torch.empty(self.belem_cap, dtype=torch.int32, device=dev)
        ne, _ = cs.cstone_build_leaves_batched(self.bsorted, self.set_offsets, 32, self.belements, self.beo,
                                               self.bcounts, None, 0, 64, ws)
        self.bne = ne
        self.ref_belements = self.belements[:ne].clone()
        torch.cuda.synchronize()


def _ws(L, fn_size, *args):
    s = sz()
    rc = getattr(L, fn_size)(*args, ctypes.byref(s))
    if rc != 0:
        raise RuntimeError(f"{fn_size} failed ({rc})")
    return torch.empty(max(int(s.value), 256), dtype=torch.uint8, device="cuda")


def _status(L, ws) -> int:
    st = ctypes.c_int()
    L.cstone_workspace_status(_ptr(ws), _stream(), ctypes.byref(st))
    return st.value


def time_sort(L, inp: Inputs, reps: int):
    n = inp.keys.numel()
    ws = _ws(L, "cstone_sort_workspace_size", n)
    out, perm = torch.empty_like(inp.keys), torch.empty_like(inp.perm)
    single = _median_ms(lambda: L.cstone_sort(_ptr(inp.keys), _ptr(out), _ptr(perm), n, _ptr(ws), ws.numel(),
                                              _stream()), reps)
    ok = _status(L, ws) == 0 and torch.equal(out, inp.sorted) and torch.equal(perm, inp.perm)
    nb = inp.bkeys.numel()
    bws = _ws(L, "cstone_sort_segmented_workspace_size", nb, 512)
    bout, bperm = torch.empty_like(inp.bkeys), torch.empty_like(inp.bperm)
    batched = _median_ms(lambda: L.cstone_sort_segmented(_ptr(inp.bkeys), _ptr(bout), _ptr(bperm), nb,
                                                         _ptr(inp.set_offsets), 512, _ptr(bws), bws.numel(),
                                                         _stream()), reps)
    ok = ok and _status(L, bws) == 0 and torch.equal(bout, inp.bsorted) and torch.equal(bperm, inp.bperm)
    return {"single_ms": single, "batched_ms": batched, "score_ms": single + batched, "bit_exact": bool(ok)}


def time_leaves(L, inp: Inputs, reps: int):
    n = inp.sorted.numel()
    cap = inp.counts.numel()
    ws = _ws(L, "cstone_leaves_workspace_size", n, cap, 64)
    leaves, counts = torch.empty_like(inp.leaves), torch.empty_like(inp.counts)
    nl, it = i64(0), i32(0)

    def single_run():
        nl.value = 0
        rc = L.cstone_build_leaves(_ptr(inp.sorted), n, 64, _ptr(leaves), cap, ctypes.byref(nl), _ptr(counts), None,
                                   64, ctypes.byref(it), _ptr(ws), ws.numel(), _stream())
        if rc != 0:
            raise RuntimeError(f"cstone_build_leaves failed ({rc})")

    single = _median_ms(single_run, reps)
    ok = nl.value == inp.n_leaves and torch.equal(leaves[: nl.value + 1], inp.ref_leaves)
    cap16 = inp.counts16.numel()
    ws16 = _ws(L, "cstone_leaves_workspace_size", n, cap16, 64)
    leaves16, counts16 = torch.empty_like(inp.leaves16), torch.empty_like(inp.counts16)

    def single16_run():
        nl.value = 0
        rc = L.cstone_build_leaves(_ptr(inp.sorted), n, 16, _ptr(leaves16), cap16, ctypes.byref(nl), _ptr(counts16),
                                   None, 64, ctypes.byref(it), _ptr(ws16), ws16.numel(), _stream())
        if rc != 0:
            raise RuntimeError(f"cstone_build_leaves failed ({rc})")

    single16 = _median_ms(single16_run, reps)
    ok = ok and nl.value == inp.n_leaves16 and torch.equal(leaves16[: nl.value + 1], inp.ref_leaves16)
    nb = inp.bsorted.numel()
    bws = _ws(L, "cstone_leaves_batched_workspace_size", inp.belem_cap, 64)
    elements, eo, bcounts = torch.empty_like(inp.belements), torch.empty_like(inp.beo), torch.empty_like(inp.bcounts)
    ne = i64(0)

    def batched_run():
        ne.value = 0
        rc = L.cstone_build_leaves_batched(_ptr(inp.bsorted), nb, _ptr(inp.set_offsets), 512, 32, _ptr(elements),
                                           inp.belem_cap, _ptr(eo), ctypes.byref(ne), _ptr(bcounts), None, 64,
                                           ctypes.byref(it), _ptr(bws), bws.numel(), _stream())
        if rc != 0:
            raise RuntimeError(f"cstone_build_leaves_batched failed ({rc})")

    batched = _median_ms(batched_run, reps)
    ok = ok and ne.value == inp.bne and torch.equal(elements[: ne.value], inp.ref_belements)
    return {"single_ms": single, "single16_ms": single16, "batched_ms": batched,
            "score_ms": single + single16 + batched, "bit_exact": bool(ok)}


def tune(n_single: int = 1 << 27, reps: int = 5, out: str = _build.TUNING, verbose: bool = True) -> dict:
    import paper_2307_06345_gb300 as cs

    _build.build()
    cs.load()
    dev = torch.device("cuda", torch.cuda.current_device())
    t0 = time.time()
    inp = Inputs(dev, n_single)
    tmp = tempfile.mkdtemp(prefix="cstone_tune_")
    jobs = [("sort", c, {"CSTONE_SORT_THREADS": c["threads"], "CSTONE_SORT_ITEMS": c["items"],
                         "CSTONE_SORT_MIN_BLOCKS": c["min_blocks"]})
            for c in SORT_CANDIDATES]
    jobs += [("leaves", c, {"CSTONE_LEAVES_ITEMS": c["items"]}) for c in LEAVES_CANDIDATES]
    results = {"sort": [], "leaves": []}
    with concurrent.futures.ThreadPoolExecutor(max_workers=max(1, (os.cpu_count() or 2) // 2)) as ex:
        libs = list(ex.map(lambda ij: _build.build_variant(ij[1][2], os.path.join(tmp, f"lib{ij[0]}.so"),
                                                           os.path.join(tmp, f"obj{ij[0]}")), enumerate(jobs)))
    for (group, cand, knobs), lib in zip(jobs, libs):
        L = _open(lib)
        r = (time_sort if group == "sort" else time_leaves)(L, inp, reps)
        r["candidate"] = cand
        results[group].append(r)
        if verbose:
            print(group, cand, {k: round(v, 3) if isinstance(v, float) else v for k, v in r.items() if k != "candidate"},
                  flush=True)
    choice = {}
    for group in results:
        good = [r for r in results[group] if r["bit_exact"]]
        if not good:
            raise RuntimeError(f"no {group} candidate reproduced the reference output")
        choice[group] = min(good, key=lambda r: r["score_ms"])["candidate"]
    doc = {"device": torch.cuda.get_device_name(dev), "choice": choice, "measurements": results,
           "workloads": {"single": f"{n_single} clump particles, Hilbert keys, Ncrit 64 (leaf loop also at 16)",
                         "batched": "512 sets, sizes log-uniform in [2^10, 2^20), Morton keys, Ncrit 32"},
           "reps": reps, "seconds": round(time.time() - t0, 1)}
    with open(out, "w") as f:
        json.dump(doc, f, indent=1)
    return doc


def main():
    ap = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    ap.add_argument("--n", type=int, default=1 << 27, help="particles of the single-set workload")
    ap.add_argument("--reps", type=int, default=5)
    ap.add_argument("--out", default=_build.TUNING)
    a = ap.parse_args()
    doc = tune(a.n, a.reps, a.out)
    print(json.dumps(doc["choice"]))


if __name__ == "__main__":
    main()
