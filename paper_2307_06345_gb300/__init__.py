"""GB300-native Cornerstone octree build (Keller et al., PASC'23, arXiv 2307.06345).

The compute path lives in the CUDA library ``libcstone.so`` (sources in ``csrc/``, C ABI in
``include/cstone.h``). This module loads it with ctypes and marshals PyTorch CUDA tensors and
streams into the C calls; the functions named ``cstone_*`` mirror the C entry points one to one.
PyTorch only provides device memory and streams: every step of the build runs in the library's
kernels, and nothing falls back to the CPU. If the library has not been built, ``load()`` raises.

``build_octree`` strings the steps together in the paper's order (keys, sort, leaves, linked
tree, count upsweep, optionally multipoles) and allocates the outputs.
"""
from __future__ import annotations

import ctypes
import os
import threading
from dataclasses import dataclass, field

import torch

from . import _build

__all__ = [
    "MORTON", "HILBERT", "CstoneError", "load", "build", "cstone_bbox", "cstone_keys", "cstone_sort",
    "cstone_build_leaves", "cstone_link_tree", "cstone_upsweep_counts", "cstone_upsweep_multipoles",
    "build_octree", "Workspace", "leaf_capacity", "n_nodes", "cstone_sort_static", "cstone_bbox_batched",
    "cstone_keys_batched", "cstone_sort_segmented", "cstone_build_leaves_batched", "cstone_link_tree_batched",
    "cstone_upsweep_counts_batched", "build_octrees_batched", "cstone_build_leaves_batched_async",
    "cstone_leaves_result", "cstone_kernel_launches", "TimeStepper", "GraphTimeStepper", "cstone_leaf_counts",
    "cstone_rebalance", "cstone_bounds", "cstone_rebalance_focus", "build_focus_leaves", "LEVELS", "LEVELS30",
    "StreamedBuilder", "records_size", "cstone_keys_records", "cstone_upsweep_multipoles_records",
    "cstone_cube_from_bounds", "cstone_decompose", "cstone_build_batched", "cstone_build_batched_result",
    "BatchBuffers", "batched_capacity",
]

MORTON, HILBERT = 0, 1
LEVELS = 21    # 63-bit keys (entry points cstone_*, int64 key tensors)
LEVELS30 = 10  # 30-bit keys (entry points cstone30_*, int32 key tensors)
KEY_END = 1 << 63
OK, ERR_INVALID_ARG, ERR_CUDA, ERR_CAPACITY, ERR_TIMEOUT, ERR_NOT_CONVERGED = range(6)

_lib = None
_lock = threading.Lock()


class CstoneError(RuntimeError):
    def __init__(self, status: int, where: str, detail: str):
        super().__init__(f"{where}: {status_string(status)} ({detail})")
        self.status = status


def build(force: bool = False) -> str:
    """Compile libcstone.so in-tree for sm_103a."""
    return _build.build(force=force)


def load():
    """Load libcstone.so (raises if it is missing or stale: run ``build()``)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(_build.LIB):
            raise RuntimeError(f"CUDA library {_build.LIB} is missing: call paper_2307_06345_gb300.build() "
                               "(the product has no CPU fallback)")
        lib = ctypes.CDLL(_build.LIB)
        P, i64, i32, u32, sz = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32, ctypes.c_uint32, ctypes.c_size_t
        pi64, pi32, psz = ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_size_t)
        sigs = {
            "cstone_status_string": (ctypes.c_char_p, [ctypes.c_int]),
            "cstone_last_error_detail": (ctypes.c_int, [ctypes.c_char_p, sz]),
            "cstone_version": (ctypes.c_int, []),
            "cstone_kernel_launches": (ctypes.c_int64, []),
            "cstone_workspace_status": (ctypes.c_int, [P, P, ctypes.POINTER(ctypes.c_int)]),
            "cstone_bbox_workspace_size": (ctypes.c_int, [i64, psz]),
            "cstone_bbox": (ctypes.c_int, [P, P, P, i64, P, P, sz, P]),
            "cstone_keys": (ctypes.c_int, [P, P, P, i64, P, ctypes.c_int, P, P]),
            "cstone_sort_workspace_size": (ctypes.c_int, [i64, psz]),
            "cstone_sort": (ctypes.c_int, [P, P, P, i64, P, sz, P]),
            "cstone_sort_static": (ctypes.c_int, [P, P, P, i64, P]),
            "cstone_leaves_workspace_size": (ctypes.c_int, [i64, i64, i32, psz]),
            "cstone_build_leaves": (ctypes.c_int, [P, i64, u32, P, i64, pi64, P, P, i32, pi32, P, sz, P]),
            "cstone_link_workspace_size": (ctypes.c_int, [i64, psz]),
            "cstone_link_tree": (ctypes.c_int, [P, i64, P, P, P, P, P, P, sz, P]),
            "cstone_upsweep_workspace_size": (ctypes.c_int, [i64, psz]),
            "cstone_upsweep_counts": (ctypes.c_int, [P, i64, P, P, P, P, P, sz, P]),
            "cstone_multipole_workspace_size": (ctypes.c_int, [i64, i64, psz]),
            "cstone_upsweep_multipoles": (ctypes.c_int, [P, P, P, P, P, i64, P, i64, P, P, P, P, P, P, P, P, sz, P]),
            "cstone_bbox_batched": (ctypes.c_int, [P, P, P, P, i32, P, P]),
            "cstone_keys_batched_workspace_size": (ctypes.c_int, [i32, psz]),
            "cstone_keys_batched": (ctypes.c_int, [P, P, P, i64, P, i32, P, ctypes.c_int, P, P, sz, P]),
            "cstone_sort_segmented_workspace_size": (ctypes.c_int, [i64, i32, psz]),
            "cstone_sort_segmented": (ctypes.c_int, [P, P, P, i64, P, i32, P, sz, P]),
            "cstone_leaves_batched_workspace_size": (ctypes.c_int, [i64, i32, psz]),
            "cstone_build_leaves_batched": (ctypes.c_int, [P, i64, P, i32, u32, P, i64, P, pi64, P, P, i32, pi32, P,
                                                          sz, P]),
            "cstone_link_batched_workspace_size": (ctypes.c_int, [i64, i32, psz]),
            "cstone_link_tree_batched": (ctypes.c_int, [P, i64, P, i32, i64, P, P, P, P, P, sz, P]),
            "cstone_upsweep_counts_batched": (ctypes.c_int, [P, i64, P, P, P, i32, P, P, sz, P]),
            "cstone_build_leaves_batched_async": (ctypes.c_int, [P, i64, P, i32, u32, P, i64, P, i32, P, P, i32, P,
                                                                sz, P]),
            "cstone_leaves_result": (ctypes.c_int, [P, i64, i32, P, pi64, pi32]),
            "cstone_leaf_counts": (ctypes.c_int, [P, i64, P, i64, P, P]),
            "cstone_bounds": (ctypes.c_int, [P, P, P, i64, P, P, sz, P]),
            "cstone_cube_from_bounds": (ctypes.c_int, [P, P, P]),
            "cstone_decompose_workspace_size": (ctypes.c_int, [i64, i32, psz]),
            "cstone_decompose": (ctypes.c_int, [P, i64, i32, P, P, sz, P]),
            "cstone_rebalance_focus": (ctypes.c_int, [P, P, i64, u32, ctypes.c_uint64, ctypes.c_uint64,
                                                      ctypes.c_double, ctypes.c_int, P, i64, pi64, pi32, P, sz, P]),
            "cstone_rebalance_workspace_size": (ctypes.c_int, [i64, psz]),
            "cstone_rebalance": (ctypes.c_int, [P, P, i64, u32, P, i64, pi64, pi32, P, sz, P]),
            "cstone_build_batched_workspace_size": (ctypes.c_int, [i64, i32, i64, i32, psz]),
            "cstone_build_batched": (ctypes.c_int, [ctypes.POINTER(_BatchInput), ctypes.POINTER(_BatchParams),
                                                    ctypes.POINTER(_BatchBuffers), P, sz, P]),
            "cstone_build_batched_result": (ctypes.c_int, [P, i64, i32, i64, i32, P, P, pi64, pi64, pi32]),
            "cstone_records_size": (ctypes.c_int, [i64, psz]),
            "cstone_keys_records_workspace_size": (ctypes.c_int, [psz]),
            "cstone_keys_records": (ctypes.c_int, [P, P, P, P, i64, P, ctypes.c_int, P, P, P, sz, P]),
            "cstone_upsweep_multipoles_records": (ctypes.c_int, [P, P, i64, P, i64, P, P, P, P, P, P, P, P, sz, P]),
            "cstone_host_workspace_size": (ctypes.c_int, [i64, i64, i32, psz]),
            "cstone_host_stage": (ctypes.c_int, [P, P, P, P, i64, i64, ctypes.POINTER(_HostSlot), P]),
            "cstone_host_build": (ctypes.c_int, [i64, i64, i32, i32, u32, i32, ctypes.POINTER(_HostSlot),
                                                 ctypes.POINTER(_HostTree), P, P]),
            "cstone_host_status": (ctypes.c_int, [i64, i64, i32, ctypes.POINTER(_HostSlot), P]),
        }
        for name in ("keys", "sort_workspace_size", "sort", "leaves_workspace_size", "build_leaves",
                     "link_workspace_size", "link_tree", "upsweep_workspace_size", "upsweep_counts",
                     "multipole_workspace_size", "upsweep_multipoles", "leaf_counts", "rebalance_workspace_size",
                     "rebalance", "rebalance_focus", "keys_records", "upsweep_multipoles_records"):
            sigs["cstone30_" + name] = sigs["cstone_" + name]
        res, args = sigs["cstone30_rebalance_focus"]
        sigs["cstone30_rebalance_focus"] = (res, args[:4] + [u32, u32] + args[6:])
        for name, (res, args) in sigs.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
        return lib


def status_string(status: int) -> str:
    if _lib is None:
        return f"status {status}"
    return _lib.cstone_status_string(status).decode()


def _detail() -> str:
    buf = ctypes.create_string_buffer(512)
    load().cstone_last_error_detail(buf, 512)
    return buf.value.decode(errors="replace")


def _check(rc: int, where: str):
    if rc != OK:
        raise CstoneError(rc, where, _detail())


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else None


def _stream(stream):
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _size(fn, *args) -> int:
    out = ctypes.c_size_t()
    _check(fn(*args, ctypes.byref(out)), fn.__name__)
    return int(out.value)


class Workspace:
    """Device scratch for the library calls, grown on demand (256-byte aligned torch buffer)."""

    def __init__(self, device=None):
        self.device = torch.device(device if device is not None else "cuda")
        self.buf = None

    def get(self, nbytes: int) -> torch.Tensor:
        if self.buf is None or self.buf.numel() < nbytes:
            self.buf = torch.empty(max(nbytes, 256), dtype=torch.uint8, device=self.device)
        return self.buf

    def status(self, stream=None) -> int:
        st = ctypes.c_int()
        _check(load().cstone_workspace_status(_ptr(self.buf), _stream(stream), ctypes.byref(st)), "workspace_status")
        return st.value


def _need(t: torch.Tensor, dtype, name):
    if not t.is_cuda or t.dtype != dtype or not t.is_contiguous():
        raise ValueError(f"{name} must be a contiguous CUDA tensor of {dtype}")


class _BatchInput(ctypes.Structure):
    _fields_ = [("x", ctypes.c_void_p), ("y", ctypes.c_void_p), ("z", ctypes.c_void_p), ("n", ctypes.c_int64),
                ("set_offsets", ctypes.c_void_p), ("n_sets", ctypes.c_int32), ("boxes", ctypes.c_void_p)]


class _BatchParams(ctypes.Structure):
    _fields_ = [("curve", ctypes.c_int32), ("ncrit", ctypes.c_uint32), ("max_iters", ctypes.c_int32),
                ("warm", ctypes.c_int32)]


class _BatchBuffers(ctypes.Structure):
    _fields_ = [("boxes_out", ctypes.c_void_p), ("keys", ctypes.c_void_p), ("sorted_keys", ctypes.c_void_p),
                ("perm", ctypes.c_void_p), ("elements", ctypes.c_void_p), ("elem_cap", ctypes.c_int64),
                ("element_offsets", ctypes.c_void_p), ("leaf_counts", ctypes.c_void_p),
                ("leaf_offsets", ctypes.c_void_p), ("node_keys", ctypes.c_void_p), ("child", ctypes.c_void_p),
                ("level_offsets", ctypes.c_void_p), ("leaf_to_node", ctypes.c_void_p),
                ("node_counts", ctypes.c_void_p), ("node_cap", ctypes.c_int64)]


class _HostSlot(ctypes.Structure):
    _fields_ = [("ws", ctypes.c_void_p), ("ws_bytes", ctypes.c_size_t), ("staged", ctypes.c_void_p),
                ("inputs_read", ctypes.c_void_p), ("built", ctypes.c_void_p), ("copied_out", ctypes.c_void_p)]


class _HostTree(ctypes.Structure):
    _fields_ = [("leaves", ctypes.c_void_p), ("leaf_counts", ctypes.c_void_p), ("node_keys", ctypes.c_void_p),
                ("child", ctypes.c_void_p), ("level_offsets", ctypes.c_void_p), ("node_counts", ctypes.c_void_p),
                ("mass", ctypes.c_void_p), ("com", ctypes.c_void_p), ("quad", ctypes.c_void_p),
                ("n_leaves", ctypes.c_int64), ("n_nodes", ctypes.c_int64), ("iters", ctypes.c_int32)]


# ------------------------------------------------------------------------- C entry points
def _family(levels: int):
    """(C function, key dtype) picker for the key length: 21 levels -> cstone_*, int64 keys;
    10 levels -> cstone30_*, int32 keys (bit patterns of uint32)."""
    lib = load()
    if levels == LEVELS:
        return (lambda name: getattr(lib, "cstone_" + name)), torch.int64
    if levels == LEVELS30:
        return (lambda name: getattr(lib, "cstone30_" + name)), torch.int32
    raise ValueError(f"levels must be {LEVELS} or {LEVELS30}, not {levels}")


def cstone_kernel_launches() -> int:
    """Kernels the library has launched in this process so far."""
    return int(load().cstone_kernel_launches())


def cstone_bbox(x, y, z, box, ws: Workspace, stream=None):
    lib = load()
    n = x.numel()
    for t, nm in ((x, "x"), (y, "y"), (z, "z")):
        _need(t, torch.float64, nm)
    _need(box, torch.float64, "box")
    need = _size(lib.cstone_bbox_workspace_size, n)
    buf = ws.get(need)
    _check(lib.cstone_bbox(_ptr(x), _ptr(y), _ptr(z), n, _ptr(box), _ptr(buf), buf.numel(), _stream(stream)),
           "cstone_bbox")


def cstone_bounds(x, y, z, bounds, ws: Workspace, stream=None):
    """bounds[6] (float64 CUDA) = per-axis minima then maxima (+inf / -inf when empty)."""
    lib = load()
    for t, nm in ((x, "x"), (y, "y"), (z, "z"), (bounds, "bounds")):
        _need(t, torch.float64, nm)
    buf = ws.get(_size(lib.cstone_bbox_workspace_size, x.numel()))
    _check(lib.cstone_bounds(_ptr(x), _ptr(y), _ptr(z), x.numel(), _ptr(bounds), _ptr(buf), buf.numel(),
                             _stream(stream)), "cstone_bounds")


def cstone_cube_from_bounds(bounds, box, stream=None):
    """box[4] (float64 CUDA) = the bounding cube of the per-axis bounds[6] (minima, maxima) reduced
    over several processes (Sec. 6)."""
    _need(bounds, torch.float64, "bounds")
    _need(box, torch.float64, "box")
    if bounds.numel() < 6 or box.numel() < 4:
        raise ValueError("bounds needs 6 entries and box 4")
    _check(load().cstone_cube_from_bounds(_ptr(bounds), _ptr(box), _stream(stream)), "cstone_cube_from_bounds")


def cstone_decompose(counts, n_leaves: int, n_ranks: int, cuts, ws: Workspace, stream=None):
    """cuts[n_ranks + 1] (int64 CUDA) = the SFC domain decomposition of the global leaf counts
    (Sec. 6): rank r owns leaves [cuts[r], cuts[r + 1])."""
    lib = load()
    _need(counts, torch.int32, "counts")
    _need(cuts, torch.int64, "cuts")
    if counts.numel() < n_leaves or cuts.numel() < n_ranks + 1:
        raise ValueError("counts needs n_leaves entries and cuts n_ranks + 1")
    buf = ws.get(_size(lib.cstone_decompose_workspace_size, n_leaves, n_ranks))
    _check(lib.cstone_decompose(_ptr(counts), n_leaves, n_ranks, _ptr(cuts), _ptr(buf), buf.numel(),
                                _stream(stream)), "cstone_decompose")


def cstone_keys(x, y, z, box, curve: int, keys, stream=None, levels: int = LEVELS):
    fn, kdt = _family(levels)
    for t, nm in ((x, "x"), (y, "y"), (z, "z"), (box, "box")):
        _need(t, torch.float64, nm)
    _need(keys, kdt, "keys")
    _check(fn("keys")(_ptr(x), _ptr(y), _ptr(z), x.numel(), _ptr(box), curve, _ptr(keys), _stream(stream)),
           "cstone_keys")


def _sort_args(keys_in, keys_out, perm, kdt, who: str):
    """Checks the sort operands: dtypes, contiguity, output sizes, and that all three tensors sit
    on the current CUDA device (the sort kernels run there)."""
    n = keys_in.numel()
    if keys_out.numel() < n or perm.numel() < n:
        raise ValueError(f"{who}: keys_out and perm need at least {n} elements "
                         f"(have {keys_out.numel()} and {perm.numel()})")
    _need(keys_in, kdt, "keys_in")
    _need(keys_out, kdt, "keys_out")
    _need(perm, torch.int32, "perm")
    cur = torch.cuda.current_device()
    for t, nm in ((keys_in, "keys_in"), (keys_out, "keys_out"), (perm, "perm")):
        if t.device.index != cur:
            raise ValueError(f"{who}: {nm} is on {t.device}, the current device is cuda:{cur}")
    return n


def cstone_sort(keys_in, keys_out, perm, ws: Workspace, stream=None, levels: int = LEVELS):
    fn, kdt = _family(levels)
    n = _sort_args(keys_in, keys_out, perm, kdt, "cstone_sort")
    buf = ws.get(_size(fn("sort_workspace_size"), n))
    _check(fn("sort")(_ptr(keys_in), _ptr(keys_out), _ptr(perm), n, _ptr(buf), buf.numel(), _stream(stream)),
           "cstone_sort")


def cstone_sort_static(keys_in, keys_out, perm, stream=None):
    """Sort without any device allocation: scratch is a static array inside the library, so at most
    2^20 keys, and calls must not overlap on the GPU (see include/cstone.h)."""
    lib = load()
    _sort_args(keys_in, keys_out, perm, torch.int64, "cstone_sort_static")
    _check(lib.cstone_sort_static(_ptr(keys_in), _ptr(keys_out), _ptr(perm), keys_in.numel(), _stream(stream)),
           "cstone_sort_static")


def cstone_build_leaves(sorted_keys, ncrit: int, leaves, counts, offsets=None, n_leaves: int = 0,
                        max_iters: int = 64, ws: Workspace | None = None, stream=None, levels: int = LEVELS):
    """Returns (n_leaves, iterations). ``leaves`` holds the initial array when n_leaves > 0."""
    fn, kdt = _family(levels)
    n = sorted_keys.numel()
    cap = counts.numel()
    _need(sorted_keys, kdt, "sorted_keys")
    _need(leaves, kdt, "leaves")
    _need(counts, torch.int32, "counts")
    if leaves.numel() < cap + 1:
        raise ValueError("leaves needs leaf_cap + 1 entries")
    if offsets is not None:
        _need(offsets, torch.int32, "offsets")
    ws = ws or Workspace(sorted_keys.device)
    buf = ws.get(_size(fn("leaves_workspace_size"), n, cap, max_iters))
    nl = ctypes.c_int64(n_leaves)
    it = ctypes.c_int32(0)
    rc = fn("build_leaves")(_ptr(sorted_keys), n, ncrit, _ptr(leaves), cap, ctypes.byref(nl), _ptr(counts),
                            _ptr(offsets), max_iters, ctypes.byref(it), _ptr(buf), buf.numel(), _stream(stream))
    if rc == ERR_CAPACITY:
        err = CstoneError(rc, "cstone_build_leaves", _detail())
        err.required = int(nl.value)
        raise err
    _check(rc, "cstone_build_leaves")
    return int(nl.value), int(it.value)


def cstone_link_tree(leaves, n_leaves: int, node_keys, child, level_offsets, leaf_to_node, parent=None,
                     ws: Workspace | None = None, stream=None, levels: int = LEVELS):
    fn, kdt = _family(levels)
    _need(leaves, kdt, "leaves")
    _need(node_keys, kdt, "node_keys")
    if level_offsets.numel() < levels + 2:
        raise ValueError(f"level_offsets needs {levels + 2} entries")
    ws = ws or Workspace(leaves.device)
    buf = ws.get(_size(fn("link_workspace_size"), n_leaves))
    _check(fn("link_tree")(_ptr(leaves), n_leaves, _ptr(node_keys), _ptr(child), _ptr(level_offsets),
                           _ptr(leaf_to_node), _ptr(parent), _ptr(buf), buf.numel(), _stream(stream)),
           "cstone_link_tree")


def cstone_upsweep_counts(leaf_counts, n_leaves: int, leaf_to_node, child, level_offsets, node_counts,
                          ws: Workspace | None = None, stream=None, levels: int = LEVELS):
    fn, _ = _family(levels)
    ws = ws or Workspace(leaf_counts.device)
    buf = ws.get(_size(fn("upsweep_workspace_size"), n_leaves))
    _check(fn("upsweep_counts")(_ptr(leaf_counts), n_leaves, _ptr(leaf_to_node), _ptr(child), _ptr(level_offsets),
                                _ptr(node_counts), _ptr(buf), buf.numel(), _stream(stream)),
           "cstone_upsweep_counts")


def cstone_upsweep_multipoles(x, y, z, m, perm, offsets, n_leaves: int, leaf_to_node, child, level_offsets, box,
                              mass, com, quad, ws: Workspace | None = None, stream=None, levels: int = LEVELS):
    fn, _ = _family(levels)
    _need(m, torch.float32, "m")
    ws = ws or Workspace(x.device)
    buf = ws.get(_size(fn("multipole_workspace_size"), x.numel(), n_leaves))
    _check(fn("upsweep_multipoles")(_ptr(x), _ptr(y), _ptr(z), _ptr(m), _ptr(perm), x.numel(), _ptr(offsets),
                                    n_leaves, _ptr(leaf_to_node), _ptr(child), _ptr(level_offsets), _ptr(box),
                                    _ptr(mass), _ptr(com), _ptr(quad), _ptr(buf), buf.numel(), _stream(stream)),
           "cstone_upsweep_multipoles")


def records_size(n: int) -> int:
    """Bytes of the multipole records of n particles (cstone_keys_records)."""
    return _size(load().cstone_records_size, n)


def cstone_keys_records(x, y, z, m, box, curve: int, keys, records, ws: Workspace, stream=None,
                        levels: int = LEVELS):
    """Keys (as cstone_keys) and the multipole records of the particles in one pass; ``records`` is
    a uint8 CUDA tensor of records_size(n) bytes. Coordinate range errors go to ws's error word."""
    fn, kdt = _family(levels)
    _need(keys, kdt, "keys")
    _need(m, torch.float32, "m")
    if records.dtype != torch.uint8 or records.numel() < records_size(x.numel()):
        raise ValueError("records must be a uint8 CUDA tensor of records_size(n) bytes")
    buf = ws.get(_size(load().cstone_keys_records_workspace_size))
    _check(fn("keys_records")(_ptr(x), _ptr(y), _ptr(z), _ptr(m), x.numel(), _ptr(box), curve, _ptr(keys),
                              _ptr(records), _ptr(buf), buf.numel(), _stream(stream)), "cstone_keys_records")


def cstone_upsweep_multipoles_records(records, perm, n: int, offsets, n_leaves: int, leaf_to_node, child,
                                      level_offsets, box, mass, com, quad, ws: Workspace | None = None, stream=None,
                                      levels: int = LEVELS):
    fn, _ = _family(levels)
    ws = ws or Workspace(perm.device)
    buf = ws.get(_size(fn("multipole_workspace_size"), 0, n_leaves))
    _check(fn("upsweep_multipoles_records")(_ptr(records), _ptr(perm), n, _ptr(offsets), n_leaves,
                                            _ptr(leaf_to_node), _ptr(child), _ptr(level_offsets), _ptr(box),
                                            _ptr(mass), _ptr(com), _ptr(quad), _ptr(buf), buf.numel(),
                                            _stream(stream)), "cstone_upsweep_multipoles_records")


def cstone_leaf_counts(sorted_keys, leaves, n_leaves: int, counts, stream=None, levels: int = LEVELS):
    """f: counts[i] = particles of sorted_keys in [leaves[i], leaves[i+1])."""
    fn, kdt = _family(levels)
    _need(sorted_keys, kdt, "sorted_keys")
    _need(leaves, kdt, "leaves")
    _need(counts, torch.int32, "counts")
    _check(fn("leaf_counts")(_ptr(sorted_keys), sorted_keys.numel(), _ptr(leaves), n_leaves, _ptr(counts),
                             _stream(stream)), "cstone_leaf_counts")


def cstone_rebalance(leaves, counts, n_leaves: int, ncrit: int, leaves_out, ws: Workspace, stream=None,
                     levels: int = LEVELS):
    """g1-g3 on the given counts; returns (n_leaves_out, changed). ``leaves_out`` holds
    leaf_cap + 1 keys."""
    fn, kdt = _family(levels)
    _need(leaves, kdt, "leaves")
    _need(leaves_out, kdt, "leaves_out")
    _need(counts, torch.int32, "counts")
    buf = ws.get(_size(fn("rebalance_workspace_size"), n_leaves))
    nl = ctypes.c_int64(0)
    ch = ctypes.c_int32(0)
    rc = fn("rebalance")(_ptr(leaves), _ptr(counts), n_leaves, ncrit, _ptr(leaves_out), leaves_out.numel() - 1,
                         ctypes.byref(nl), ctypes.byref(ch), _ptr(buf), buf.numel(), _stream(stream))
    if rc == ERR_CAPACITY:
        err = CstoneError(rc, "cstone_rebalance", _detail())
        err.required = int(nl.value)
        raise err
    _check(rc, "cstone_rebalance")
    return int(nl.value), bool(ch.value)


def cstone_rebalance_focus(leaves, counts, n_leaves: int, ncrit: int, f_start: int, f_end: int, theta: float,
                           curve: int, leaves_out, ws: Workspace, stream=None, levels: int = LEVELS):
    """g1^LE-g3 of the tree focused on the key range [f_start, f_end) (Sec. 7); returns
    (n_leaves_out, changed)."""
    fn, kdt = _family(levels)
    _need(leaves, kdt, "leaves")
    _need(leaves_out, kdt, "leaves_out")
    _need(counts, torch.int32, "counts")
    buf = ws.get(_size(fn("rebalance_workspace_size"), n_leaves))
    nl = ctypes.c_int64(0)
    ch = ctypes.c_int32(0)
    rc = fn("rebalance_focus")(_ptr(leaves), _ptr(counts), n_leaves, ncrit, f_start, f_end, theta, curve,
                               _ptr(leaves_out), leaves_out.numel() - 1, ctypes.byref(nl), ctypes.byref(ch),
                               _ptr(buf), buf.numel(), _stream(stream))
    if rc == ERR_CAPACITY:
        err = CstoneError(rc, "cstone_rebalance_focus", _detail())
        err.required = int(nl.value)
        raise err
    _check(rc, "cstone_rebalance_focus")
    return int(nl.value), bool(ch.value)


def build_focus_leaves(sorted_keys, ncrit: int, f_start: int, f_end: int, theta: float, curve: int,
                       warm_leaves=None, max_iters: int = 64, ws: Workspace | None = None, levels: int = LEVELS):
    """The locally essential tree of one process focused on the key range [f_start, f_end) (Sec. 7):
    f (cstone_leaf_counts) and g1^LE-g3 (cstone_rebalance_focus) until nothing changes, from the
    root or from ``warm_leaves``. Returns (leaves [n_l + 1], counts [n_l], passes)."""
    dev = sorted_keys.device
    kdt = sorted_keys.dtype
    ws = ws or Workspace(dev)
    if warm_leaves is None:
        end = 1 << (3 * levels)
        K = torch.tensor([0, end - (1 << 64) if end >= 1 << 63 else end], dtype=kdt, device=dev)
    else:
        K = warm_leaves
    nl = K.numel() - 1
    for it in range(1, max_iters + 1):
        N = torch.empty(nl, dtype=torch.int32, device=dev)
        cstone_leaf_counts(sorted_keys, K, nl, N, levels=levels)
        out = torch.empty(8 * nl + 2, dtype=kdt, device=dev)
        nl2, changed = cstone_rebalance_focus(K, N, nl, ncrit, f_start, f_end, theta, curve, out, ws, levels=levels)
        if not changed:
            return K[: nl + 1], N, it
        K, nl = out[: nl2 + 1], nl2
    raise CstoneError(ERR_NOT_CONVERGED, "build_focus_leaves", f"not converged after {max_iters} passes")


# ------------------------------------------------------------------------- whole build
def leaf_capacity(n: int, ncrit: int) -> int:
    """A first guess for the leaf capacity; build_octree grows it if the tree needs more."""
    return int(min(1 << 28, 16 * (n // (ncrit + 1)) + 4096))


def n_nodes(n_leaves: int) -> int:
    return n_leaves + (n_leaves - 1) // 7


@dataclass
class OctreeBuffers:
    """Reusable device buffers for repeated builds of the same size (outputs and scratch)."""
    device: torch.device
    n: int
    cap: int
    keys: torch.Tensor = None
    sorted_keys: torch.Tensor = None
    perm: torch.Tensor = None
    box: torch.Tensor = None
    leaves: torch.Tensor = None
    counts: torch.Tensor = None
    offsets: torch.Tensor = None
    ws: Workspace = None
    tree: dict = field(default_factory=dict)
    levels: int = LEVELS
    records: torch.Tensor = None  # multipole records (cstone_keys_records), allocated on first use
    rws: Workspace = None         # error word of the record-writing key pass

    @classmethod
    def allocate(cls, n: int, cap: int, device="cuda", levels: int = LEVELS):
        d = torch.device(device)
        kdt = torch.int64 if levels == LEVELS else torch.int32
        b = cls(device=d, n=n, cap=cap, levels=levels)
        b.keys = torch.empty(n, dtype=kdt, device=d)
        b.sorted_keys = torch.empty(n, dtype=kdt, device=d)
        b.perm = torch.empty(n, dtype=torch.int32, device=d)
        b.box = torch.empty(4, dtype=torch.float64, device=d)
        b.leaves = torch.empty(cap + 1, dtype=kdt, device=d)
        b.counts = torch.empty(cap, dtype=torch.int32, device=d)
        b.offsets = torch.empty(cap + 1, dtype=torch.int32, device=d)
        b.ws = Workspace(d)
        return b

    def tree_buffers(self, n_leaves: int):
        nn = n_nodes(n_leaves)
        t = self.tree
        if t.get("cap_nodes", 0) < nn:
            d = self.device
            cap_nodes = max(nn, int(1.25 * nn))
            t.clear()
            t["cap_nodes"] = cap_nodes
            t["NK"] = torch.empty(cap_nodes, dtype=self.keys.dtype, device=d)
            t["CO"] = torch.empty(cap_nodes, dtype=torch.int32, device=d)
            t["LO"] = torch.empty(self.levels + 2, dtype=torch.int32, device=d)
            t["leaf_to_node"] = torch.empty(max(self.cap, 1), dtype=torch.int32, device=d)
            t["parent"] = torch.empty(max(cap_nodes // 8, 1), dtype=torch.int32, device=d)
            t["counts"] = torch.empty(cap_nodes, dtype=torch.int32, device=d)
        return t


def build_octree(x, y, z, curve: int = HILBERT, ncrit: int = 64, box=None, masses=None, buffers=None,
                 warm_leaves=None, max_iters: int = 64, stream=None, levels: int = LEVELS):
    """Full build: keys -> sort -> cornerstone leaves -> linked octree -> node counts
    (-> multipoles when ``masses`` is given). Coordinates are float64 CUDA tensors.

    ``box`` is a float64 tensor {lo_x, lo_y, lo_z, side} (CUDA); when None the bounding cube is
    computed on the device. ``warm_leaves`` (CUDA, n_l + 1 keys) warm-starts the leaf loop.
    ``levels``: 21 (63-bit keys in int64 tensors) or 10 (30-bit keys in int32 tensors).
    With masses, the keys and the multipole records are written in one pass
    (cstone_keys_records); a coordinate outside the box's fixed-point range is recorded in the
    error word of ``buffers.rws``.
    Returns a dict of device tensors sized to the built tree plus 'n_leaves' and 'iters'.
    """
    n = x.numel()
    if buffers is None or buffers.n != n or buffers.levels != levels:
        buffers = OctreeBuffers.allocate(n, leaf_capacity(n, ncrit), x.device, levels)
    b = buffers
    if box is None:
        cstone_bbox(x, y, z, b.box, b.ws, stream)
        box = b.box
    if masses is not None:  # keys and multipole records from one read of the coordinates
        _need(masses, torch.float32, "masses")
        if b.records is None or b.records.numel() < records_size(n):
            b.records = torch.empty(records_size(n), dtype=torch.uint8, device=b.device)
            b.rws = Workspace(b.device)
        cstone_keys_records(x, y, z, masses, box, curve, b.keys, b.records, b.rws, stream, levels)
    else:
        cstone_keys(x, y, z, box, curve, b.keys, stream, levels)
    cstone_sort(b.keys, b.sorted_keys, b.perm, b.ws, stream, levels)
    while True:
        nl0 = 0
        if warm_leaves is not None:
            nl0 = warm_leaves.numel() - 1
            if nl0 > b.cap:
                b = _grow(b, nl0)
            b.leaves[: nl0 + 1].copy_(warm_leaves)
        try:
            nl, iters = cstone_build_leaves(b.sorted_keys, ncrit, b.leaves, b.counts, b.offsets, nl0, max_iters,
                                            b.ws, stream, levels)
            break
        except CstoneError as e:
            if e.status != ERR_CAPACITY:
                raise
            b = _grow(b, max(getattr(e, "required", 0), 2 * b.cap))
    t = b.tree_buffers(nl)
    nn = n_nodes(nl)
    cstone_link_tree(b.leaves, nl, t["NK"], t["CO"], t["LO"], t["leaf_to_node"], t["parent"], b.ws, stream, levels)
    cstone_upsweep_counts(b.counts, nl, t["leaf_to_node"], t["CO"], t["LO"], t["counts"], b.ws, stream, levels)
    out = {
        "buffers": b, "box": box, "keys": b.keys, "sorted_keys": b.sorted_keys, "perm": b.perm,
        "leaves": b.leaves[: nl + 1], "leaf_counts": b.counts[:nl], "leaf_offsets": b.offsets[: nl + 1],
        "n_leaves": nl, "iters": iters, "NK": t["NK"][:nn], "CO": t["CO"][:nn], "LO": t["LO"],
        "leaf_to_node": t["leaf_to_node"][:nl], "parent": t["parent"][: (nn - 1) // 8], "node_counts": t["counts"][:nn],
    }
    if masses is not None:
        if "mass" not in t or t["mass"].numel() < nn:
            cap_nodes = t["cap_nodes"]
            t["mass"] = torch.empty(cap_nodes, dtype=torch.float32, device=b.device)
            t["com"] = torch.empty(3 * cap_nodes, dtype=torch.float64, device=b.device)
            t["quad"] = torch.empty(6 * cap_nodes, dtype=torch.float32, device=b.device)
        mass, com, quad = t["mass"][:nn], t["com"][: 3 * nn], t["quad"][: 6 * nn]
        cstone_upsweep_multipoles_records(b.records, b.perm, n, b.offsets, nl, t["leaf_to_node"], t["CO"], t["LO"],
                                          box, mass, com, quad, b.ws, stream, levels)
        out.update({"mass": mass, "com": com.view(3, nn), "quad": quad.view(6, nn)})
    return out


# ------------------------------------------------------------------------- batched sets
def cstone_bbox_batched(x, y, z, set_offsets, boxes, stream=None):
    _check(load().cstone_bbox_batched(_ptr(x), _ptr(y), _ptr(z), _ptr(set_offsets), set_offsets.numel() - 1,
                                      _ptr(boxes), _stream(stream)), "cstone_bbox_batched")


def cstone_keys_batched(x, y, z, set_offsets, boxes, curve: int, keys, ws: Workspace, stream=None):
    lib = load()
    s = set_offsets.numel() - 1
    buf = ws.get(_size(lib.cstone_keys_batched_workspace_size, s))
    _check(lib.cstone_keys_batched(_ptr(x), _ptr(y), _ptr(z), x.numel(), _ptr(set_offsets), s, _ptr(boxes), curve,
                                   _ptr(keys), _ptr(buf), buf.numel(), _stream(stream)), "cstone_keys_batched")


def cstone_sort_segmented(keys_in, keys_out, perm, seg_offsets, ws: Workspace, stream=None):
    lib = load()
    n, s = keys_in.numel(), seg_offsets.numel() - 1
    buf = ws.get(_size(lib.cstone_sort_segmented_workspace_size, n, s))
    _check(lib.cstone_sort_segmented(_ptr(keys_in), _ptr(keys_out), _ptr(perm), n, _ptr(seg_offsets), s, _ptr(buf),
                                     buf.numel(), _stream(stream)), "cstone_sort_segmented")


def cstone_build_leaves_batched(sorted_keys, set_offsets, ncrit: int, elements, element_offsets, counts,
                                offsets=None, n_elements: int = 0, max_iters: int = 64, ws: Workspace | None = None,
                                stream=None):
    """Returns (n_elements, iterations)."""
    lib = load()
    ws = ws or Workspace(sorted_keys.device)
    cap = elements.numel()
    buf = ws.get(_size(lib.cstone_leaves_batched_workspace_size, cap, max_iters))
    ne = ctypes.c_int64(n_elements)
    it = ctypes.c_int32(0)
    rc = lib.cstone_build_leaves_batched(_ptr(sorted_keys), sorted_keys.numel(), _ptr(set_offsets),
                                         set_offsets.numel() - 1, ncrit, _ptr(elements), cap, _ptr(element_offsets),
                                         ctypes.byref(ne), _ptr(counts), _ptr(offsets), max_iters, ctypes.byref(it),
                                         _ptr(buf), buf.numel(), _stream(stream))
    if rc == ERR_CAPACITY:
        err = CstoneError(rc, "cstone_build_leaves_batched", _detail())
        err.required = int(ne.value)
        raise err
    _check(rc, "cstone_build_leaves_batched")
    return int(ne.value), int(it.value)


def cstone_build_leaves_batched_async(sorted_keys, set_offsets, ncrit: int, elements, element_offsets, counts,
                                      offsets=None, warm: bool = False, max_iters: int = 64,
                                      ws: Workspace | None = None, stream=None):
    """Batched leaf loop without host synchronisation (capturable in a CUDA graph); the outcome is
    read afterwards with cstone_leaves_result on the same workspace."""
    lib = load()
    ws = ws or Workspace(sorted_keys.device)
    cap = elements.numel()
    buf = ws.get(_size(lib.cstone_leaves_batched_workspace_size, cap, max_iters))
    _check(lib.cstone_build_leaves_batched_async(_ptr(sorted_keys), sorted_keys.numel(), _ptr(set_offsets),
                                                 set_offsets.numel() - 1, ncrit, _ptr(elements), cap,
                                                 _ptr(element_offsets), 1 if warm else 0, _ptr(counts), _ptr(offsets),
                                                 max_iters, _ptr(buf), buf.numel(), _stream(stream)),
           "cstone_build_leaves_batched_async")


def cstone_leaves_result(ws: Workspace, elem_cap: int, max_iters: int = 64, stream=None):
    """(n_elements, iterations) of the last asynchronous batched leaf loop on ``ws``; raises
    CstoneError (with ``required`` on a capacity overflow) if it failed."""
    lib = load()
    ne = ctypes.c_int64(0)
    it = ctypes.c_int32(0)
    rc = lib.cstone_leaves_result(_ptr(ws.buf), elem_cap, max_iters, _stream(stream), ctypes.byref(ne),
                                  ctypes.byref(it))
    if rc == ERR_CAPACITY:
        err = CstoneError(rc, "cstone_build_leaves_batched_async", _detail())
        err.required = int(ne.value)
        raise err
    _check(rc, "cstone_build_leaves_batched_async")
    return int(ne.value), int(it.value)


def cstone_link_tree_batched(elements, n_elements: int, element_offsets, n_nodes: int, node_keys, child,
                             level_offsets, leaf_to_node, ws: Workspace | None = None, stream=None):
    lib = load()
    ws = ws or Workspace(elements.device)
    s = element_offsets.numel() - 1
    buf = ws.get(_size(lib.cstone_link_batched_workspace_size, n_elements, s))
    _check(lib.cstone_link_tree_batched(_ptr(elements), n_elements, _ptr(element_offsets), s, n_nodes,
                                        _ptr(node_keys), _ptr(child), _ptr(level_offsets), _ptr(leaf_to_node),
                                        _ptr(buf), buf.numel(), _stream(stream)), "cstone_link_tree_batched")


def cstone_upsweep_counts_batched(elem_counts, n_elements: int, leaf_to_node, child, level_offsets, n_sets: int,
                                  node_counts, ws: Workspace | None = None, stream=None):
    lib = load()
    ws = ws or Workspace(elem_counts.device)
    buf = ws.get(_size(lib.cstone_upsweep_workspace_size, 1))
    _check(lib.cstone_upsweep_counts_batched(_ptr(elem_counts), n_elements, _ptr(leaf_to_node), _ptr(child),
                                             _ptr(level_offsets), n_sets, _ptr(node_counts), _ptr(buf), buf.numel(),
                                             _stream(stream)), "cstone_upsweep_counts_batched")


def batched_capacity(n: int, n_sets: int, ncrit: int) -> int:
    """Element capacity of a first batched build (grown if the trees need more)."""
    return max(4 * n_sets, 16 * (n // (ncrit + 1)) + 2 * n_sets + 4096)


@dataclass
class BatchBuffers:
    """Device buffers of cstone_build_batched at an element capacity (node capacity
    elem_cap + elem_cap / 7 + S), reusable by later builds of the same sets."""
    n: int
    n_sets: int
    elem_cap: int
    node_cap: int
    t: dict

    @classmethod
    def allocate(cls, n: int, n_sets: int, elem_cap: int, device, keep=None):
        d = torch.device(device)
        node_cap = elem_cap + elem_cap // 7 + n_sets
        t = {} if keep is None else {k: keep.t[k] for k in ("boxes", "keys", "sorted_keys", "perm", "element_offsets",
                                                             "LO")}
        if keep is None:
            t["boxes"] = torch.empty((n_sets, 4), dtype=torch.float64, device=d)
            t["keys"] = torch.empty(max(n, 1), dtype=torch.int64, device=d)
            t["sorted_keys"] = torch.empty(max(n, 1), dtype=torch.int64, device=d)
            t["perm"] = torch.empty(max(n, 1), dtype=torch.int32, device=d)
            t["element_offsets"] = torch.empty(n_sets + 1, dtype=torch.int64, device=d)
            t["LO"] = torch.empty((n_sets, LEVELS + 2), dtype=torch.int32, device=d)
        t["elements"] = torch.empty(elem_cap, dtype=torch.int64, device=d)
        t["leaf_counts"] = torch.empty(elem_cap, dtype=torch.int32, device=d)
        t["leaf_offsets"] = torch.empty(elem_cap, dtype=torch.int32, device=d)
        t["leaf_to_node"] = torch.empty(elem_cap, dtype=torch.int32, device=d)
        t["NK"] = torch.empty(node_cap, dtype=torch.int64, device=d)
        t["CO"] = torch.empty(node_cap, dtype=torch.int32, device=d)
        t["node_counts"] = torch.empty(node_cap, dtype=torch.int32, device=d)
        return cls(n=n, n_sets=n_sets, elem_cap=elem_cap, node_cap=node_cap, t=t)

    def c_struct(self) -> _BatchBuffers:
        t = self.t
        return _BatchBuffers(t["boxes"].data_ptr(), t["keys"].data_ptr(), t["sorted_keys"].data_ptr(),
                             t["perm"].data_ptr(), t["elements"].data_ptr(), self.elem_cap,
                             t["element_offsets"].data_ptr(), t["leaf_counts"].data_ptr(),
                             t["leaf_offsets"].data_ptr(), t["NK"].data_ptr(), t["CO"].data_ptr(),
                             t["LO"].data_ptr(), t["leaf_to_node"].data_ptr(), t["node_counts"].data_ptr(),
                             self.node_cap)


def cstone_build_batched(x, y, z, set_offsets, bufs: BatchBuffers, curve: int, ncrit: int, boxes=None,
                         warm: bool = False, max_iters: int = 64, ws: Workspace | None = None, stream=None):
    """The whole batched build in one C call (no host synchronisation; capturable in a CUDA graph).
    ``boxes`` [S, 4] or None (bounding cubes into bufs.t["boxes"]); ``warm``: bufs' elements and
    element offsets hold the previous arrays. Read the outcome with cstone_build_batched_result."""
    lib = load()
    for t, nm in ((x, "x"), (y, "y"), (z, "z")):
        _need(t, torch.float64, nm)
    _need(set_offsets, torch.int64, "set_offsets")
    s = set_offsets.numel() - 1
    if s != bufs.n_sets or x.numel() != bufs.n:
        raise ValueError("the buffers were allocated for other sets")
    if boxes is not None:
        _need(boxes, torch.float64, "boxes")
    ws = ws or Workspace(x.device)
    buf = ws.get(_size(lib.cstone_build_batched_workspace_size, x.numel(), s, bufs.elem_cap, max_iters))
    inp = _BatchInput(x.data_ptr(), y.data_ptr(), z.data_ptr(), x.numel(), set_offsets.data_ptr(), s,
                      boxes.data_ptr() if boxes is not None else None)
    prm = _BatchParams(curve, ncrit, max_iters, 1 if warm else 0)
    out = bufs.c_struct()
    _check(lib.cstone_build_batched(ctypes.byref(inp), ctypes.byref(prm), ctypes.byref(out), _ptr(buf), buf.numel(),
                                    _stream(stream)), "cstone_build_batched")
    return ws


def cstone_build_batched_result(ws: Workspace, bufs: BatchBuffers, max_iters: int = 64, stream=None):
    """(n_elements, n_nodes, iterations) of the last cstone_build_batched on ``ws``; raises
    CstoneError (with ``required`` on a capacity overflow) if it failed."""
    lib = load()
    ne, nn, it = ctypes.c_int64(0), ctypes.c_int64(0), ctypes.c_int32(0)
    rc = lib.cstone_build_batched_result(_ptr(ws.buf), bufs.n, bufs.n_sets, bufs.elem_cap, max_iters,
                                         _ptr(bufs.t["LO"]), _stream(stream), ctypes.byref(ne), ctypes.byref(nn),
                                         ctypes.byref(it))
    if rc == ERR_CAPACITY:
        err = CstoneError(rc, "cstone_build_batched", _detail())
        err.required = int(ne.value)
        raise err
    _check(rc, "cstone_build_batched")
    return int(ne.value), int(nn.value), int(it.value)


def _batched_result(bufs: BatchBuffers, ne: int, nn: int, iters: int, ws) -> dict:
    """Result dict of a batched build: device tensors cut to the built sizes, and host copies of the
    element and node offsets (read from the device)."""
    t = bufs.t
    eo_host = t["element_offsets"].cpu().tolist()
    node_offsets = t["LO"][:, 0].cpu().tolist() + [nn]
    return {"boxes": t["boxes"], "keys": t["keys"][: bufs.n], "sorted_keys": t["sorted_keys"][: bufs.n],
            "perm": t["perm"][: bufs.n], "elements": t["elements"][:ne], "n_elements": ne,
            "element_offsets": t["element_offsets"], "element_offsets_host": eo_host,
            "leaf_counts": t["leaf_counts"][:ne], "leaf_offsets": t["leaf_offsets"][:ne], "iters": iters,
            "NK": t["NK"][:nn], "CO": t["CO"][:nn], "LO": t["LO"], "leaf_to_node": t["leaf_to_node"][:ne],
            "node_counts": t["node_counts"][:nn], "node_offsets_host": node_offsets, "ws": ws, "buffers": bufs}


def build_octrees_batched(x, y, z, set_offsets, curve: int = MORTON, ncrit: int = 32, boxes=None, warm=None,
                          max_iters: int = 64, ws: Workspace | None = None, stream=None, buffers=None):
    """Octrees of many independent sets stored back to back, one launch per phase for all sets
    (the single C call cstone_build_batched, then one read of its outcome).

    ``set_offsets``: int64 CUDA tensor of S+1 particle offsets. ``boxes``: float64 CUDA tensor [S, 4]
    (bounding cubes are computed when None). ``warm``: a previous result of this function for the
    same sets (its elements and element offsets warm-start the leaf loop). ``buffers``: a
    BatchBuffers to reuse. Returns a dict with the concatenated per-set outputs and host copies of
    the element and node offsets."""
    dev = x.device
    n = x.numel()
    s = set_offsets.numel() - 1
    ws = ws or Workspace(dev)
    cap = batched_capacity(n, s, ncrit)
    if warm is not None:
        cap = max(cap, 2 * warm["n_elements"])
    bufs = buffers if (buffers is not None and buffers.n == n and buffers.n_sets == s and buffers.elem_cap >= cap) \
        else BatchBuffers.allocate(n, s, cap, dev)
    while True:
        if warm is not None:
            ne0 = warm["n_elements"]
            if warm["elements"].data_ptr() != bufs.t["elements"].data_ptr():
                bufs.t["elements"][:ne0].copy_(warm["elements"][:ne0])
            if warm["element_offsets"].data_ptr() != bufs.t["element_offsets"].data_ptr():
                bufs.t["element_offsets"].copy_(warm["element_offsets"])
        cstone_build_batched(x, y, z, set_offsets, bufs, curve, ncrit, boxes=boxes, warm=warm is not None,
                             max_iters=max_iters, ws=ws, stream=stream)
        try:
            ne, nn, iters = cstone_build_batched_result(ws, bufs, max_iters, stream)
            break
        except CstoneError as e:
            if e.status != ERR_CAPACITY:
                raise
            if warm is not None and warm["elements"].data_ptr() == bufs.t["elements"].data_ptr():
                warm = None  # the failed loop left root arrays in place of the warm ones: start cold
            bufs = BatchBuffers.allocate(n, s, max(2 * bufs.elem_cap, getattr(e, "required", 0) + 1024), dev,
                                         keep=bufs)
    out = _batched_result(bufs, ne, nn, iters, ws)
    if boxes is not None:
        out["boxes"] = boxes
    return out


def _grow(b: OctreeBuffers, want: int) -> OctreeBuffers:
    cap = int(min(1 << 28, max(want, 2 * b.cap)))
    nb = OctreeBuffers.allocate(b.n, cap, b.device, b.levels)
    nb.keys, nb.sorted_keys, nb.perm, nb.box, nb.ws = b.keys, b.sorted_keys, b.perm, b.box, b.ws
    nb.records, nb.rws = b.records, b.rws
    return nb


# ------------------------------------------------------------------------- host-resident input
class StreamedBuilder:
    """Full builds (as ``build_octree``, with multipoles) of a sequence of particle sets held in
    pinned host memory, with the host<->device transfers overlapped with the builds: the C entry
    points cstone_host_stage (copy-in) and cstone_host_build (build and copy-out) on two device
    slots and three CUDA streams. While set k is built on the compute stream, set k+1 is copied in
    on the copy-in stream and set k-1's tree is copied out on the copy-out stream (the link carries
    both directions at once); the slots' events order every reuse of their memory. The results are
    pinned host tensors, valid once ``run`` returns (or, for set k, once its copy-out event has
    completed). 63-bit keys. ``leaf_cap`` (default: the bound of ``leaf_capacity``) sizes the slots;
    a tree that needs more leaves raises CstoneError (ERR_CAPACITY) from ``run``.
    """

    OUT = ("leaves", "leaf_counts", "NK", "CO", "LO", "node_counts", "mass", "com", "quad")

    def __init__(self, n: int, device="cuda", curve: int = HILBERT, ncrit: int = 64, levels: int = LEVELS,
                 leaf_cap: int | None = None, max_iters: int = 64):
        if levels != LEVELS:
            raise ValueError("StreamedBuilder builds 63-bit keys (levels = 21)")
        lib = load()
        self.n, self.curve, self.ncrit, self.levels, self.max_iters = n, curve, ncrit, levels, max_iters
        self.device = torch.device(device)
        self.cap = leaf_cap if leaf_cap is not None else leaf_capacity(n, ncrit)
        self.node_cap = self.cap + (self.cap - 1) // 7
        self.s_comp = torch.cuda.Stream(self.device)
        self.s_in = torch.cuda.Stream(self.device)
        self.s_out = torch.cuda.Stream(self.device)
        nbytes = _size(lib.cstone_host_workspace_size, n, self.cap, 1)
        self.slots, self.events, self.ws, self.host = [], [], [], []
        for _ in range(2):
            ws = torch.empty(max(nbytes, 256), dtype=torch.uint8, device=self.device)
            evs = [torch.cuda.Event() for _ in range(4)]  # staged, inputs_read, built, copied_out
            for e in evs:  # creates the events (completed) so that their handles exist
                e.record(self.s_comp)
            self.ws.append(ws)
            self.events.append(evs)
            self.slots.append(_HostSlot(ws.data_ptr(), nbytes, *(e.cuda_event for e in evs)))
            cap, nc = self.cap, self.node_cap
            pin = lambda k, dt: torch.empty(max(k, 1), dtype=dt, pin_memory=True)  # noqa: E731
            self.host.append({"leaves": pin(cap + 1, torch.int64), "leaf_counts": pin(cap, torch.int32),
                              "NK": pin(nc, torch.int64), "CO": pin(nc, torch.int32),
                              "LO": pin(LEVELS + 2, torch.int32), "node_counts": pin(nc, torch.int32),
                              "mass": pin(nc, torch.float32), "com": pin(3 * nc, torch.float64),
                              "quad": pin(6 * nc, torch.float32)})
        self.s_comp.synchronize()

    def _tree(self, slot: int) -> _HostTree:
        h = self.host[slot]
        return _HostTree(*(h[k].data_ptr() for k in self.OUT), 0, 0, 0)

    def _stage(self, slot: int, src):
        x, y, z, m = src
        _check(load().cstone_host_stage(_ptr(x), _ptr(y), _ptr(z), _ptr(m), self.n, self.cap,
                                        ctypes.byref(self.slots[slot]), _stream(self.s_in)), "cstone_host_stage")

    def _build(self, slot: int) -> dict:
        lib = load()
        tree = self._tree(slot)
        rc = lib.cstone_host_build(self.n, self.cap, 1, self.curve, self.ncrit, self.max_iters,
                                   ctypes.byref(self.slots[slot]), ctypes.byref(tree), _stream(self.s_comp),
                                   _stream(self.s_out))
        _check(rc, "cstone_host_build")
        nl, nn = int(tree.n_leaves), int(tree.n_nodes)
        h = self.host[slot]
        sizes = {"leaves": nl + 1, "leaf_counts": nl, "NK": nn, "CO": nn, "LO": LEVELS + 2, "node_counts": nn,
                 "mass": nn, "com": 3 * nn, "quad": 6 * nn}
        res = {k: h[k][: sizes[k]] for k in self.OUT}
        res["n_leaves"], res["iters"] = nl, int(tree.iters)
        return res

    def status(self, slot: int) -> int:
        """Device errors recorded by the last build on ``slot`` (raises CstoneError)."""
        _check(load().cstone_host_status(self.n, self.cap, 1, ctypes.byref(self.slots[slot]), _stream(self.s_comp)),
               "cstone_host_status")
        return 0

    def run(self, sets, on_result=None, events=None, build_starts=None):
        """Builds every (x, y, z, m) of ``sets`` (pinned host tensors: float64 coordinates, float32
        masses, n particles each). Returns the number of bytes copied in and out; ``on_result(k,
        result)`` receives set k's host result dict once its copy-out has completed (a result's
        tensors are reused two sets later). ``events`` = (start, stop) CUDA events, recorded before
        the first copy-in and after the last copy-out. ``build_starts``, a list, receives one timing
        event per set, recorded on the compute stream ahead of the set's build."""
        sets = list(sets)
        for src in sets:
            if (len(src) != 4 or any(t.numel() != self.n or t.is_cuda or not t.is_contiguous() for t in src)
                    or any(t.dtype != torch.float64 for t in src[:3]) or src[3].dtype != torch.float32):
                raise ValueError("every set is (x, y, z, m) contiguous host tensors of n particles "
                                 "(float64 coordinates, float32 masses)")
        h2d = d2h = 0
        pending = []
        if events is not None:
            events[0].record(self.s_in)
        if sets:
            self._stage(0, sets[0])
        for k in range(len(sets)):
            slot = k % 2
            if k + 1 < len(sets):
                self._stage((k + 1) % 2, sets[k + 1])  # queued before this build's host synchronisation
            if build_starts is not None:
                ev = torch.cuda.Event(enable_timing=True)
                ev.record(self.s_comp)
                build_starts.append(ev)
            res = self._build(slot)
            if events is not None and k + 1 == len(sets):
                events[1].record(self.s_out)
            h2d += sum(t.numel() * t.element_size() for t in sets[k])
            d2h += sum(res[k2].numel() * res[k2].element_size() for k2 in self.OUT)
            pending.append((k, slot, res))
            while pending and (len(pending) > 1 or k + 1 == len(sets)):
                kk, sl, r = pending.pop(0)
                self.events[sl][3].synchronize()  # the slot's tree is on the host
                if on_result is not None:
                    on_result(kk, r)
        return h2d, d2h


# ------------------------------------------------------------------------- time steps
def padded_boxes(boxes, pad: float = 0.1):
    """Each bounding cube grown by `pad` of its side on every side (boxes [S, 4], float64 CUDA)."""
    out = boxes.clone()
    out[:, :3] -= pad * boxes[:, 3:4]
    out[:, 3] *= 1.0 + 2.0 * pad
    return out


class TimeStepper:
    """Rebuilds the octrees of several independent runs after every step of a particle simulation.

    The runs are stored back to back (``set_offsets``); each rebuild is one batched build of all
    runs in a box fixed at step 0, warm-started from the previous step's leaf arrays (Sec. 4: a
    single f/g update per step keeps a slowly moving distribution balanced)."""

    def __init__(self, x, y, z, set_offsets, curve: int = HILBERT, ncrit: int = 64, pad: float = 0.1):
        self.x, self.y, self.z, self.set_offsets = x, y, z, set_offsets
        self.curve, self.ncrit = curve, ncrit
        self.ws = Workspace(x.device)
        cube = torch.empty((set_offsets.numel() - 1, 4), dtype=torch.float64, device=x.device)
        cstone_bbox_batched(x, y, z, set_offsets, cube)
        self.boxes = padded_boxes(cube, pad)
        self.last = None

    def rebuild(self, warm: bool = True):
        prev = self.last
        out = build_octrees_batched(self.x, self.y, self.z, self.set_offsets, curve=self.curve, ncrit=self.ncrit,
                                    boxes=self.boxes, warm=prev if warm else None, ws=self.ws,
                                    buffers=prev["buffers"] if prev is not None else None)
        self.last = out
        return out


class GraphTimeStepper:
    """Time-step driver whose whole rebuild (keys, segmented sort, warm-started batched leaf loop,
    linked octrees, node counts: the one C call cstone_build_batched) is one CUDA graph, replayed
    once per step.

    Every buffer is allocated at a capacity (``elem_cap`` elements over all runs; the node arrays
    hold elem_cap + elem_cap / 7 + S nodes), the leaf loop takes its warm-start count from the
    device, and the link and count phases run on the capacities with the exact counts on the
    device, so no phase needs the host between the launches. After each replay one read-back
    (cstone_build_batched_result) fetches the outcome. The capacity is never below the batched
    builder's first estimate (``elem_cap`` raises it, never lowers it). The first rebuild (cold,
    from the roots) runs without the graph; the warm rebuild is captured on its first use. A
    capacity overflow grows the capacity, drops the graph and rebuilds cold."""

    def __init__(self, x, y, z, set_offsets, curve: int = HILBERT, ncrit: int = 64, pad: float = 0.1,
                 elem_cap: int | None = None, max_iters: int = 64):
        dev = x.device
        self.device = dev
        self.x, self.y, self.z, self.set_offsets = x, y, z, set_offsets
        self.curve, self.ncrit, self.max_iters = curve, ncrit, max_iters
        n, s = x.numel(), set_offsets.numel() - 1
        self.n, self.n_sets = n, s
        cube = torch.empty((s, 4), dtype=torch.float64, device=dev)
        cstone_bbox_batched(x, y, z, set_offsets, cube)
        self.boxes = padded_boxes(cube, pad)
        self.fixed_cap = elem_cap is not None
        self.ws = Workspace(dev)
        # never below the estimate the batched builder starts from, so that a cold build does not
        # overflow its capacity in practice
        self.min_cap = batched_capacity(n, s, ncrit)
        self.bufs = BatchBuffers.allocate(n, s, max(elem_cap or 0, self.min_cap), dev)
        self.graph = None
        self.have_arrays = False

    @property
    def elem_cap(self) -> int:
        return self.bufs.elem_cap

    def _grow(self, cap: int):
        self.bufs = BatchBuffers.allocate(self.n, self.n_sets, int(cap), self.device, keep=self.bufs)
        self.graph = None

    def _launch(self, warm: bool):
        cstone_build_batched(self.x, self.y, self.z, self.set_offsets, self.bufs, self.curve, self.ncrit,
                             boxes=self.boxes, warm=warm, max_iters=self.max_iters, ws=self.ws)

    def _result(self):
        ne, nn, iters = cstone_build_batched_result(self.ws, self.bufs, self.max_iters)
        out = _batched_result(self.bufs, ne, nn, iters, self.ws)
        out["boxes"] = self.boxes
        return out

    def _cold(self):
        # from the roots, outside any graph; an overflow grows the capacity and starts again
        while True:
            self._launch(False)
            try:
                out = self._result()
                break
            except CstoneError as e:
                if e.status != ERR_CAPACITY:
                    raise
                self._grow(max(2 * self.elem_cap, getattr(e, "required", 0) + 1024))
        ne = out["n_elements"]
        tight = max(2 * ne + 64 * self.n_sets + 4096, self.min_cap)
        if not self.fixed_cap and tight < self.elem_cap:
            old = self.bufs
            self.bufs = BatchBuffers.allocate(self.n, self.n_sets, tight, self.device, keep=old)
            self.bufs.t["elements"][:ne].copy_(old.t["elements"][:ne])  # the warm start of the next step
            self.graph = None
            # the tree outputs stay in the old buffers (returned as they are); the elements, which
            # the next warm step reads in place, now live in the new ones
            out = dict(out, elements=self.bufs.t["elements"][:ne])
        self.have_arrays = True
        return out

    def rebuild(self, warm: bool = True):
        if not warm or not self.have_arrays:
            return self._cold()
        if self.graph is None:
            self._launch(True)  # sizes the workspace before the capture
            try:
                self._result()
            except CstoneError as e:
                if e.status != ERR_CAPACITY:
                    raise
                self._grow(max(2 * self.elem_cap, getattr(e, "required", 0) + 1024))
                return self._cold()  # the failed pass left root arrays: start again from the roots
            self.graph = torch.cuda.CUDAGraph()
            with torch.cuda.graph(self.graph, capture_error_mode="thread_local"):
                self._launch(True)
        self.graph.replay()
        try:
            return self._result()
        except CstoneError as e:
            if e.status != ERR_CAPACITY:
                raise
            self._grow(max(2 * self.elem_cap, getattr(e, "required", 0) + 1024))
            return self._cold()
