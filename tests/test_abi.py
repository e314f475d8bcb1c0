"""The C-ABI library builds, loads and exports every entry point declared in include/cstone.h.
Host-side argument checks and workspace-size queries run without a GPU (no kernel is launched)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "cstone.h")


@pytest.fixture(scope="module")
def clib():
    import paper_2307_06345_gb300 as cs
    cs.build()
    return cs.load()


def declared_symbols():
    text = open(HEADER).read()
    return sorted(set(re.findall(r"CSTONE_API\s+[\w\s\*]*?\b(cstone_\w+)\s*\(", text)))


def test_header_declares_the_path():
    syms = declared_symbols()
    for name in ("cstone_keys", "cstone_sort", "cstone_build_leaves", "cstone_link_tree", "cstone_upsweep_counts",
                 "cstone_upsweep_multipoles", "cstone_bbox"):
        assert name in syms


def test_every_declared_symbol_is_exported(clib):
    for name in declared_symbols():
        assert hasattr(clib, name), name


def test_status_strings(clib):
    for code in range(6):
        s = clib.cstone_status_string(code)
        assert s and s.decode()
    assert clib.cstone_status_string(99).decode() == "unknown status"
    assert clib.cstone_version() >= 100
    clib.cstone_kernel_launches.restype = ctypes.c_int64
    assert clib.cstone_kernel_launches() >= 0


def test_workspace_queries_and_argument_checks(clib):
    sz = ctypes.c_size_t()
    assert clib.cstone_sort_workspace_size(1 << 20, ctypes.byref(sz)) == 0
    # the sort needs the alternate key/value buffers (12 bytes per key) plus the per-tile digit counts and offsets
    assert sz.value >= 12 * (1 << 20)
    assert clib.cstone_sort_workspace_size(-1, ctypes.byref(sz)) == 1
    assert clib.cstone_sort_workspace_size(1 << 30, ctypes.byref(sz)) == 1
    assert clib.cstone_leaves_workspace_size(1000, 100, 64, ctypes.byref(sz)) == 0
    assert clib.cstone_leaves_workspace_size(1000, 100, 0, ctypes.byref(sz)) == 1
    assert clib.cstone_link_workspace_size(15, ctypes.byref(sz)) == 0
    assert clib.cstone_link_workspace_size(0, ctypes.byref(sz)) == 1
    # link: n_leaves must be 1 + 7k; rejected before any device work
    dummy = ctypes.c_void_p(256)
    rc = clib.cstone_link_tree(dummy, 3, dummy, dummy, dummy, dummy, None, dummy, 1 << 20, None)
    assert rc == 1
    buf = ctypes.create_string_buffer(512)
    clib.cstone_last_error_detail(buf, 512)
    assert b"n_leaves" in buf.value
    # keys: unknown curve
    rc = clib.cstone_keys(dummy, dummy, dummy, 10, dummy, 7, dummy, None)
    assert rc == 1
    # sort: workspace too small
    rc = clib.cstone_sort(dummy, dummy, dummy, 1000, dummy, 16, None)
    assert rc == 1
    # leaves: initial leaf count beyond the capacity
    nl = ctypes.c_int64(50)
    rc = clib.cstone_build_leaves(dummy, 100, 8, dummy, 10, ctypes.byref(nl), dummy, None, 64, None, dummy, 1 << 20,
                                  None)
    assert rc == 1


def test_sort_bindings_reject_undersized_outputs(clib):
    """The Python bindings of both sorts refuse outputs smaller than the input before any launch (an
    undersized perm or keys_out would otherwise be written out of bounds)."""
    import torch

    import paper_2307_06345_gb300 as cs

    kin = torch.zeros(100, dtype=torch.int64)
    for fn in (lambda ko, p: cs.cstone_sort(kin, ko, p, None), lambda ko, p: cs.cstone_sort_static(kin, ko, p)):
        with pytest.raises(ValueError, match="at least 100"):
            fn(torch.zeros(100, dtype=torch.int64), torch.zeros(99, dtype=torch.int32))
        with pytest.raises(ValueError, match="at least 100"):
            fn(torch.zeros(50, dtype=torch.int64), torch.zeros(100, dtype=torch.int32))


def test_one_call_batched_build_checks_its_capacities(clib):
    """cstone_build_batched rejects an element capacity below 2 S and a node capacity below
    elem_cap + elem_cap / 7 + S before any device work."""
    import paper_2307_06345_gb300 as cs
    inp = cs._BatchInput(256, 256, 256, 10, 256, 3, None)
    prm = cs._BatchParams(0, 16, 64, 0)
    small_elems = cs._BatchBuffers(*([256] * 5), 4, *([256] * 8), 100)
    assert clib.cstone_build_batched(ctypes.byref(inp), ctypes.byref(prm), ctypes.byref(small_elems), None, 0,
                                     None) == 1
    small_nodes = cs._BatchBuffers(*([256] * 5), 70, *([256] * 8), 70 + 10 + 2)
    assert clib.cstone_build_batched(ctypes.byref(inp), ctypes.byref(prm), ctypes.byref(small_nodes), None, 0,
                                     None) == 1
    buf = ctypes.create_string_buffer(512)
    clib.cstone_last_error_detail(buf, 512)
    assert b"node_cap" in buf.value
    sz = ctypes.c_size_t()
    assert clib.cstone_build_batched_workspace_size(1000, 3, 70, 64, ctypes.byref(sz)) == 0 and sz.value > 0
    assert clib.cstone_build_batched_workspace_size(1000, 5000, 20000, 64, ctypes.byref(sz)) == 1  # > 4096 sets


def test_host_build_queries_and_argument_checks(clib):
    # the end-to-end entry points: workspace sizing and the checks made before any CUDA call
    import paper_2307_06345_gb300 as cs
    sz, sz_m = ctypes.c_size_t(), ctypes.c_size_t()
    n, cap = 100_000, cs.leaf_capacity(100_000, 64)
    assert clib.cstone_host_workspace_size(n, cap, 0, ctypes.byref(sz)) == 0
    assert clib.cstone_host_workspace_size(n, cap, 1, ctypes.byref(sz_m)) == 0
    # inputs (28 bytes per particle), keys, sorted keys and permutation at least; masses add the
    # 32-byte records and the node multipoles
    assert sz.value >= 48 * n and sz_m.value >= sz.value + 32 * n
    assert clib.cstone_host_workspace_size(0, cap, 1, ctypes.byref(sz)) == 1
    assert clib.cstone_host_workspace_size(n, 0, 1, ctypes.byref(sz)) == 1
    dummy = ctypes.c_void_p(256)
    slot = cs._HostSlot(256, sz_m.value, 0, 0, 0, 0)  # events missing
    assert clib.cstone_host_stage(dummy, dummy, dummy, None, n, cap, ctypes.byref(slot), None) == 1
    slot = cs._HostSlot(256, 1024, 8, 8, 8, 8)  # workspace too small
    assert clib.cstone_host_stage(dummy, dummy, dummy, None, n, cap, ctypes.byref(slot), None) == 1
    tree = cs._HostTree()
    assert clib.cstone_host_build(n, cap, 1, 1, 64, 64, ctypes.byref(slot), ctypes.byref(tree), None, None) == 1
    assert clib.cstone_host_build(n, cap, 1, 1, 64, 64, None, ctypes.byref(tree), None, None) == 1
