"""cstone_sort_static: the sort entry point for callers that cannot allocate device memory.

Code running inside a memory allocator's callbacks, or inside a framework that owns every byte of
device memory, cannot call cudaMalloc or hand the library a workspace. cstone_sort_static serves
them from a static scratch array inside the library. This file runs last so that a failure here
comes after every other test; it must pass alone in a fresh process as well as after the others.
The new entry point is called through the C ABI and compared with the workspace-based
cstone_sort bit for bit (the sort is integer work), on two calls in a row that share the array.
"""
import ctypes

import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu

LIMIT = 1 << 20


def _keys(seed, n):
    rng = np.random.default_rng(seed)
    k = rng.integers(0, 1 << 63, n, dtype=np.uint64)
    k[rng.integers(0, n, n // 4)] = k[0]  # plenty of equal keys: stability matters
    return torch.from_numpy(k.view(np.int64)).cuda()


def test_static_sort_matches_workspace_sort_on_consecutive_calls(lib):
    clib = lib.load()
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    ws = lib.Workspace()
    for call, n in enumerate((300_001, LIMIT)):  # two calls in a row; the second at the size limit
        kin = _keys(100 + call, n)
        ref_keys, ref_perm = torch.empty_like(kin), torch.empty(n, dtype=torch.int32, device="cuda")
        lib.cstone_sort(kin, ref_keys, ref_perm, ws)
        out_keys = torch.full_like(kin, -1)
        out_perm = torch.full((n,), -1, dtype=torch.int32, device="cuda")
        rc = clib.cstone_sort_static(ctypes.c_void_p(kin.data_ptr()), ctypes.c_void_p(out_keys.data_ptr()),
                                     ctypes.c_void_p(out_perm.data_ptr()), n, stream)
        assert rc == lib.OK
        torch.cuda.synchronize()
        assert torch.equal(out_keys, ref_keys), f"keys differ on call {call}"
        assert torch.equal(out_perm, ref_perm), f"permutation differs on call {call}"


def test_static_sort_rejects_sizes_beyond_its_scratch(lib):
    clib = lib.load()
    dummy = ctypes.c_void_p(256)
    assert clib.cstone_sort_static(dummy, dummy, dummy, LIMIT + 1, None) == lib.ERR_INVALID_ARG
    buf = ctypes.create_string_buffer(512)
    clib.cstone_last_error_detail(buf, 512)
    assert b"static scratch limit" in buf.value
