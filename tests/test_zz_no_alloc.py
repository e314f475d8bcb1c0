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


def test_static_sort_matches_the_oracle(lib, oracle):
    """The static sort compared with the oracle's stable sort directly, not only with cstone_sort."""
    clib = lib.load()
    n = 77_777
    kin = _keys(7, n)
    ref_keys, ref_perm = oracle.sort(kin.cpu().numpy().view(np.uint64))
    out_keys = torch.empty_like(kin)
    out_perm = torch.empty(n, dtype=torch.int32, device="cuda")
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    assert clib.cstone_sort_static(ctypes.c_void_p(kin.data_ptr()), ctypes.c_void_p(out_keys.data_ptr()),
                                   ctypes.c_void_p(out_perm.data_ptr()), n, stream) == lib.OK
    torch.cuda.synchronize()
    assert np.array_equal(out_keys.cpu().numpy().view(np.uint64), ref_keys)
    assert np.array_equal(out_perm.cpu().numpy().view(np.uint32), ref_perm)


def test_static_sort_empty_and_in_place_on_a_side_stream(lib):
    """n = 0 is a no-op; keys_out may alias keys_in (the header allows it), here on a non-default
    stream, and the result equals cstone_sort's bit for bit."""
    clib = lib.load()
    side = torch.cuda.Stream()
    sp = ctypes.c_void_p(side.cuda_stream)
    one = torch.zeros(1, dtype=torch.int64, device="cuda")
    pone = torch.zeros(1, dtype=torch.int32, device="cuda")
    assert clib.cstone_sort_static(ctypes.c_void_p(one.data_ptr()), ctypes.c_void_p(one.data_ptr()),
                                   ctypes.c_void_p(pone.data_ptr()), 0, sp) == lib.OK
    n = 123_457
    kin = _keys(11, n)
    ref_keys, ref_perm = torch.empty_like(kin), torch.empty(n, dtype=torch.int32, device="cuda")
    lib.cstone_sort(kin, ref_keys, ref_perm, lib.Workspace())
    torch.cuda.synchronize()
    inplace = kin.clone()
    perm = torch.full((n,), -1, dtype=torch.int32, device="cuda")
    torch.cuda.synchronize()
    assert clib.cstone_sort_static(ctypes.c_void_p(inplace.data_ptr()), ctypes.c_void_p(inplace.data_ptr()),
                                   ctypes.c_void_p(perm.data_ptr()), n, sp) == lib.OK
    side.synchronize()
    assert torch.equal(inplace, ref_keys)
    assert torch.equal(perm, ref_perm)


def test_static_sort_rejects_sizes_beyond_its_scratch(lib):
    clib = lib.load()
    dummy = ctypes.c_void_p(256)
    assert clib.cstone_sort_static(dummy, dummy, dummy, LIMIT + 1, None) == lib.ERR_INVALID_ARG
    buf = ctypes.create_string_buffer(512)
    clib.cstone_last_error_detail(buf, 512)
    assert b"static scratch limit" in buf.value
