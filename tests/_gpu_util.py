"""Helpers shared by the GPU parity tests (not collected by pytest)."""
import numpy as np
import torch

L = 21
KEY_END = 1 << 63


def dev(a, dtype=None):
    """numpy -> CUDA tensor (uint64 / uint32 are carried as int64 / int32 bit patterns)."""
    a = np.ascontiguousarray(a)
    if a.dtype == np.uint64:
        a = a.view(np.int64)
    elif a.dtype == np.uint32:
        a = a.view(np.int32)
    t = torch.from_numpy(a)
    if dtype is not None:
        t = t.to(dtype)
    return t.cuda()


def u64(t) -> np.ndarray:
    return t.detach().cpu().numpy().view(np.uint64)


def u32(t) -> np.ndarray:
    return t.detach().cpu().numpy().view(np.uint32)


def i32(t) -> np.ndarray:
    return t.detach().cpu().numpy().astype(np.int64)


def node_level(nk) -> np.ndarray:
    """Level of each placeholder node key (1 << 3 level) | prefix: the number of levels l >= 1 with
    key >= 1 << 3l (exact integer comparisons)."""
    nk = np.asarray(nk, np.uint64)
    lev = np.zeros(nk.shape, np.int64)
    for lv in range(1, L + 1):
        lev += nk >= np.uint64(1 << (3 * lv))
    return lev


def multipole_errors(M_ref, com_ref, q_ref, M, com, q, node_side):
    """Per-moment error metrics over non-empty nodes.

    mass: |dM| / M; centre: max-norm |d com| / node side; quadrupole: max_ab |dQ_ab| / max_ab |Q_ab|
    (normwise, relative to the largest component; the denominator is floored at 1e-12 M side^2 so
    that nodes whose particles coincide, where the FP64 reference is rounding noise, stay defined).
    Empty nodes must be exactly zero."""
    nz = M_ref > 0
    if not nz.any():
        return {"mass": 0.0, "com": 0.0, "quad": 0.0}
    e_m = np.max(np.abs(M[nz] - M_ref[nz]) / M_ref[nz])
    e_c = np.max(np.max(np.abs(com[nz] - com_ref[nz]), axis=1) / node_side[nz])
    qn = np.maximum(np.max(np.abs(q_ref), axis=1), 1e-12 * M_ref * node_side ** 2)
    dq = np.max(np.abs(q - q_ref), axis=1)
    e_q = np.max(dq[nz] / qn[nz])
    empty = ~nz
    assert np.all(M[empty] == 0) and np.all(com[empty] == 0) and np.all(q[empty] == 0)
    return {"mass": float(e_m), "com": float(e_c), "quad": float(e_q)}
