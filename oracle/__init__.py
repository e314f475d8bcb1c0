"""Plain CPU oracle for the Cornerstone octree build (Keller et al., PASC'23).

TEST INFRASTRUCTURE ONLY. The test-suite, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` are the only callers; the product package never imports this module and shares no
code with it. The arithmetic lives in ``cstone_oracle.c`` (plain C, one routine per step of the
paper, double precision, no FMA contraction); this module only compiles it and marshals numpy
arrays through ctypes.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "cstone_oracle.c")
_HDR = os.path.join(_HERE, "cstone_oracle.h")
# one build of the C source per number of levels: 21 (63-bit keys) and 10 (30-bit keys)
_LIBS = {21: os.path.join(_HERE, "liboracle.so"), 10: os.path.join(_HERE, "liboracle30.so")}
_LIB = _LIBS[21]
_lock = threading.Lock()
_libs = {}

L = 21
KEY_END = 1 << 63
MORTON, HILBERT = 0, 1


def key_end(levels: int = L) -> int:
    """8^L, one past the last key."""
    return 1 << (3 * levels)


class OracleError(RuntimeError):
    pass


def build(force: bool = False) -> str:
    """Compile the oracle shared libraries in-tree (gcc, -O2 -ffp-contract=off), one per number of
    levels."""
    for levels, path in _LIBS.items():
        stale = (not os.path.exists(path)) or any(os.path.getmtime(s) > os.path.getmtime(path) for s in (_SRC, _HDR))
        if force or stale:
            tmp = path + f".tmp{os.getpid()}"
            cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fopenmp", "-fPIC", "-shared",
                   f"-DORACLE_L={levels}", "-o", tmp, _SRC, "-lm"]
            subprocess.run(cmd, check=True)
            os.replace(tmp, path)
    return _LIB


def _load(levels: int = L):
    with _lock:
        if levels not in _libs:
            if levels not in _LIBS:
                raise ValueError(f"the oracle is built for {sorted(_LIBS)} levels, not {levels}")
            build()
            lib = ctypes.CDLL(_LIBS[levels])
            P = ctypes.c_void_p
            i64, u32, i32, dbl = ctypes.c_int64, ctypes.c_uint32, ctypes.c_int, ctypes.c_double
            sigs = {
                "oracle_set_threads": (None, [i32]),
                "oracle_get_threads": (i32, []),
                "oracle_bounding_cube": (i32, [P, P, P, i64, P]),
                "oracle_grid_coord": (u32, [dbl, dbl, dbl]),
                "oracle_scale": (dbl, [dbl]),
                "oracle_morton_key": (ctypes.c_uint64, [u32, u32, u32]),
                "oracle_morton_decode": (None, [ctypes.c_uint64, P, P, P]),
                "oracle_hilbert_key_order": (ctypes.c_uint64, [u32, u32, u32, i32]),
                "oracle_hilbert_decode_order": (None, [ctypes.c_uint64, i32, P, P, P]),
                "oracle_hilbert_key": (ctypes.c_uint64, [u32, u32, u32]),
                "oracle_keys": (i32, [P, P, P, i64, P, i32, P]),
                "oracle_sort": (i32, [P, i64, P, P]),
                "oracle_lower_bound": (i64, [P, i64, ctypes.c_uint64]),
                "oracle_histogram": (i32, [P, i64, P, i64, P]),
                "oracle_rebalance_decision": (i32, [P, P, i64, u32, P]),
                "oracle_exclusive_scan": (i32, [P, i64, P]),
                "oracle_rebalance": (i32, [P, P, P, i64, P]),
                "oracle_build_leaves": (i32, [P, i64, u32, P, i64, P, i64, P, P, i32, P]),
                "oracle_canonical_leaves": (i32, [P, i64, u32, P, i64, P]),
                "oracle_check_cornerstone": (i32, [P, i64]),
                "oracle_link": (i32, [P, i64, P, P, P, P, P]),
                "oracle_cube_from_bounds": (i32, [P, P]),
                "oracle_decompose": (i32, [P, i64, i32, P]),
                "oracle_node_counts": (i32, [P, i64, P, i64, P]),
                "oracle_multipoles": (i32, [P, P, P, P, P, P, i64, P, P, i64, P, P, P]),
                "oracle_focus_tiles": (i32, [ctypes.c_uint64, ctypes.c_uint64, P, P, i32]),
                "oracle_mac_passes": (i32, [ctypes.c_uint64, i32, ctypes.c_uint64, ctypes.c_uint64, dbl, i32]),
                "oracle_focus_decision": (i32, [P, P, i64, u32, ctypes.c_uint64, ctypes.c_uint64, dbl, i32, P]),
                "oracle_build_focus_leaves": (i32, [P, i64, u32, ctypes.c_uint64, ctypes.c_uint64, dbl, i32, P, i64,
                                                    P, i64, P, P, i32, P]),
                "oracle_canonical_focus_leaves": (i32, [P, i64, u32, ctypes.c_uint64, ctypes.c_uint64, dbl, i32, P,
                                                        i64, P]),
            }
            for name, (res, args) in sigs.items():
                fn = getattr(lib, name)
                fn.restype = res
                fn.argtypes = args
            _libs[levels] = lib
    return _libs[levels]


def set_threads(threads: int = 0) -> int:
    """Threads of the oracle's parallel loops in both builds (0 = all cores, 1 = sequential);
    returns the number in effect. Results do not depend on it."""
    for levels in _LIBS:
        _load(levels).oracle_set_threads(int(threads))
    return int(_load().oracle_get_threads())


def get_threads() -> int:
    return int(_load().oracle_get_threads())


def _ptr(a: np.ndarray):
    return ctypes.c_void_p(a.ctypes.data) if a is not None else None


def _c(a, dtype):
    return np.ascontiguousarray(a, dtype=dtype)


def _check(rc: int, what: str):
    if rc != 0:
        raise OracleError(f"{what} failed with code {rc}")


# ---------------------------------------------------------------- Sec. 3: keys
def bounding_cube(x, y, z) -> np.ndarray:
    x, y, z = (_c(a, np.float64) for a in (x, y, z))
    box = np.zeros(4, np.float64)
    _check(_load().oracle_bounding_cube(_ptr(x), _ptr(y), _ptr(z), x.size, _ptr(box)), "bounding_cube")
    return box


def grid_coord(x: float, lo: float, side: float, levels: int = L) -> int:
    lib = _load(levels)
    return int(lib.oracle_grid_coord(x, lo, lib.oracle_scale(side)))


def morton_key(ix: int, iy: int, iz: int, levels: int = L) -> int:
    return int(_load(levels).oracle_morton_key(ix, iy, iz))


def morton_decode(key: int, levels: int = L):
    a, b, c = ctypes.c_uint32(), ctypes.c_uint32(), ctypes.c_uint32()
    _load(levels).oracle_morton_decode(key, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c))
    return a.value, b.value, c.value


def hilbert_key(ix: int, iy: int, iz: int, order: int = L) -> int:
    return int(_load().oracle_hilbert_key_order(ix, iy, iz, order))


def hilbert_decode(key: int, order: int = L):
    a, b, c = ctypes.c_uint32(), ctypes.c_uint32(), ctypes.c_uint32()
    _load().oracle_hilbert_decode_order(key, order, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c))
    return a.value, b.value, c.value


def keys(x, y, z, box, curve: int, levels: int = L) -> np.ndarray:
    x, y, z = (_c(a, np.float64) for a in (x, y, z))
    box = _c(box, np.float64)
    out = np.empty(x.size, np.uint64)
    _check(_load(levels).oracle_keys(_ptr(x), _ptr(y), _ptr(z), x.size, _ptr(box), curve, _ptr(out)), "keys")
    return out


# ---------------------------------------------------------------- Sec. 4: sort + leaves
def sort(keys_in):
    k = _c(keys_in, np.uint64)
    s = np.empty_like(k)
    p = np.empty(k.size, np.uint32)
    _check(_load().oracle_sort(_ptr(k), k.size, _ptr(s), _ptr(p)), "sort")
    return s, p


def lower_bound(P, key: int) -> int:
    P = _c(P, np.uint64)
    return int(_load().oracle_lower_bound(_ptr(P), P.size, key))


def histogram(P, K) -> np.ndarray:
    P, K = _c(P, np.uint64), _c(K, np.uint64)
    N = np.empty(K.size - 1, np.uint32)
    _check(_load().oracle_histogram(_ptr(P), P.size, _ptr(K), K.size - 1, _ptr(N)), "histogram")
    return N


def rebalance_decision(K, N, ncrit: int, levels: int = L) -> np.ndarray:
    K, N = _c(K, np.uint64), _c(N, np.uint32)
    O = np.empty(K.size, np.uint32)
    _check(_load(levels).oracle_rebalance_decision(_ptr(K), _ptr(N), K.size - 1, ncrit, _ptr(O)), "g1")
    return O


def exclusive_scan(O) -> np.ndarray:
    O = _c(O, np.uint32)
    out = np.empty(O.size, np.uint64)
    _check(_load().oracle_exclusive_scan(_ptr(O), O.size, _ptr(out)), "g2")
    return out


def rebalance(K, O, Oprime, levels: int = L) -> np.ndarray:
    K, O, Op = _c(K, np.uint64), _c(O, np.uint32), _c(Oprime, np.uint64)
    nl = K.size - 1
    out = np.empty(int(Op[nl]) + 1, np.uint64)
    _check(_load(levels).oracle_rebalance(_ptr(K), _ptr(O), _ptr(Op), nl, _ptr(out)), "g3")
    return out


def leaf_capacity_bound(n: int, ncrit: int, levels: int = L) -> int:
    """Upper bound on the leaves of a balanced tree: every split needs more than Ncrit particles in
    the node, so each level holds at most n / (Ncrit + 1) split nodes, each adding 7 leaves."""
    return 1 + 7 * levels * (n // (ncrit + 1) + 1)


def build_leaves(P, ncrit: int, K_init=None, max_iters: int = 64, cap: int | None = None, levels: int = L):
    """Literal f/g iteration of Sec. 4. Returns (K, N, iterations)."""
    P = _c(P, np.uint64)
    if cap is None:
        cap = leaf_capacity_bound(P.size, ncrit, levels)
    Kout = np.empty(cap + 1, np.uint64)
    Nout = np.empty(cap, np.uint32)
    nl = ctypes.c_int64()
    it = ctypes.c_int()
    if K_init is None:
        kin, nl_init = None, 0
    else:
        kin = _c(K_init, np.uint64)
        nl_init = kin.size - 1
    rc = _load(levels).oracle_build_leaves(_ptr(P), P.size, ncrit, _ptr(kin) if kin is not None else None, nl_init,
                                     _ptr(Kout), cap, ctypes.byref(nl), _ptr(Nout), max_iters, ctypes.byref(it))
    _check(rc, "build_leaves")
    return Kout[: nl.value + 1].copy(), Nout[: nl.value].copy(), it.value


def canonical_leaves(P, ncrit: int, cap: int | None = None, levels: int = L) -> np.ndarray:
    """The balanced octree by its definition (top-down), for comparison with the iteration."""
    P = _c(P, np.uint64)
    if cap is None:
        cap = leaf_capacity_bound(P.size, ncrit, levels)
    Kout = np.empty(cap + 1, np.uint64)
    nl = ctypes.c_int64()
    _check(_load(levels).oracle_canonical_leaves(_ptr(P), P.size, ncrit, _ptr(Kout), cap, ctypes.byref(nl)),
           "canonical_leaves")
    return Kout[: nl.value + 1].copy()


def check_cornerstone(K, levels: int = L) -> bool:
    K = _c(K, np.uint64)
    return _load(levels).oracle_check_cornerstone(_ptr(K), K.size - 1) == 0


# ---------------------------------------------------------------- Sec. 6: distributed tree
def cube_from_bounds(bounds) -> np.ndarray:
    """Cube {lo_x, lo_y, lo_z, side} from per-axis bounds reduced over processes."""
    b = _c(bounds, np.float64)
    box = np.zeros(4, np.float64)
    _check(_load().oracle_cube_from_bounds(_ptr(b), _ptr(box)), "cube_from_bounds")
    return box


def decompose(N, n_ranks: int) -> np.ndarray:
    """The n_ranks + 1 leaf cuts of the SFC domain decomposition of the leaf counts N."""
    N = _c(N, np.uint32)
    cuts = np.empty(n_ranks + 1, np.int64)
    _check(_load().oracle_decompose(_ptr(N), N.size, n_ranks, _ptr(cuts)), "decompose")
    return cuts


# ---------------------------------------------------------------- Sec. 5: linked octree
def link(K, levels: int = L):
    """Returns dict NK, CO, LO, leaf_to_node, parent."""
    K = _c(K, np.uint64)
    nl = K.size - 1
    n = nl + (nl - 1) // 7
    NK = np.empty(n, np.uint64)
    CO = np.empty(n, np.int32)
    LO = np.empty(levels + 2, np.int32)
    l2n = np.empty(nl, np.int32)
    parent = np.empty(max((n - 1) // 8, 1), np.int32)
    _check(_load(levels).oracle_link(_ptr(K), nl, _ptr(NK), _ptr(CO), _ptr(LO), _ptr(l2n), _ptr(parent)), "link")
    return {"NK": NK, "CO": CO, "LO": LO, "leaf_to_node": l2n, "parent": parent[: (n - 1) // 8]}


def node_counts(P, NK, levels: int = L) -> np.ndarray:
    P, NK = _c(P, np.uint64), _c(NK, np.uint64)
    out = np.empty(NK.size, np.uint32)
    _check(_load(levels).oracle_node_counts(_ptr(P), P.size, _ptr(NK), NK.size, _ptr(out)), "node_counts")
    return out


def multipoles(x, y, z, m, P, perm, NK, nodes=None, levels: int = L):
    """FP64 monopole / centre of mass / second moments of the selected nodes (all by default)."""
    x, y, z = (_c(a, np.float64) for a in (x, y, z))
    m = _c(m, np.float32)
    P, perm, NK = _c(P, np.uint64), _c(perm, np.uint32), _c(NK, np.uint64)
    if nodes is None:
        nodes = np.arange(NK.size, dtype=np.int64)
    nodes = _c(nodes, np.int64)
    M = np.empty(nodes.size, np.float64)
    com = np.empty((nodes.size, 3), np.float64)
    quad = np.empty((nodes.size, 6), np.float64)
    _check(_load(levels).oracle_multipoles(_ptr(x), _ptr(y), _ptr(z), _ptr(m), _ptr(P), _ptr(perm), P.size, _ptr(NK),
                                     _ptr(nodes), nodes.size, _ptr(M), _ptr(com), _ptr(quad)), "multipoles")
    return M, com, quad


# ---------------------------------------------------------------- Sec. 7: focused (locally essential) tree
def focus_tiles(f_start: int, f_end: int, levels: int = L):
    """The maximal octree nodes tiling the key range [f_start, f_end): list of (start, level)."""
    cap = 2 * 7 * (levels + 1)
    ts = np.empty(cap, np.uint64)
    tl = np.empty(cap, np.int32)
    nt = _load(levels).oracle_focus_tiles(f_start, f_end, _ptr(ts), _ptr(tl), cap)
    if nt < 0:
        raise OracleError(f"focus_tiles failed with code {nt}")
    return [(int(ts[i]), int(tl[i])) for i in range(nt)]


def mac_passes(start: int, level: int, f_start: int, f_end: int, theta: float, curve: int, levels: int = L) -> bool:
    """Minimum-distance MAC of the node (start, level) against every point of the focus."""
    return bool(_load(levels).oracle_mac_passes(start, level, f_start, f_end, theta, curve))


def focus_decision(K, N, ncrit: int, f_start: int, f_end: int, theta: float, curve: int, levels: int = L):
    K, N = _c(K, np.uint64), _c(N, np.uint32)
    O = np.empty(K.size, np.uint32)
    _check(_load(levels).oracle_focus_decision(_ptr(K), _ptr(N), K.size - 1, ncrit, f_start, f_end, theta, curve,
                                               _ptr(O)), "focus_decision")
    return O


def build_focus_leaves(P, ncrit: int, f_start: int, f_end: int, theta: float, curve: int, K_init=None,
                       max_iters: int = 64, cap: int | None = None, levels: int = L):
    """Literal f / g1^LE / g2 / g3 iteration of Sec. 7 on one process. Returns (K, N, iterations)."""
    P = _c(P, np.uint64)
    if cap is None:
        cap = leaf_capacity_bound(P.size, ncrit, levels)
    Kout = np.empty(cap + 1, np.uint64)
    Nout = np.empty(cap, np.uint32)
    nl = ctypes.c_int64()
    it = ctypes.c_int()
    kin, nl_init = (None, 0) if K_init is None else (_c(K_init, np.uint64), len(K_init) - 1)
    rc = _load(levels).oracle_build_focus_leaves(_ptr(P), P.size, ncrit, f_start, f_end, theta, curve,
                                                 _ptr(kin) if kin is not None else None, nl_init, _ptr(Kout), cap,
                                                 ctypes.byref(nl), _ptr(Nout), max_iters, ctypes.byref(it))
    _check(rc, "build_focus_leaves")
    return Kout[: nl.value + 1].copy(), Nout[: nl.value].copy(), it.value


def canonical_focus_leaves(P, ncrit: int, f_start: int, f_end: int, theta: float, curve: int,
                           cap: int | None = None, levels: int = L):
    """The focused tree by its definition (top-down)."""
    P = _c(P, np.uint64)
    if cap is None:
        cap = leaf_capacity_bound(P.size, ncrit, levels)
    Kout = np.empty(cap + 1, np.uint64)
    nl = ctypes.c_int64()
    _check(_load(levels).oracle_canonical_focus_leaves(_ptr(P), P.size, ncrit, f_start, f_end, theta, curve,
                                                       _ptr(Kout), cap, ctypes.byref(nl)), "canonical_focus_leaves")
    return Kout[: nl.value + 1].copy()


def full_build(x, y, z, curve: int, ncrit: int, box=None, levels: int = L):
    """The whole path in the paper's order; returns a dict of every intermediate result."""
    if box is None:
        box = bounding_cube(x, y, z)
    k = keys(x, y, z, box, curve, levels)
    P, perm = sort(k)
    K, N, iters = build_leaves(P, ncrit, levels=levels)
    tree = link(K, levels)
    counts = node_counts(P, tree["NK"], levels)
    out = {"box": np.asarray(box, np.float64), "keys": k, "P": P, "perm": perm, "K": K, "N": N, "iters": iters,
           "counts": counts}
    out.update(tree)
    return out
