// One f/g step with the leaf counts supplied from outside (Sec. 4, Eqs. histogram and g1-g3).
//
// The single-GPU leaf loop (leaves.cu) keeps f and g inside one persistent launch. A build whose
// particles are spread over several processes (the global tree of Sec. 6, f_glob = f_r o f)
// needs the two halves apart: every rank counts its own particles per leaf (f), the counts are
// summed over the ranks (one allreduce of n_l integers), and every rank applies the same g to the
// same summed counts, so the leaf arrays stay identical on all ranks.
//
// f: one thread per leaf, two binary searches in the sorted keys. g: three launches: the decision
// O_i of every leaf with per-tile sums, one block scanning the tile sums, and a per-tile scan that
// places every kept, merged-into or split leaf (Eqs. rebalancecopy / rebalancesplit).
//
// The locally essential tree of Sec. 7 (focused on the key range F = [f_start, f_end)) uses the
// same g2 and g3 after its own decision g1^LE: inside F (and for nodes overlapping it) the rule
// of g1; outside F a leaf splits only when it also fails the minimum-distance MAC r_min > l / theta
// against F, and 8 sibling leaves merge when their parent holds at most N_crit particles or lies
// outside F and passes the MAC. r_min is the smallest distance between the node's cube and the
// cubes of the maximal octree nodes that tile F (at most 2 * 7 * L of them, decoded once per
// block); distances are in cells of the 2^L grid, r_min^2 an exact integer, (l / theta)^2 two IEEE
// double roundings.
#include "common.cuh"

namespace CST_NS {
namespace {

constexpr int kThreads = 256;
constexpr int kItems = 8;
constexpr int kTile = kThreads * kItems;  // entries of O per tile

struct RebalanceState {
    u32 total;    // n_l of the new array
    u32 changed;  // some O_i != 1
};

__device__ __forceinline__ u32 lower_bound_keys(const Key* __restrict__ P, u32 n, Key key) {
    u32 lo = 0, len = n;
    while (len > 0) {
        const u32 half = len >> 1;
        if (P[lo + half] < key) {
            lo += half + 1;
            len -= half + 1;
        } else {
            len = half;
        }
    }
    return lo;
}

// f (Eq. histogram): N_i = lb(P, K_{i+1}) - lb(P, K_i).
__global__ void __launch_bounds__(kThreads) leaf_counts_kernel(const Key* __restrict__ P, u32 n,
                                                               const Key* __restrict__ K, u32 nl,
                                                               u32* __restrict__ counts) {
    for (u32 i = blockIdx.x * kThreads + threadIdx.x; i < nl; i += gridDim.x * kThreads)
        counts[i] = lower_bound_keys(P, n, K[i + 1]) - lower_bound_keys(P, n, K[i]);
}

// g1 (Eq. g1) for leaf i: split (8) when it holds more than ncrit particles and is not a single
// key; remove (0) when it is sibling j >= 1 of 8 sibling leaves that together hold at most ncrit
// particles (the first sibling stays and becomes their parent); else keep (1).
__device__ __forceinline__ u32 decision(const Key* __restrict__ K, const u32* __restrict__ N, u32 nl, u32 i,
                                        u32 ncrit) {
    const Key ke = K[i];
    const Key delta = K[i + 1] - ke;
    if (N[i] > ncrit && delta > 1) return 8u;
    if (delta < kKeyEnd) {
        const u32 j = static_cast<u32>((ke >> key_ffs(delta)) & 7u);
        if (j >= 1u && j <= i && i - j + 8u <= nl) {
            const u32 first = i - j;
            if (K[first] + static_cast<Key>(8) * delta == K[first + 8]) {
                u32 sum = 0;
#pragma unroll
                for (int s = 0; s < 8; ++s) sum += N[first + s];
                if (sum <= ncrit) return 0u;
            }
        }
    }
    return 1u;
}

__device__ __forceinline__ u32 block_exclusive_scan(u32 v, u32* s_warp, u32* total) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    u32 incl = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const u32 t = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += t;
    }
    if (lane == 31) s_warp[warp] = incl;
    __syncthreads();
    u32 before = 0, all = 0;
#pragma unroll
    for (int w = 0; w < kThreads / 32; ++w) {
        const u32 x = s_warp[w];
        before += w < warp ? x : 0u;
        all += x;
    }
    __syncthreads();
    *total = all;
    return before + incl - v;
}

// O for entries [tile * kTile, ...) of the nl + 1 entries (O_nl = 0), and the tile's sum.
__global__ void __launch_bounds__(kThreads) rebalance_ops_kernel(const Key* __restrict__ K, const u32* __restrict__ N,
                                                                 u32 nl, u32 ncrit, unsigned char* __restrict__ O,
                                                                 u32* __restrict__ tile_sums, RebalanceState* st) {
    __shared__ u32 s_warp[kThreads / 32];
    const u32 base = blockIdx.x * kTile + threadIdx.x * kItems;
    u32 sum = 0;
    bool changed = false;
#pragma unroll
    for (int k = 0; k < kItems; ++k) {
        const u32 i = base + k;
        if (i > nl) break;
        const u32 op = i < nl ? decision(K, N, nl, i, ncrit) : 0u;
        O[i] = static_cast<unsigned char>(op);
        sum += op;
        changed |= i < nl && op != 1u;
    }
    if (__syncthreads_or(changed) && threadIdx.x == 0) atomicOr(&st->changed, 1u);
    u32 total;
    block_exclusive_scan(sum, s_warp, &total);
    if (threadIdx.x == 0) tile_sums[blockIdx.x] = total;
}

// Exclusive scan of the tile sums in one block (in place); the grand total is the new n_l.
__global__ void __launch_bounds__(1024) rebalance_scan_kernel(u32* __restrict__ tile_sums, u32 ntiles,
                                                              RebalanceState* st) {
    __shared__ u32 s_part[1024];
    const u32 per = (ntiles + 1023) / 1024;
    const u32 b0 = threadIdx.x * per, b1 = min(b0 + per, ntiles);
    u32 sum = 0;
    for (u32 q = b0; q < b1; ++q) sum += tile_sums[q];
    s_part[threadIdx.x] = sum;
    __syncthreads();
    for (int o = 1; o < 1024; o <<= 1) {
        const u32 v = threadIdx.x >= static_cast<unsigned>(o) ? s_part[threadIdx.x - o] : 0u;
        __syncthreads();
        s_part[threadIdx.x] += v;
        __syncthreads();
    }
    u32 run = s_part[threadIdx.x] - sum;
    for (u32 q = b0; q < b1; ++q) {
        const u32 v = tile_sums[q];
        tile_sums[q] = run;
        run += v;
    }
    if (threadIdx.x == 1023) st->total = s_part[1023];
}

// g2 + g3: O' by a scan inside the tile plus the tile's offset, then every kept leaf copies its
// key to K'[O'_i] (Eq. rebalancecopy) and every split leaf writes its 8 children
// K_i + c delta_i / 8 to K'[O'_i + c] (Eq. rebalancesplit); K'[n_l'] = 8^L. Writes past the
// capacity are dropped (the host reports the overflow).
__global__ void __launch_bounds__(kThreads) rebalance_scatter_kernel(const Key* __restrict__ K,
                                                                     const unsigned char* __restrict__ O, u32 nl,
                                                                     const u32* __restrict__ tile_offsets,
                                                                     Key* __restrict__ Kout, u32 cap_entries,
                                                                     const RebalanceState* st) {
    __shared__ u32 s_warp[kThreads / 32];
    const u32 base = blockIdx.x * kTile + threadIdx.x * kItems;
    u32 op[kItems];
    u32 sum = 0;
#pragma unroll
    for (int k = 0; k < kItems; ++k) {
        const u32 i = base + k;
        op[k] = i <= nl ? O[i] : 0u;
        sum += op[k];
    }
    u32 total;
    u32 at = tile_offsets[blockIdx.x] + block_exclusive_scan(sum, s_warp, &total);
#pragma unroll
    for (int k = 0; k < kItems; ++k) {
        const u32 i = base + k;
        if (op[k] == 1u) {
            if (at < cap_entries) Kout[at] = K[i];
        } else if (op[k] == 8u) {
            const Key ke = K[i];
            const Key step = (K[i + 1] - ke) >> 3;
#pragma unroll
            for (int c = 0; c < 8; ++c)
                if (at + c < cap_entries) Kout[at + c] = ke + static_cast<Key>(c) * step;
        }
        at += op[k];
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        const u32 nl_new = st->total;
        if (nl_new < cap_entries) Kout[nl_new] = kKeyEnd;
    }
}

// ------------------------------------------------------------------ focused decision (Sec. 7)
constexpr int kMaxFocusTiles = 2 * 7 * (kLevels + 1);

struct FocusParams {
    Key start[kMaxFocusTiles];
    unsigned char level[kMaxFocusTiles];
    int n_tiles;
    Key f_start, f_end;
    double theta;
    int curve;
};

// Grid cell (2^L per axis) of a key: the Morton de-interleave, or the Hilbert state machine run
// backwards from the top level.
__device__ __forceinline__ void key_cell(Key key, int curve, const unsigned short* dec, u32 c[3]) {
    u32 x = 0, y = 0, z = 0, state = 0;
    for (int l = kLevels - 1; l >= 0; --l) {
        u32 o = static_cast<u32>((key >> (3 * l)) & 7u);
        if (curve == CSTONE_HILBERT) {
            const u32 e = dec[state * 8 + o];
            o = e & 7u;
            state = e >> 3;
        }
        x = (x << 1) | (o >> 2);
        y = (y << 1) | ((o >> 1) & 1u);
        z = (z << 1) | (o & 1u);
    }
    c[0] = x;
    c[1] = y;
    c[2] = z;
}

__device__ __forceinline__ bool outside_focus(Key start, Key size, Key f_start, Key f_end) {
    return f_end <= f_start || start + size <= f_start || start >= f_end;
}

// MAC of the cube [c, c + edge)^3 against the focus tiles held in shared memory.
__device__ __forceinline__ bool mac_passes(const u32 c[3], u32 edge, const u32 (*tc)[4], int nt, double theta) {
    if (nt == 0) return true;  // an empty focus accepts every node
    u64 best = ~0ULL;
    for (int t = 0; t < nt && best != 0; ++t) {
        u64 r2 = 0;
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            const u64 a0 = c[d], a1 = a0 + edge, b0 = tc[t][d], b1 = b0 + tc[t][3];
            const u64 gap = b0 > a1 ? b0 - a1 : (a0 > b1 ? a0 - b1 : 0);
            r2 += gap * gap;
        }
        best = r2 < best ? r2 : best;
    }
    const double q = __ddiv_rn(static_cast<double>(edge), theta);
    return __ull2double_rn(best) > __dmul_rn(q, q);
}

__global__ void __launch_bounds__(kThreads) focus_ops_kernel(const Key* __restrict__ K, const u32* __restrict__ N,
                                                             u32 nl, u32 ncrit, const __grid_constant__ FocusParams fp,
                                                             const __grid_constant__ HilbertDecodeTable dt,
                                                             unsigned char* __restrict__ O,
                                                             u32* __restrict__ tile_sums, RebalanceState* st) {
    __shared__ u32 s_warp[kThreads / 32];
    __shared__ u32 s_tile[kMaxFocusTiles][4];  // cube corner and edge of every focus tile
    __shared__ unsigned short s_dec[kHilbertStates * 8];
    for (int i = threadIdx.x; i < kHilbertStates * 8; i += kThreads) s_dec[i] = dt.one[i];
    __syncthreads();
    for (int t = threadIdx.x; t < fp.n_tiles; t += kThreads) {
        u32 c[3];
        key_cell(fp.start[t], fp.curve, s_dec, c);
        const u32 edge = 1u << (kLevels - fp.level[t]);
        for (int d = 0; d < 3; ++d) s_tile[t][d] = c[d] & ~(edge - 1u);
        s_tile[t][3] = edge;
    }
    __syncthreads();
    const u32 base = blockIdx.x * kTile + threadIdx.x * kItems;
    u32 sum = 0;
    bool changed = false;
    for (int k = 0; k < kItems; ++k) {
        const u32 i = base + k;
        if (i > nl) break;
        u32 op = 0;
        if (i < nl) {
            const Key ke = K[i];
            const Key delta = K[i + 1] - ke;
            const int level = kLevels - key_ffs(delta) / 3;
            const u32 edge = 1u << (kLevels - level);
            bool cube_known = false;
            u32 c[3];
            auto cube = [&]() {
                if (!cube_known) {
                    key_cell(ke, fp.curve, s_dec, c);
                    for (int d = 0; d < 3; ++d) c[d] &= ~(edge - 1u);
                    cube_known = true;
                }
            };
            bool split = N[i] > ncrit && delta > 1;
            if (split && outside_focus(ke, delta, fp.f_start, fp.f_end)) {
                cube();
                split = !mac_passes(c, edge, s_tile, fp.n_tiles, fp.theta);
            }
            op = 1u;
            if (split) {
                op = 8u;
            } else if (delta < kKeyEnd) {
                const u32 j = static_cast<u32>((ke >> key_ffs(delta)) & 7u);
                if (j >= 1u && j <= i && i - j + 8u <= nl) {
                    const u32 first = i - j;
                    if (K[first] + static_cast<Key>(8) * delta == K[first + 8]) {
                        u32 s8 = 0;
#pragma unroll
                        for (int q = 0; q < 8; ++q) s8 += N[first + q];
                        bool merge = s8 <= ncrit;
                        if (!merge && outside_focus(K[first], static_cast<Key>(8) * delta, fp.f_start, fp.f_end)) {
                            cube();
                            u32 pc[3];
                            for (int d = 0; d < 3; ++d) pc[d] = c[d] & ~(2u * edge - 1u);
                            merge = mac_passes(pc, 2u * edge, s_tile, fp.n_tiles, fp.theta);
                        }
                        if (merge) op = 0u;
                    }
                }
            }
        }
        O[i] = static_cast<unsigned char>(op);
        sum += op;
        changed |= i < nl && op != 1u;
    }
    if (__syncthreads_or(changed) && threadIdx.x == 0) atomicOr(&st->changed, 1u);
    u32 total;
    block_exclusive_scan(sum, s_warp, &total);
    if (threadIdx.x == 0) tile_sums[blockIdx.x] = total;
}

struct RebalanceLayout {
    RebalanceState* st;
    u32* tile_sums;
    unsigned char* O;
    u32 ntiles;
    size_t bytes;
};

RebalanceLayout rebalance_layout(void* ws, long long nl) {
    RebalanceLayout l;
    Carver c(ws);
    l.ntiles = static_cast<u32>((nl + 1 + kTile - 1) / kTile);
    l.st = c.take<RebalanceState>(1);
    l.tile_sums = c.take<u32>(l.ntiles);
    l.O = c.take<unsigned char>((size_t)nl + 1);
    l.bytes = c.size();
    return l;
}

}  // namespace

size_t rebalance_ws_bytes(long long nl) { return rebalance_layout(nullptr, nl).bytes; }

int launch_leaf_counts(const Key* P, long long n, const Key* K, long long nl, u32* counts, cudaStream_t st) {
    const long long want = (nl + kThreads - 1) / kThreads;
    const int grid = static_cast<int>(want < (long long)sm_count() * 8 ? want : (long long)sm_count() * 8);
    leaf_counts_kernel<<<grid, kThreads, 0, st>>>(P, static_cast<u32>(n), K, static_cast<u32>(nl), counts);
    CST_LAUNCHED("leaf_counts_kernel");
    return CSTONE_OK;
}

// The maximal octree nodes tiling [f_start, f_end), in key order (host).
int focus_tiles(Key f_start, Key f_end, FocusParams& fp) {
    fp.n_tiles = 0;
    Key s = f_start;
    while (s < f_end) {
        int level = 0;
        for (; level <= kLevels; ++level) {
            const Key size = static_cast<Key>(1) << (3 * (kLevels - level));
            if (s % size == 0 && s + size <= f_end) break;
        }
        if (fp.n_tiles >= kMaxFocusTiles) return fail(CSTONE_ERR_INVALID_ARG, "focus range needs too many tiles");
        fp.start[fp.n_tiles] = s;
        fp.level[fp.n_tiles] = static_cast<unsigned char>(level);
        ++fp.n_tiles;
        s += static_cast<Key>(1) << (3 * (kLevels - level));
    }
    return CSTONE_OK;
}

// focus == nullptr: the plain g1; else g1^LE of the focus
int launch_rebalance(const Key* K, const u32* N, long long nl, u32 ncrit, Key* Kout, long long cap, long long* nl_out,
                     int* changed, void* ws, cudaStream_t st, const FocusParams* focus = nullptr) {
    RebalanceLayout l = rebalance_layout(ws, nl);
    CST_CUDA(cudaMemsetAsync(ws, 0, sizeof(WsHeader), st));
    CST_CUDA(cudaMemsetAsync(l.st, 0, sizeof(RebalanceState), st));
    if (focus) {
        focus_ops_kernel<<<l.ntiles, kThreads, 0, st>>>(K, N, static_cast<u32>(nl), ncrit, *focus,
                                                        hilbert_decode_table(), l.O, l.tile_sums, l.st);
        CST_LAUNCHED("focus_ops_kernel");
    } else {
        rebalance_ops_kernel<<<l.ntiles, kThreads, 0, st>>>(K, N, static_cast<u32>(nl), ncrit, l.O, l.tile_sums,
                                                            l.st);
        CST_LAUNCHED("rebalance_ops_kernel");
    }
    rebalance_scan_kernel<<<1, 1024, 0, st>>>(l.tile_sums, l.ntiles, l.st);
    CST_LAUNCHED("rebalance_scan_kernel");
    rebalance_scatter_kernel<<<l.ntiles, kThreads, 0, st>>>(K, l.O, static_cast<u32>(nl), l.tile_sums, Kout,
                                                            static_cast<u32>(cap + 1), l.st);
    CST_LAUNCHED("rebalance_scatter_kernel");
    RebalanceState h;
    CST_CUDA(cudaMemcpyAsync(&h, l.st, sizeof(h), cudaMemcpyDeviceToHost, st));
    CST_CUDA(cudaStreamSynchronize(st));
    *nl_out = h.total;
    *changed = h.changed ? 1 : 0;
    if (h.total > cap)
        return fail(CSTONE_ERR_CAPACITY, CST_STR(CSTONE_FN(rebalance)) ": %u leaves needed, capacity %lld", h.total,
                    cap);
    return CSTONE_OK;
}

}  // namespace CST_NS

extern "C" {

int CSTONE_FN(leaf_counts)(const CST_KEY_C* sorted_keys, int64_t n, const CST_KEY_C* leaves, int64_t n_leaves,
                           uint32_t* counts, void* stream) {
    if (n < 0 || n >= CSTONE_MAX_PARTICLES || n_leaves < 1 || n_leaves > CSTONE_MAX_LEAVES || !leaves || !counts ||
        (n > 0 && !sorted_keys))
        return cst::fail(CSTONE_ERR_INVALID_ARG, CST_STR(CSTONE_FN(leaf_counts)) ": bad argument");
    return CST_NS::launch_leaf_counts(reinterpret_cast<const CST_NS::Key*>(sorted_keys), n,
                                      reinterpret_cast<const CST_NS::Key*>(leaves), n_leaves, counts,
                                      cst::as_stream(stream));
}

int CSTONE_FN(rebalance_workspace_size)(int64_t n_leaves, size_t* bytes) {
    if (!bytes || n_leaves < 1 || n_leaves > CSTONE_MAX_LEAVES)
        return cst::fail(CSTONE_ERR_INVALID_ARG, CST_STR(CSTONE_FN(rebalance_workspace_size)) ": bad argument");
    *bytes = CST_NS::rebalance_ws_bytes(n_leaves);
    return CSTONE_OK;
}

int CSTONE_FN(rebalance)(const CST_KEY_C* leaves, const uint32_t* counts, int64_t n_leaves, uint32_t ncrit,
                         CST_KEY_C* leaves_out, int64_t leaf_cap, int64_t* n_leaves_out, int32_t* changed, void* ws,
                         size_t ws_bytes, void* stream) {
    if (n_leaves < 1 || n_leaves > CSTONE_MAX_LEAVES || leaf_cap < 1 || leaf_cap > CSTONE_MAX_LEAVES || !leaves ||
        !counts || !leaves_out || !n_leaves_out || !changed || leaves == leaves_out)
        return cst::fail(CSTONE_ERR_INVALID_ARG, CST_STR(CSTONE_FN(rebalance)) ": bad argument");
    if (int rc = cst::check_ws(ws, ws_bytes, CST_NS::rebalance_ws_bytes(n_leaves), CST_STR(CSTONE_FN(rebalance))))
        return rc;
    long long nl = 0;
    int ch = 0;
    const int rc = CST_NS::launch_rebalance(reinterpret_cast<const CST_NS::Key*>(leaves), counts, n_leaves, ncrit,
                                            reinterpret_cast<CST_NS::Key*>(leaves_out), leaf_cap, &nl, &ch, ws,
                                            cst::as_stream(stream));
    *n_leaves_out = nl;
    *changed = ch;
    return rc;
}

int CSTONE_FN(rebalance_focus)(const CST_KEY_C* leaves, const uint32_t* counts, int64_t n_leaves, uint32_t ncrit,
                               CST_KEY_C f_start, CST_KEY_C f_end, double theta, int curve, CST_KEY_C* leaves_out,
                               int64_t leaf_cap, int64_t* n_leaves_out, int32_t* changed, void* ws, size_t ws_bytes,
                               void* stream) {
    if (n_leaves < 1 || n_leaves > CSTONE_MAX_LEAVES || leaf_cap < 1 || leaf_cap > CSTONE_MAX_LEAVES || !leaves ||
        !counts || !leaves_out || !n_leaves_out || !changed || leaves == leaves_out || !(theta > 0.0) ||
        (curve != CSTONE_MORTON && curve != CSTONE_HILBERT) || f_end > CST_NS::kKeyEnd || f_start > f_end)
        return cst::fail(CSTONE_ERR_INVALID_ARG, CST_STR(CSTONE_FN(rebalance_focus)) ": bad argument");
    if (int rc = cst::check_ws(ws, ws_bytes, CST_NS::rebalance_ws_bytes(n_leaves),
                               CST_STR(CSTONE_FN(rebalance_focus))))
        return rc;
    CST_NS::FocusParams fp;
    if (int rc = CST_NS::focus_tiles(f_start, f_end, fp)) return rc;
    fp.f_start = f_start;
    fp.f_end = f_end;
    fp.theta = theta;
    fp.curve = curve;
    long long nl = 0;
    int ch = 0;
    const int rc = CST_NS::launch_rebalance(reinterpret_cast<const CST_NS::Key*>(leaves), counts, n_leaves, ncrit,
                                            reinterpret_cast<CST_NS::Key*>(leaves_out), leaf_cap, &nl, &ch, ws,
                                            cst::as_stream(stream), &fp);
    *n_leaves_out = nl;
    *changed = ch;
    return rc;
}

}  // extern "C"
