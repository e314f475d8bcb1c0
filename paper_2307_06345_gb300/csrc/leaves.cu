// Cornerstone leaf array: the f / g iteration of Sec. 4 (Eqs. histogram, g1, g2, g3) in one
// persistent cooperative kernel.
//
// Alongside K the kernel keeps pos_i = lower_bound(P, K_i) for every key of the array. Then the
// histogram of Eq. (histogram) is N_i = pos_{i+1} - pos_i, and the combined count of 8 sibling
// leaves is pos_{i-j+8} - pos_{i-j}. pos survives rebalancing: a copied key keeps its position,
// the end key keeps n, and the 8 child keys of a split leaf are searched for only inside the
// parent's particle range [pos_i, pos_{i+1}) - the same lower bounds the paper's two binary
// searches per bin give, found in a small window instead of the whole of P.
//
// One pass (g1 + g2 + g3) is a single sweep over tiles of the array: each thread decides O_i for
// a run of leaves, the block scans the decisions, the tile's offset comes from decoupled
// look-back over the preceding tiles (claimed in order through an atomic counter), and every
// leaf is copied, split into 8 or dropped at its scanned position. A bounded grid barrier closes
// the pass; all blocks then read the "changed" flag and either start the next pass or, once a
// pass changed nothing, write the converged array out. The whole loop is one launch and needs no
// host round trip.
#include "common.cuh"

namespace cst {
namespace {

constexpr int kThreads = 256;
constexpr int kItems = 2;
constexpr int kTile = kThreads * kItems;  // leaf indices per tile
constexpr int kMaxIters = 256;
constexpr int kSplitChunks = 16;                 // keys per lane loaded at once when counting a split
constexpr u32 kLinearSplit = 32 * kSplitChunks;  // split ranges up to this size are counted, not searched
constexpr u64 kLookAggregate = 1ULL << 62;
constexpr u64 kLookPrefix = 2ULL << 62;
constexpr u64 kLookValue = (1ULL << 62) - 1ULL;

struct LoopState {
    u32 nl[kMaxIters + 1];       // leaves entering pass t (nl[0] = initial)
    u32 changed[kMaxIters];      // pass t changed the array
    u32 tile_counter[kMaxIters]; // tile dispenser of pass t
    GridBarrier bar;
    u32 iters;                   // passes executed (set at convergence)
    u32 converged;
    u32 required;                // leaves needed when the capacity was exceeded
    u32 final_buf;               // buffer holding the converged array
};

struct LeafBufs {
    u64* K[2];
    u32* pos[2];
};

__device__ __forceinline__ u64 ld_volatile64(const u64* p) { return *reinterpret_cast<const volatile u64*>(p); }
__device__ __forceinline__ void st_volatile64(u64* p, u64 v) { *reinterpret_cast<volatile u64*>(p) = v; }

// First position in P[lo, hi) whose key is >= key.
__device__ __forceinline__ u32 lower_bound_in(const u64* __restrict__ P, u32 lo, u32 hi, u64 key) {
    while (lo < hi) {
        u32 mid = lo + ((hi - lo) >> 1);
        if (__ldg(P + mid) < key)
            lo = mid + 1;
        else
            hi = mid;
    }
    return lo;
}

// Eq. (g1) for leaf i < nl. Split when N_i > ncrit (a single key at depth L stays); merge away
// the octants 1..7 of a parent whose 8 children are consecutive leaves holding <= ncrit in total
// (octant 0 keeps its key, which is the parent's); keep otherwise.
__device__ __forceinline__ u32 decide(const u64* __restrict__ K, const u32* __restrict__ pos, u32 i, u32 nl, u32 ncrit) {
    u64 ki = K[i], delta = K[i + 1] - ki;
    u32 cnt = pos[i + 1] - pos[i];
    if (cnt > ncrit && delta > 1ULL) return 8u;
    if (delta < kKeyEnd) {
        u32 j = static_cast<u32>((ki >> (__ffsll(static_cast<long long>(delta)) - 1)) & 7ULL);
        if (j >= 1u && j <= i && i - j + 8u <= nl) {
            u32 first = i - j;
            if (K[first] + 8ULL * delta == K[first + 8] && pos[first + 8] - pos[first] <= ncrit) return 0u;
        }
    }
    return 1u;
}

__global__ void __launch_bounds__(kThreads) leaves_loop_kernel(const u64* __restrict__ P, u32 n, u32 ncrit,
                                                               LeafBufs b, u32 cap, int max_iters, int warm,
                                                               u64* look, u32 max_tiles, LoopState* ls,
                                                               WsHeader* hdr, u64* out_keys, u32* out_counts,
                                                               u32* out_offsets) {
    __shared__ u32 s_warp[kThreads / 32];
    __shared__ unsigned char s_op[kTile];
    __shared__ unsigned short s_split[kTile];
    __shared__ u32 s_nsplit;
    __shared__ u32 s_off[kTile];
    __shared__ u32 s_tile;
    __shared__ u64 s_prefix;
    __shared__ int s_any;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const u32 gtid = blockIdx.x * kThreads + tid, gthreads = gridDim.x * kThreads;

    // ---- initial array in buffer 0 with the particle position of every key
    if (!warm) {
        if (gtid == 0) {
            b.K[0][0] = 0ULL;
            b.K[0][1] = kKeyEnd;
            b.pos[0][0] = 0u;
            b.pos[0][1] = n;
        }
    } else {
        u32 nl0 = ls->nl[0];
        for (u32 i = gtid; i <= nl0; i += gthreads) b.pos[0][i] = lower_bound_in(P, 0u, n, b.K[0][i]);
    }
    grid_barrier(&ls->bar, hdr);

    int t = 0;
    for (; t < max_iters; ++t) {
        if (ld_volatile(&hdr->err)) break;
        const u64* K = b.K[t & 1];
        const u32* pos = b.pos[t & 1];
        u64* Kn = b.K[(t + 1) & 1];
        u32* posn = b.pos[(t + 1) & 1];
        const u32 nl = ld_volatile(&ls->nl[t]);
        const u32 ntiles = (nl + 1 + kTile - 1) / kTile;  // indices 0..nl, nl is the end sentinel
        u64* look_t = look + (size_t)t * max_tiles;
        int any_change = 0;

        for (;;) {
            if (tid == 0) {
                s_tile = atomicAdd(&ls->tile_counter[t], 1u);
                s_nsplit = 0;
            }
            __syncthreads();
            const u32 tile = s_tile;
            __syncthreads();
            if (tile >= ntiles) break;

            // g1, striped: item j of the tile is leaf tile * kTile + j, handled by thread j % kThreads
            const u32 t0 = tile * kTile;
#pragma unroll
            for (int k = 0; k < kItems; ++k) {
                const u32 j = k * kThreads + tid;
                const u32 i = t0 + j;
                u32 o = (i < nl) ? decide(K, pos, i, nl, ncrit) : 0u;
                if (i < nl && o != 1u) any_change = 1;
                s_op[j] = static_cast<unsigned char>(o);
            }
            __syncthreads();
            // g2: exclusive scan of O over the tile (blocked runs of kItems per thread), then the
            // tile's offset by decoupled look-back
            u32 run[kItems];
            u32 sum = 0;
#pragma unroll
            for (int k = 0; k < kItems; ++k) {
                run[k] = sum;
                sum += s_op[tid * kItems + k];
            }
            u32 incl = sum;
            for (int s = 1; s < 32; s <<= 1) {
                u32 v = __shfl_up_sync(0xffffffffu, incl, s);
                if (lane >= s) incl += v;
            }
            if (lane == 31) s_warp[warp] = incl;
            __syncthreads();
            u32 wpre = 0, total = 0;
            for (int w = 0; w < kThreads / 32; ++w) {
                u32 v = s_warp[w];
                if (w < warp) wpre += v;
                total += v;
            }
            const u32 excl_in_tile = wpre + incl - sum;
#pragma unroll
            for (int k = 0; k < kItems; ++k) s_off[tid * kItems + k] = excl_in_tile + run[k];

            // decoupled look-back by warp 0: 32 predecessor descriptors per step
            if (warp == 0) {
                u64* mine = look_t + tile;
                u64 prefix = 0;
                if (tile == 0) {
                    if (lane == 0) st_volatile64(mine, kLookPrefix | total);
                } else {
                    if (lane == 0) st_volatile64(mine, kLookAggregate | total);
                    long long top = (long long)tile - 1;
                    long long polls = 0;
                    for (;;) {
                        const long long jj = top - lane;
                        const u64 v = jj >= 0 ? ld_volatile64(look_t + jj) : kLookPrefix;
                        const u64 flag = v & ~kLookValue;
                        const u32 pmask = __ballot_sync(0xffffffffu, flag == kLookPrefix);
                        const u32 xmask = __ballot_sync(0xffffffffu, flag == 0ULL);
                        const int first_p = pmask ? __ffs(pmask) - 1 : 32;
                        const u32 before = first_p == 32 ? 0xffffffffu : ((1u << first_p) - 1u);
                        if (xmask & before) {  // a nearer predecessor has not published yet
                            __nanosleep(32);
                            if (++polls > kSpinLimit || ld_volatile(&hdr->err) != 0u) {
                                if (lane == 0) raise_error(hdr, CSTONE_ERR_TIMEOUT, 0x2000u);
                                break;
                            }
                            continue;
                        }
                        u64 part = lane <= first_p ? (v & kLookValue) : 0ULL;
                        for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
                        prefix += part;
                        if (first_p < 32) break;
                        top -= 32;
                    }
                    if (lane == 0) st_volatile64(mine, kLookPrefix | (prefix + total));
                }
                if (lane == 0) s_prefix = prefix;
            }
            __syncthreads();

            // g3, striped: copy, split or drop each leaf at its scanned position. A split writes its
            // 8 child keys and queues itself; the child particle offsets are found below.
            const u64 prefix = s_prefix;
#pragma unroll 1
            for (int k = 0; k < kItems; ++k) {
                const u32 j = k * kThreads + tid;
                const u32 i = t0 + j;
                if (i > nl) break;
                const u64 o_pos = prefix + s_off[j];
                if (i == nl) {  // end sentinel: K'_{n_l'} = 8^L, and n_l' itself
                    if (o_pos <= cap) {
                        Kn[o_pos] = kKeyEnd;
                        posn[o_pos] = n;
                    }
                    ls->nl[t + 1] = static_cast<u32>(o_pos > 0xffffffffULL ? 0xffffffffULL : o_pos);
                    if (o_pos > cap) {
                        ls->required = static_cast<u32>(o_pos > 0xffffffffULL ? 0xffffffffULL : o_pos);
                        raise_error(hdr, CSTONE_ERR_CAPACITY, 0u);
                    }
                    break;
                }
                const u32 o = s_op[j];
                if (o == 1u) {
                    if (o_pos < cap) {
                        Kn[o_pos] = K[i];
                        posn[o_pos] = pos[i];
                    }
                } else if (o == 8u) {
                    const u64 ki = K[i];
                    const u64 step = (K[i + 1] - ki) >> 3;
                    if (o_pos + 8 <= cap) {
#pragma unroll
                        for (int c = 0; c < 8; ++c) Kn[o_pos + c] = ki + static_cast<u64>(c) * step;
                        posn[o_pos] = pos[i];
                    }
                    s_split[atomicAdd(&s_nsplit, 1u)] = static_cast<unsigned short>(j);
                }
            }
            __syncthreads();
            // particle offsets of the 7 inner children of every split leaf, one warp per split: the
            // child of a particle is one octal digit of its key, so a short range is counted with
            // ballots over coalesced loads; a long range (early passes) is binary-searched, one
            // child boundary per lane
            const u32 nsplit = s_nsplit;
            for (u32 q = warp; q < nsplit; q += kThreads / 32) {
                const u32 j = s_split[q];
                const u32 i = t0 + j;
                const u64 o_pos = prefix + s_off[j];
                const u64 ki = K[i];
                const u64 delta = K[i + 1] - ki;
                const u32 lo = pos[i], cnt_all = pos[i + 1] - lo;
                const int child_shift = __ffsll(static_cast<long long>(delta)) - 1 - 3;
                u32 below = 0;  // lane c in 1..7: particles whose child digit is < c
                if (cnt_all <= kLinearSplit) {
                    u32 dg[kSplitChunks];
#pragma unroll
                    for (int b = 0; b < kSplitChunks; ++b) {  // every load issued before any use
                        const u32 jj = b * 32 + lane;
                        dg[b] = jj < cnt_all ? static_cast<u32>((__ldg(P + lo + jj) >> child_shift) & 7ULL) : 8u;
                    }
#pragma unroll
                    for (int b = 0; b < kSplitChunks; ++b) {
                        if (b * 32 >= static_cast<int>(cnt_all)) break;
#pragma unroll
                        for (u32 c = 1; c < 8; ++c) {
                            const u32 bal = __ballot_sync(0xffffffffu, dg[b] < c);
                            if (lane == c) below += __popc(bal);
                        }
                    }
                } else if (lane >= 1 && lane < 8) {
                    const u64 key = ki + static_cast<u64>(lane) * (delta >> 3);
                    for (u32 st = 1u << (31 - __clz(cnt_all)); st > 0; st >>= 1) {
                        const u32 probe = below + st;
                        if (probe <= cnt_all && __ldg(P + lo + probe - 1) < key) below = probe;
                    }
                }
                if (lane >= 1 && lane < 8 && o_pos + 8 <= cap) posn[o_pos + lane] = lo + below;
            }
            __syncthreads();  // s_op / s_off are rewritten by the next tile
        }
        if (tid == 0) s_any = 0;
        __syncthreads();
        if (any_change) s_any = 1;
        __syncthreads();
        if (tid == 0 && s_any) atomicOr(&ls->changed[t], 1u);
        grid_barrier(&ls->bar, hdr);
        if (ld_volatile(&hdr->err)) break;
        if (ld_volatile(&ls->changed[t]) == 0u) {
            ++t;  // this pass confirmed convergence; its output equals its input
            break;
        }
    }

    if (ld_volatile(&hdr->err)) return;
    const bool converged = (t <= max_iters) && ld_volatile(&ls->changed[t - 1]) == 0u;
    if (gtid == 0) {
        ls->iters = static_cast<u32>(t);
        ls->converged = converged ? 1u : 0u;
        ls->final_buf = static_cast<u32>(t & 1);
    }
    if (!converged) return;
    const u32 nl = ld_volatile(&ls->nl[t]);
    const u64* K = b.K[t & 1];
    const u32* pos = b.pos[t & 1];
    for (u32 i = gtid; i <= nl; i += gthreads) {
        out_keys[i] = K[i];
        if (i < nl) out_counts[i] = pos[i + 1] - pos[i];
        if (out_offsets) out_offsets[i] = pos[i];
    }
}

struct LeavesLayout {
    LoopState* ls;
    LeafBufs bufs;
    u64* look;
    u32 max_tiles;
    size_t bytes;
};

LeavesLayout leaves_layout(void* ws, long long cap, int max_iters) {
    LeavesLayout l;
    Carver c(ws);
    l.ls = c.take<LoopState>(1);
    for (int k = 0; k < 2; ++k) {
        l.bufs.K[k] = c.take<u64>((size_t)cap + 1);
        l.bufs.pos[k] = c.take<u32>((size_t)cap + 1);
    }
    l.max_tiles = static_cast<u32>((cap + 1 + kTile - 1) / kTile);
    l.look = c.take<u64>((size_t)l.max_tiles * (size_t)max_iters);
    l.bytes = c.size();
    return l;
}

int leaves_grid() { return cooperative_grid(reinterpret_cast<const void*>(leaves_loop_kernel), kThreads, 0, 8); }

}  // namespace

size_t leaves_ws_bytes(long long cap, int max_iters) { return leaves_layout(nullptr, cap, max_iters).bytes; }

int launch_build_leaves(const u64* P, long long n, u32 ncrit, u64* leaves, long long cap, long long* n_leaves,
                        u32* counts, u32* offsets, int max_iters, int* iters, void* ws, cudaStream_t st) {
    LeavesLayout l = leaves_layout(ws, cap, max_iters);
    WsHeader* hdr = reinterpret_cast<WsHeader*>(ws);
    const long long nl0 = *n_leaves;
    CST_CUDA(cudaMemsetAsync(hdr, 0, sizeof(WsHeader), st));
    CST_CUDA(cudaMemsetAsync(l.ls, 0, sizeof(LoopState), st));
    CST_CUDA(cudaMemsetAsync(l.look, 0, (size_t)l.max_tiles * max_iters * sizeof(u64), st));
    int warm = nl0 > 0 ? 1 : 0;
    u32 nl_start = warm ? static_cast<u32>(nl0) : 1u;
    CST_CUDA(cudaMemcpyAsync(&l.ls->nl[0], &nl_start, sizeof(u32), cudaMemcpyHostToDevice, st));
    if (warm)
        CST_CUDA(cudaMemcpyAsync(l.bufs.K[0], leaves, (size_t)(nl0 + 1) * sizeof(u64), cudaMemcpyDeviceToDevice, st));

    const u64* P_ = P;
    u32 n_ = static_cast<u32>(n), ncrit_ = ncrit, cap_ = static_cast<u32>(cap), max_tiles = l.max_tiles;
    int max_iters_ = max_iters;
    LeafBufs bufs = l.bufs;
    u64* look = l.look;
    LoopState* ls = l.ls;
    u64* out_keys = leaves;
    u32* out_counts = counts;
    u32* out_offsets = offsets;
    void* args[] = {&P_, &n_, &ncrit_, &bufs, &cap_, &max_iters_, &warm, &look, &max_tiles, &ls, &hdr,
                    &out_keys, &out_counts, &out_offsets};
    CST_CUDA(cudaLaunchCooperativeKernel(reinterpret_cast<void*>(leaves_loop_kernel), dim3(leaves_grid()),
                                         dim3(kThreads), args, 0, st));

    WsHeader h;
    LoopState s;
    CST_CUDA(cudaMemcpyAsync(&h, hdr, sizeof(h), cudaMemcpyDeviceToHost, st));
    CST_CUDA(cudaMemcpyAsync(&s, l.ls, sizeof(s), cudaMemcpyDeviceToHost, st));
    CST_CUDA(cudaStreamSynchronize(st));
    if (iters) *iters = static_cast<int>(s.iters);
    if (h.err == CSTONE_ERR_CAPACITY) {
        *n_leaves = s.required;
        return fail(CSTONE_ERR_CAPACITY, "cstone_build_leaves: %u leaves needed, capacity %lld", s.required, cap);
    }
    if (h.err) return fail(static_cast<int>(h.err), "cstone_build_leaves: device error %u (info 0x%x)", h.err,
                           h.err_info);
    if (!s.converged)
        return fail(CSTONE_ERR_NOT_CONVERGED, "cstone_build_leaves: not converged after %d passes", max_iters);
    *n_leaves = s.nl[s.iters];
    return CSTONE_OK;
}

}  // namespace cst

extern "C" {

int cstone_leaves_workspace_size(int64_t n, int64_t leaf_cap, int32_t max_iters, size_t* bytes) {
    if (!bytes || n < 0 || n >= CSTONE_MAX_PARTICLES || leaf_cap < 1 || leaf_cap > CSTONE_MAX_LEAVES ||
        max_iters < 1 || max_iters > 256)
        return cst::fail(CSTONE_ERR_INVALID_ARG, "cstone_leaves_workspace_size: bad argument");
    *bytes = cst::leaves_ws_bytes(leaf_cap, max_iters);
    return CSTONE_OK;
}

int cstone_build_leaves(const uint64_t* sorted_keys, int64_t n, uint32_t ncrit, uint64_t* leaves, int64_t leaf_cap,
                        int64_t* n_leaves, uint32_t* counts, uint32_t* offsets, int32_t max_iters, int32_t* iters,
                        void* ws, size_t ws_bytes, void* stream) {
    if (n < 0 || n >= CSTONE_MAX_PARTICLES || leaf_cap < 1 || leaf_cap > CSTONE_MAX_LEAVES || !leaves || !counts ||
        !n_leaves || max_iters < 1 || max_iters > 256 || (n > 0 && !sorted_keys))
        return cst::fail(CSTONE_ERR_INVALID_ARG, "cstone_build_leaves: bad argument");
    if (*n_leaves < 0 || *n_leaves > leaf_cap)
        return cst::fail(CSTONE_ERR_INVALID_ARG, "cstone_build_leaves: initial n_leaves %lld outside [0, %lld]",
                         (long long)*n_leaves, (long long)leaf_cap);
    if (int rc = cst::check_ws(ws, ws_bytes, cst::leaves_ws_bytes(leaf_cap, max_iters), "cstone_build_leaves"))
        return rc;
    long long nl = *n_leaves;
    int it = 0;
    int rc = cst::launch_build_leaves(reinterpret_cast<const cst::u64*>(sorted_keys), n, ncrit,
                                      reinterpret_cast<cst::u64*>(leaves), leaf_cap, &nl, counts, offsets, max_iters,
                                      &it, ws, cst::as_stream(stream));
    *n_leaves = nl;
    if (iters) *iters = it;
    return rc;
}

}  // extern "C"
