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
// The array is handled as a list of elements: the leaves followed by the end key 8^L, which is
// kept (O = 1) like any unchanged leaf. The same kernel then builds many independent arrays at
// once (batched sets): they are stored back to back, each ending with its own 8^L, and every
// element carries its set id so that a merge never reaches across two sets.
//
// One pass (g1 + g2 + g3) takes two sweeps over tiles of the elements (block b of the G co-resident
// blocks takes tiles b, b + G, b + 2G, ...), so that no tile ever waits on another: the first sweep
// decides O for every element of the tile (kept, one byte per element) and records the tile's op
// total and split count; after a grid barrier the second sweep gives each tile its offsets as the
// totals of all earlier tiles (each block adds them up itself), scans the tile, and copies, splits
// or drops every element at its scanned position. A split takes its slot in the pass's split
// queue with what the split phase needs (its particle range, its first child's position, the
// child digit's shift). A pass in which g1 changes nothing ends after the first sweep: its input
// is the converged array. The whole loop is one launch and needs no host round trip.
#include "common.cuh"

namespace CST_NS {
namespace {

constexpr int kThreads = 256;
// Elements per thread and tile (a tuning knob, set by the build from the autotuner's choice).
#ifndef CSTONE_LEAVES_ITEMS
#define CSTONE_LEAVES_ITEMS 8
#endif
constexpr int kItems = CSTONE_LEAVES_ITEMS;
constexpr int kTile = kThreads * kItems;  // elements per tile
static_assert(kItems <= 8, "the staged tile (keys, positions, sets, ops, offsets) must fit 48 KB of shared memory");
constexpr int kMaxIters = 256;
constexpr int kSplitChunks = 16;                 // keys per lane loaded at once when counting a split
constexpr u32 kLinearSplit = 32 * kSplitChunks;  // split ranges up to this size are counted, not searched
// A tile's op total (low 32 bits) and split count (high 32 bits) in one word: a pass has at most 2^28
// elements, so sums of op totals stay below 2^31 and never carry into the split count.

struct LoopState {
    unsigned long long stamp[kMaxIters + 1];  // %globaltimer at the start of pass t (ns), for profiling
    u32 ne[kMaxIters + 1];        // elements entering pass t (ne[0] = initial)
    u32 changed[kMaxIters];       // pass t changed an array
    u32 nsplit[kMaxIters];        // splits queued in pass t (written by the pass's last tile)
    GridBarrier bar;
    u32 iters;                    // passes executed (set at convergence)
    u32 converged;
    u32 required;                 // elements needed when the capacity was exceeded
    u32 final_buf;                // buffer holding the converged arrays
    unsigned long long phase_stamp[kMaxIters][2];  // %globaltimer after pass t's first and second sweep
};

struct LeafBufs {
    uint4* split_q;   // [ecap] queued splits: first particle, particle count, first child's position,
                      // shift of the child digit
    unsigned char* ops;  // [ecap] O of every element of the current pass
    u64* tile_sum;       // [tiles] op total and split count of every tile of the current pass
    Key* K[2];
    u32* pos[2];   // lower bound of the element's key among its set's sorted keys (global index)
    u32* set[2];   // set of the element (batched builds only)
};

struct SetView {  // batched builds
    const long long* particle_offsets;  // [S+1] first particle of each set
    long long* element_offsets;         // [S+1] in (warm start) / out: first element of each set
    int n_sets;
};


// Asynchronous 16-byte copy from global (through L2 only) to shared memory: src_bytes (0..16) are
// copied and the rest of the 16 bytes is zero-filled.
__device__ __forceinline__ void cp_async16(void* smem, const void* gmem, int src_bytes) {
    const unsigned s = static_cast<unsigned>(__cvta_generic_to_shared(smem));
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(s), "l"(gmem), "r"(src_bytes) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

// Stages elements [e_first, e_first + count) of a device array into shared memory (element e_first
// + i at dst[i]) with 16-byte copies; elements outside [0, ne) read as zero. e_first and the array
// start must be 16-byte aligned in bytes.
template <class T>
__device__ __forceinline__ void stage_async(T* dst, const T* src, long long e_first, int count, u32 ne, int tid) {
    constexpr int kPer = 16 / static_cast<int>(sizeof(T));
    const int chunks = (count + kPer - 1) / kPer;
    for (int c = tid; c < chunks; c += kThreads) {
        const long long e0 = e_first + (long long)c * kPer;
        long long valid = (long long)ne - e0;
        valid = valid < 0 ? 0 : (valid > kPer ? kPer : valid);
        const bool inside = e0 >= 0 && valid > 0;
        cp_async16(dst + c * kPer, inside ? static_cast<const void*>(src + e0) : static_cast<const void*>(src),
                   inside ? static_cast<int>(valid * sizeof(T)) : 0);
    }
}

// First position in P[lo, hi) whose key is >= key.
__device__ __forceinline__ u32 lower_bound_in(const Key* __restrict__ P, u32 lo, u32 hi, Key key) {
    while (lo < hi) {
        u32 mid = lo + ((hi - lo) >> 1);
        if (__ldg(P + mid) < key)
            lo = mid + 1;
        else
            hi = mid;
    }
    return lo;
}

// Eq. (g1) for element e of ne. The end key 8^L of a set is kept. A leaf splits when N > ncrit
// (a single key at depth L stays); the octants 1..7 of a parent whose 8 children are consecutive
// leaves of one set holding <= ncrit in total are merged away (octant 0 keeps its key, which is
// the parent's); anything else is kept. K, pos and set are the tile's staged window in shared
// memory: element e sits at index e - h0.
template <bool BATCH>
__device__ __forceinline__ u32 decide(const Key* K, const u32* pos, const u32* set, u32 e, u32 ne, u32 ncrit,
                                      long long h0) {
    const long long i = (long long)e - h0;
    const Key ke = K[i];
    if (ke == kKeyEnd) return 1u;
    const Key delta = K[i + 1] - ke;
    const u32 cnt = pos[i + 1] - pos[i];
    if (cnt > ncrit && delta > 1ULL) return 8u;
    if (delta < kKeyEnd) {
        const u32 j = static_cast<u32>((ke >> key_ffs(delta)) & 7u);
        if (j >= 1u && j <= e && e - j + 8u < ne) {
            const long long f = i - j;
            if (!BATCH || (set[f] == set[i] && set[f + 8] == set[i]))
                if (K[f] + static_cast<Key>(8) * delta == K[f + 8] && pos[f + 8] - pos[f] <= ncrit) return 0u;
        }
    }
    return 1u;
}

constexpr u32 kDeviceCount = 0xffffffffu;  // ne_start: take the element count from the device

// Outputs of a failed asynchronous build: every set gets its root array {0, 8^L}, so that the
// phases queued after it stay within their buffers. The failure itself is in the workspace.
template <bool BATCH>
__device__ void write_root_arrays(const Key* P, u32 n, SetView sv, u32 gtid, u32 gthreads, Key* out_keys,
                                  u32* out_counts, u32* out_offsets) {
    const u32 ns = BATCH ? static_cast<u32>(sv.n_sets) : 1u;
    for (u32 q = gtid; q < ns; q += gthreads) {
        const u32 lo = BATCH ? static_cast<u32>(sv.particle_offsets[q]) : 0u;
        const u32 hi = BATCH ? static_cast<u32>(sv.particle_offsets[q + 1]) : n;
        out_keys[2 * q] = 0;
        out_keys[2 * q + 1] = kKeyEnd;
        out_counts[2 * q] = hi - lo;
        if (BATCH) {
            out_counts[2 * q + 1] = 0u;
            sv.element_offsets[q] = 2 * q;
            if (q == 0) sv.element_offsets[ns] = 2 * ns;
        }
        if (out_offsets) {
            out_offsets[2 * q] = lo;
            out_offsets[2 * q + 1] = hi;
        }
    }
}

#ifndef CSTONE_LEAVES_MIN_BLOCKS
#define CSTONE_LEAVES_MIN_BLOCKS 5
#endif
template <bool BATCH>
__global__ void __launch_bounds__(kThreads, CSTONE_LEAVES_MIN_BLOCKS) leaves_loop_kernel(const Key* __restrict__ P, u32 n, u32 ncrit,
                                                               LeafBufs b, u32 ecap, int max_iters, int warm,
                                                               u32 ne_start, int fallback, LoopState* ls, WsHeader* hdr, SetView sv,
                                                               Key* out_keys, u32* out_counts, u32* out_offsets) {
    __shared__ u32 s_warp[kThreads / 32];
    __shared__ __align__(16) unsigned char s_op[kTile];
    __shared__ u32 s_wsplit[kThreads / 32];
    __shared__ u64 s_part[kThreads / 32];
    __shared__ u32 s_nsplit;
    __shared__ u32 s_off[kTile];
    __shared__ int s_any;
    // the tile's elements with a halo of kHalo on each side (the merge test reads up to 7 back
    // and 8 ahead, the split and count tests one ahead), staged once per tile
    constexpr int kHalo = 8;
    __shared__ __align__(16) Key s_K[kTile + 2 * kHalo];
    __shared__ __align__(16) u32 s_pos[kTile + 2 * kHalo];
    __shared__ __align__(16) u32 s_set[BATCH ? kTile + 2 * kHalo : 4];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const u32 gtid = blockIdx.x * kThreads + tid, gthreads = gridDim.x * kThreads;

    // ---- initial arrays in buffer 0, with the particle position of every key. A warm start reads
    // the previous arrays from the output buffers; their element count is ne_start, or the last
    // element offset on the device when ne_start is kDeviceCount.
    const int ns = BATCH ? sv.n_sets : 1;
    u32 ne_init = 2u * static_cast<u32>(ns);
    if (warm) ne_init = ne_start != kDeviceCount ? ne_start : static_cast<u32>(sv.element_offsets[sv.n_sets]);
    if (ne_init < 2u * static_cast<u32>(ns) || ne_init > ecap) {  // the same decision in every block
        if (gtid == 0) raise_error(hdr, CSTONE_ERR_INVALID_ARG, 0x60000u);
        ne_init = 0;
    }
    if (gtid == 0) ls->ne[0] = ne_init;
    if (!warm) {  // every set starts from its root {0, 8^L}
        for (u32 q = gtid; q < static_cast<u32>(ns); q += gthreads) {
            b.K[0][2 * q] = 0;
            b.K[0][2 * q + 1] = kKeyEnd;
            b.pos[0][2 * q] = BATCH ? static_cast<u32>(sv.particle_offsets[q]) : 0u;
            b.pos[0][2 * q + 1] = BATCH ? static_cast<u32>(sv.particle_offsets[q + 1]) : n;
            if (BATCH) b.set[0][2 * q] = b.set[0][2 * q + 1] = q;
        }
    } else {
        const u32 ne0 = ne_init;
        for (u32 e = gtid; e < ne0; e += gthreads) {
            u32 lo = 0, hi = n;
            if (BATCH) {
                int a = 0, c = sv.n_sets;  // last set whose first element is <= e
                while (c - a > 1) {
                    const int mid = (a + c) >> 1;
                    if (sv.element_offsets[mid] <= e)
                        a = mid;
                    else
                        c = mid;
                }
                b.set[0][e] = static_cast<u32>(a);
                lo = static_cast<u32>(sv.particle_offsets[a]);
                hi = static_cast<u32>(sv.particle_offsets[a + 1]);
            }
            const Key k = out_keys[e];
            b.K[0][e] = k;
            b.pos[0][e] = k == kKeyEnd ? hi : lower_bound_in(P, lo, hi, k);
        }
    }
    grid_barrier(&ls->bar, hdr);

    int t = 0;
    bool converged = false;
    for (; t < max_iters; ++t) {
        if (gtid == 0) {
            unsigned long long now;
            asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(now));
            ls->stamp[t] = now;
        }
        if (ld_volatile(&hdr->err)) break;
        const Key* K = b.K[t & 1];
        const u32* pos = b.pos[t & 1];
        const u32* set = b.set[t & 1];
        Key* Kn = b.K[(t + 1) & 1];
        u32* posn = b.pos[(t + 1) & 1];
        u32* setn = b.set[(t + 1) & 1];
        const u32 ne = ld_volatile(&ls->ne[t]);
        const u32 ntiles = (ne + kTile - 1) / kTile;

        // ---- g1 for every tile of this block: the decisions are kept (one byte per element), and
        // each tile's op total and split count go to tile_sum
        int any_change = 0;
        for (u32 tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
            // stage the tile's window (written by other blocks in the previous pass: read through
            // L2, never through a read-only cache)
            const u32 t0 = tile * kTile;
            const long long h0 = (long long)t0 - kHalo;
            stage_async(s_K, K, h0, kTile + 2 * kHalo, ne, tid);
            stage_async(s_pos, pos, h0, kTile + 2 * kHalo, ne, tid);
            if (BATCH) stage_async(s_set, set, h0, kTile + 2 * kHalo, ne, tid);
            cp_async_wait_all();
            __syncthreads();
            // striped: item j of the tile is element tile * kTile + j, handled by thread j % kThreads
            u32 sum = 0, nspl = 0;
#pragma unroll
            for (int k = 0; k < kItems; ++k) {
                const u32 j = k * kThreads + tid;
                const u32 e = t0 + j;
                if (e < ne) {
                    const u32 o = decide<BATCH>(s_K, s_pos, s_set, e, ne, ncrit, h0);
                    b.ops[e] = static_cast<unsigned char>(o);
                    any_change |= o != 1u;
                    sum += o;
                    nspl += o == 8u ? 1u : 0u;
                }
            }
            for (int o = 16; o > 0; o >>= 1) {
                sum += __shfl_xor_sync(0xffffffffu, sum, o);
                nspl += __shfl_xor_sync(0xffffffffu, nspl, o);
            }
            if (lane == 0) {
                s_warp[warp] = sum;
                s_wsplit[warp] = nspl;
            }
            __syncthreads();
            if (tid == 0) {
                u32 tot = 0, spl = 0;
                for (int w = 0; w < kThreads / 32; ++w) {
                    tot += s_warp[w];
                    spl += s_wsplit[w];
                }
                b.tile_sum[tile] = (static_cast<u64>(spl) << 32) | tot;
            }
            __syncthreads();  // the staging arrays are rewritten by the next tile
        }
        if (tid == 0) s_any = 0;
        __syncthreads();
        if (any_change) s_any = 1;
        __syncthreads();
        if (tid == 0 && s_any) atomicOr(&ls->changed[t], 1u);
        grid_barrier(&ls->bar, hdr);
        if (gtid == 0) {
            unsigned long long now;
            asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(now));
            ls->phase_stamp[t][0] = now;
        }
        if (ld_volatile(&hdr->err)) break;
        if (ld_volatile(&ls->changed[t]) == 0u) {  // this pass confirms convergence: K is final
            converged = true;
            ++t;
            break;
        }

        // ---- g2 + g3 for every tile of this block: the tile's offsets are the totals of all earlier
        // tiles (each block adds the totals up itself: its tiles are blockIdx.x + k gridDim.x), then
        // every element is copied, split into 8 or dropped at its scanned position. A split also
        // takes its slot in the split queue, carrying what the split phase needs.
        u64 prefix = 0;  // tile_sum over [0, done)
        u32 done = 0;
        for (u32 tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
            u64 part = 0;
            for (u32 q = done + tid; q < tile; q += kThreads) part += __ldcg(b.tile_sum + q);
            for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
            if (lane == 0) s_part[warp] = part;
            const u32 t0 = tile * kTile;
            // the tile's elements, one more key and position (a split's gap and range end), its ops
            stage_async(s_K, K, t0, kTile + 1, ne, tid);
            stage_async(s_pos, pos, t0, kTile + 1, ne, tid);
            if (BATCH) stage_async(s_set, set, t0, kTile + 1, ne, tid);
            stage_async(s_op, b.ops, t0, kTile, ne, tid);
            if (tid == 0) s_nsplit = 0;
            cp_async_wait_all();
            __syncthreads();
            for (int w = 0; w < kThreads / 32; ++w) prefix += s_part[w];
            done = tile + 1;
            // exclusive scan of O over the tile (blocked runs of kItems per thread)
            u32 run[kItems];
            u32 sum = 0;
#pragma unroll
            for (int k = 0; k < kItems; ++k) {
                run[k] = sum;
                sum += s_op[tid * kItems + k];
            }
            u32 incl = sum;
            for (int sft = 1; sft < 32; sft <<= 1) {
                u32 v = __shfl_up_sync(0xffffffffu, incl, sft);
                if (lane >= sft) incl += v;
            }
            if (lane == 31) s_warp[warp] = incl;
            __syncthreads();
            u32 wpre = 0;
            for (int w = 0; w < warp; ++w) wpre += s_warp[w];
            const u32 excl_in_tile = wpre + incl - sum;
#pragma unroll
            for (int k = 0; k < kItems; ++k) s_off[tid * kItems + k] = excl_in_tile + run[k];
            __syncthreads();
            const u64 own = __ldcg(b.tile_sum + tile);
            const u64 base_pos = prefix & 0xffffffffULL;
            const u32 qbase = static_cast<u32>(prefix >> 32);
            if (tile == ntiles - 1 && tid == 0) ls->nsplit[t] = static_cast<u32>((prefix + own) >> 32);
#pragma unroll 1
            for (int k = 0; k < kItems; ++k) {
                const u32 j = k * kThreads + tid;
                const u32 e = t0 + j;
                if (e >= ne) break;
                const u64 o_pos = base_pos + s_off[j];
                const u32 o = s_op[j];
                if (o == 1u) {
                    if (o_pos < ecap) {
                        Kn[o_pos] = s_K[j];
                        posn[o_pos] = s_pos[j];
                        if (BATCH) setn[o_pos] = s_set[j];
                    }
                    if (e == ne - 1) {  // the last element is an end key: the new element count
                        const u64 ne_next = o_pos + 1;
                        ls->ne[t + 1] = static_cast<u32>(ne_next > 0xffffffffULL ? 0xffffffffULL : ne_next);
                        if (ne_next > ecap) {
                            ls->required = static_cast<u32>(ne_next > 0xffffffffULL ? 0xffffffffULL : ne_next);
                            raise_error(hdr, CSTONE_ERR_CAPACITY, 0u);
                        }
                    }
                } else if (o == 8u) {
                    const Key ke = s_K[j];
                    const Key delta = s_K[j + 1] - ke;
                    const Key step = delta >> 3;
                    if (o_pos + 8 <= ecap) {
#pragma unroll
                        for (int c = 0; c < 8; ++c) {
                            Kn[o_pos + c] = ke + static_cast<Key>(c) * step;
                            if (BATCH) setn[o_pos + c] = s_set[j];
                        }
                        posn[o_pos] = s_pos[j];
                    }
                    const u32 q = qbase + atomicAdd(&s_nsplit, 1u);
                    if (q < ecap)  // always, unless a barrier timed out (then the error is recorded)
                        b.split_q[q] = make_uint4(s_pos[j], s_pos[j + 1] - s_pos[j], static_cast<u32>(o_pos),
                                              static_cast<u32>(key_ffs(delta) - 3));
                }
            }
            prefix += own;
            __syncthreads();  // the staging arrays and s_nsplit are rewritten by the next tile
        }
        // particle offsets of the 7 inner children of every split leaf, one warp of the whole grid per
        // split (early passes have few leaves but long particle ranges): the child of a particle is
        // one octal digit of its key, so a short range is counted with ballots over coalesced
        // loads; a long range is narrowed by 32 probes at once and then binary-searched, one child
        // boundary per lane. A warp loads its next queue entry before it works on the current one.
        grid_barrier(&ls->bar, hdr);
        if (gtid == 0) {
            unsigned long long now;
            asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(now));
            ls->phase_stamp[t][1] = now;
        }
        {
            const u32 nsplit = ld_volatile(&ls->nsplit[t]);
            const u32 gwarp = gtid >> 5, nwarps = gthreads >> 5;
            uint4 cur = gwarp < nsplit ? __ldcg(b.split_q + gwarp) : make_uint4(0, 0, 0, 0);
            for (u32 q = gwarp; q < nsplit; q += nwarps) {
                const u32 qn = q + nwarps;
                const uint4 nxt = qn < nsplit ? __ldcg(b.split_q + qn) : make_uint4(0, 0, 0, 0);
                const u32 lo = cur.x, cnt_all = cur.y, o_pos = cur.z;
                const int child_shift = static_cast<int>(cur.w);
                cur = nxt;
                if (lo > n || cnt_all > n - lo || child_shift < 0 || child_shift > kKeyBits - 3) {
                    // self-check: a particle range outside P is never read
                    if (lane == 0) raise_error(hdr, CSTONE_ERR_INVALID_ARG, 0x70000u);
                    continue;
                }
                if (static_cast<u64>(o_pos) + 8 > ecap) continue;  // over capacity: reported, nothing to write
                u32 below = 0;  // lane c in 1..7: particles whose child digit is < c
                if (cnt_all <= kLinearSplit) {
                    // the child digits of the range do not decrease: the offset of child c is the first
                    // position whose digit is >= c. Lane c first writes the range end (no particle of
                    // digit >= c), then the lane at each digit change writes the children it opens.
                    u32 dg[kSplitChunks];
#pragma unroll
                    for (int c = 0; c < kSplitChunks; ++c) {  // every load issued before any use
                        const u32 jj = c * 32 + lane;
                        dg[c] = jj < cnt_all ? static_cast<u32>((__ldg(P + lo + jj) >> child_shift) & 7ULL) : 8u;
                    }
                    if (lane >= 1 && lane < 8) posn[o_pos + lane] = lo + cnt_all;
                    __syncwarp();
                    u32 prev_last = 0;  // digit of the element before this chunk (0 before the first)
#pragma unroll
                    for (int c = 0; c < kSplitChunks; ++c) {
                        if (c * 32 >= static_cast<int>(cnt_all)) break;
                        const u32 up = __shfl_up_sync(0xffffffffu, dg[c], 1);
                        const u32 before_me = lane == 0 ? prev_last : up;
                        const u32 mine = dg[c] < 7u ? dg[c] : 7u;
                        for (u32 d = before_me + 1; d <= mine; ++d) posn[o_pos + d] = lo + c * 32 + lane;
                        prev_last = __shfl_sync(0xffffffffu, dg[c], 31);
                    }
                    continue;  // the boundaries are written
                }
                // one round of 32 probes spread over the range: the child digits of the probes do not
                // decrease, so for child c the first n_c probes (digit < c) bound its offset to
                // (probe n_c - 1, probe n_c], about cnt_all / 33 particles; lane c then
                // binary-searches that interval for the first key >= the child's key. The parent's
                // key is the first child's, written by g3 above.
                const Key ke = __ldcg(Kn + o_pos);
                const u32 qk = static_cast<u32>((static_cast<u64>(lane + 1) * cnt_all) / 33u);
                const u32 gk = static_cast<u32>((__ldg(P + lo + qk) >> child_shift) & 7ULL);
                u32 a = 0, hi = cnt_all;  // lane c in 1..7: its offset lies in [a, hi]
#pragma unroll
                for (u32 d = 1; d < 8; ++d) {
                    const u32 nc = __popc(__ballot_sync(0xffffffffu, gk < d));
                    const u32 q_lo = __shfl_sync(0xffffffffu, qk, nc > 0 ? nc - 1 : 0);
                    const u32 q_hi = __shfl_sync(0xffffffffu, qk, nc < 32 ? nc : 31);
                    if (lane == d) {
                        a = nc > 0 ? q_lo + 1 : 0;
                        hi = nc < 32 ? q_hi : cnt_all;
                    }
                }
                if (lane >= 1 && lane < 8) {
                    const Key key = ke + (static_cast<Key>(lane) << child_shift);
                    below = a;  // the particle before offset a (a probe of digit < c) is below key
                    if (hi > a)
                        for (u32 st = 1u << (31 - __clz(hi - a)); st > 0; st >>= 1) {
                            const u32 probe = below + st;
                            if (probe <= hi && __ldg(P + lo + probe - 1) < key) below = probe;
                        }
                    posn[o_pos + lane] = lo + below;
                }
            }
        }
        grid_barrier(&ls->bar, hdr);
    }

    if (ld_volatile(&hdr->err)) {
        if (fallback) write_root_arrays<BATCH>(P, n, sv, gtid, gthreads, out_keys, out_counts, out_offsets);
        return;
    }
    // converged: the last pass (t - 1) changed nothing, so its input arrays are the result
    const int last = t - 1;
    if (gtid == 0) {
        unsigned long long now;
        asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(now));
        ls->stamp[t] = now;
        ls->iters = static_cast<u32>(t);
        ls->converged = converged ? 1u : 0u;
        ls->final_buf = static_cast<u32>(last & 1);
    }
    if (!converged) {
        if (fallback) write_root_arrays<BATCH>(P, n, sv, gtid, gthreads, out_keys, out_counts, out_offsets);
        return;
    }
    const u32 ne = ld_volatile(&ls->ne[last]);
    const Key* K = b.K[last & 1];
    const u32* pos = b.pos[last & 1];
    const u32* set = b.set[last & 1];
    for (u32 e = gtid; e < ne; e += gthreads) {
        const Key k = K[e];
        out_keys[e] = k;
        if (BATCH) {
            out_counts[e] = k == kKeyEnd ? 0u : pos[e + 1] - pos[e];
            if (e == 0 || K[e - 1] == kKeyEnd) sv.element_offsets[set[e]] = e;
            if (e == 0) sv.element_offsets[sv.n_sets] = ne;
        } else if (e + 1 < ne) {
            out_counts[e] = pos[e + 1] - pos[e];
        }
        if (out_offsets) out_offsets[e] = pos[e];
    }
}

struct LeavesLayout {
    LoopState* ls;
    LeafBufs bufs;
    size_t bytes;
};

LeavesLayout leaves_layout(void* ws, long long ecap, int max_iters, bool batch) {
    (void)max_iters;
    LeavesLayout l;
    Carver c(ws);
    l.ls = c.take<LoopState>(1);
    l.bufs.split_q = c.take<uint4>((size_t)ecap);
    l.bufs.ops = c.take<unsigned char>((size_t)ecap);
    l.bufs.tile_sum = c.take<u64>((size_t)((ecap + kTile - 1) / kTile));
    for (int k = 0; k < 2; ++k) {
        l.bufs.K[k] = c.take<Key>((size_t)ecap);
        l.bufs.pos[k] = c.take<u32>((size_t)ecap);
        l.bufs.set[k] = batch ? c.take<u32>((size_t)ecap) : nullptr;
    }
    l.bytes = c.size();
    return l;
}

template <bool BATCH>
int leaves_grid() {
    return cooperative_grid(reinterpret_cast<const void*>(leaves_loop_kernel<BATCH>), kThreads, 0, 8);
}

// Outcome of the loop recorded in a workspace: status, passes, element count (or, on a capacity
// overflow, the count needed). Synchronises the stream.
int read_leaves_result(void* ws, cudaStream_t st, long long ecap, int max_iters, long long* ne_out, int* iters,
                       const char* who) {
    LoopState* lsp = reinterpret_cast<LoopState*>(static_cast<char*>(ws) + sizeof(WsHeader));
    WsHeader h;
    LoopState s;
    CST_CUDA(cudaMemcpyAsync(&h, ws, sizeof(h), cudaMemcpyDeviceToHost, st));
    CST_CUDA(cudaMemcpyAsync(&s, lsp, sizeof(s), cudaMemcpyDeviceToHost, st));
    CST_CUDA(cudaStreamSynchronize(st));
    if (iters) *iters = static_cast<int>(s.iters);
    if (h.err == CSTONE_ERR_CAPACITY) {
        *ne_out = s.required;
        return fail(CSTONE_ERR_CAPACITY, "%s: %u array elements needed, capacity %lld", who, s.required, ecap);
    }
    if (h.err) return fail(static_cast<int>(h.err), "%s: device error %u (info 0x%x)", who, h.err, h.err_info);
    if (!s.converged) return fail(CSTONE_ERR_NOT_CONVERGED, "%s: not converged after %d passes", who, max_iters);
    *ne_out = s.ne[s.iters - 1];  // the last pass changed nothing: its input is the result
    return CSTONE_OK;
}

// Runs the loop. ne0: element count of the warm-start arrays held in `leaves` (0 = cold start from
// the roots, -1 = warm start with the count read on the device). With sync, *ne_out is the element
// count of the converged arrays on success; without, nothing is read back (the outcome stays in
// the workspace for read_leaves_result) and a failure leaves every set's root array as output.
template <bool BATCH>
int run_leaves(const Key* P, long long n, u32 ncrit, Key* leaves, long long ecap, long long ne0, long long* ne_out,
               u32* counts, u32* offsets, int max_iters, int* iters, SetView sv, void* ws, cudaStream_t st,
               const char* who, bool sync = true) {
    LeavesLayout l = leaves_layout(ws, ecap, max_iters, BATCH);
    WsHeader* hdr = reinterpret_cast<WsHeader*>(ws);
    CST_CUDA(cudaMemsetAsync(hdr, 0, sizeof(WsHeader), st));
    CST_CUDA(cudaMemsetAsync(l.ls, 0, sizeof(LoopState), st));
    int warm = ne0 != 0 ? 1 : 0;
    u32 ne_start = ne0 < 0 ? kDeviceCount : static_cast<u32>(ne0);
    int fallback = sync ? 0 : 1;

    const Key* P_ = P;
    u32 n_ = static_cast<u32>(n), ncrit_ = ncrit, ecap_ = static_cast<u32>(ecap);
    int max_iters_ = max_iters;
    LeafBufs bufs = l.bufs;
    LoopState* ls = l.ls;
    Key* out_keys = leaves;
    u32* out_counts = counts;
    u32* out_offsets = offsets;
    void* args[] = {&P_,       &n_,   &ncrit_,    &bufs, &ecap_, &max_iters_, &warm,     &ne_start,   &fallback,
                    &ls,       &hdr,  &sv,    &out_keys,   &out_counts, &out_offsets};
    CST_COOP(cudaLaunchCooperativeKernel(reinterpret_cast<void*>(leaves_loop_kernel<BATCH>), dim3(leaves_grid<BATCH>()),
                                         dim3(kThreads), args, 0, st));
    if (!sync) return CSTONE_OK;
    return read_leaves_result(ws, st, ecap, max_iters, ne_out, iters, who);
}

}  // namespace

size_t leaves_ws_bytes(long long cap, int max_iters) { return leaves_layout(nullptr, cap + 1, max_iters, false).bytes; }
size_t leaves_batched_ws_bytes(long long ecap, int max_iters) {
    return leaves_layout(nullptr, ecap, max_iters, true).bytes;
}

int launch_build_leaves(const Key* P, long long n, u32 ncrit, Key* leaves, long long cap, long long* n_leaves,
                        u32* counts, u32* offsets, int max_iters, int* iters, void* ws, cudaStream_t st) {
    const long long ne0 = *n_leaves > 0 ? *n_leaves + 1 : 0;
    long long ne = 0;
    const int rc = run_leaves<false>(P, n, ncrit, leaves, cap + 1, ne0, &ne, counts, offsets, max_iters, iters,
                                     SetView{nullptr, nullptr, 1}, ws, st, CST_STR(CSTONE_FN(build_leaves)));
    if (rc == CSTONE_ERR_CAPACITY) {
        *n_leaves = ne - 1;
        return rc;
    }
    if (rc == CSTONE_OK) *n_leaves = ne - 1;
    return rc;
}

int launch_build_leaves_batched_async(const Key* P, long long n, const long long* particle_offsets, int n_sets,
                                      u32 ncrit, Key* leaves, long long ecap, long long* element_offsets, int warm,
                                      u32* counts, u32* offsets, int max_iters, void* ws, cudaStream_t st) {
    return run_leaves<true>(P, n, ncrit, leaves, ecap, warm ? -1 : 0, nullptr, counts, offsets, max_iters, nullptr,
                            SetView{particle_offsets, element_offsets, n_sets}, ws, st,
                            "cstone_build_leaves_batched_async", false);
}

int launch_build_leaves_batched(const Key* P, long long n, const long long* particle_offsets, int n_sets, u32 ncrit,
                                Key* leaves, long long ecap, long long* element_offsets, long long* n_elements,
                                u32* counts, u32* offsets, int max_iters, int* iters, void* ws, cudaStream_t st) {
    long long ne = 0;
    const int rc = run_leaves<true>(P, n, ncrit, leaves, ecap, *n_elements, &ne, counts, offsets, max_iters, iters,
                                    SetView{particle_offsets, element_offsets, n_sets}, ws, st,
                                    "cstone_build_leaves_batched");
    if (rc == CSTONE_OK || rc == CSTONE_ERR_CAPACITY) *n_elements = ne;
    return rc;
}

}  // namespace CST_NS

extern "C" {

int CSTONE_FN(leaves_workspace_size)(int64_t n, int64_t leaf_cap, int32_t max_iters, size_t* bytes) {
    if (!bytes || n < 0 || n >= CSTONE_MAX_PARTICLES || leaf_cap < 1 || leaf_cap > CSTONE_MAX_LEAVES ||
        max_iters < 1 || max_iters > 256)
        return cst::fail(CSTONE_ERR_INVALID_ARG, CST_STR(CSTONE_FN(leaves_workspace_size)) ": bad argument");
    *bytes = CST_NS::leaves_ws_bytes(leaf_cap, max_iters);
    return CSTONE_OK;
}

int CSTONE_FN(build_leaves)(const CST_KEY_C* sorted_keys, int64_t n, uint32_t ncrit, CST_KEY_C* leaves,
                            int64_t leaf_cap, int64_t* n_leaves, uint32_t* counts, uint32_t* offsets,
                            int32_t max_iters, int32_t* iters, void* ws, size_t ws_bytes, void* stream) {
    if (n < 0 || n >= CSTONE_MAX_PARTICLES || leaf_cap < 1 || leaf_cap > CSTONE_MAX_LEAVES || !leaves || !counts ||
        !n_leaves || max_iters < 1 || max_iters > 256 || (n > 0 && !sorted_keys))
        return cst::fail(CSTONE_ERR_INVALID_ARG, CST_STR(CSTONE_FN(build_leaves)) ": bad argument");
    if (*n_leaves < 0 || *n_leaves > leaf_cap)
        return cst::fail(CSTONE_ERR_INVALID_ARG, CST_STR(CSTONE_FN(build_leaves)) ": initial n_leaves %lld outside "
                         "[0, %lld]", (long long)*n_leaves, (long long)leaf_cap);
    if (int rc = cst::check_ws(ws, ws_bytes, CST_NS::leaves_ws_bytes(leaf_cap, max_iters),
                               CST_STR(CSTONE_FN(build_leaves))))
        return rc;
    long long nl = *n_leaves;
    int it = 0;
    int rc = CST_NS::launch_build_leaves(reinterpret_cast<const CST_NS::Key*>(sorted_keys), n, ncrit,
                                         reinterpret_cast<CST_NS::Key*>(leaves), leaf_cap, &nl, counts, offsets,
                                         max_iters, &it, ws, cst::as_stream(stream));
    *n_leaves = nl;
    if (iters) *iters = it;
    return rc;
}

#ifndef CSTONE_KEY32  // batched builds exist for 63-bit keys only
int cstone_leaves_batched_workspace_size(int64_t elem_cap, int32_t max_iters, size_t* bytes) {
    if (!bytes || elem_cap < 2 || elem_cap > CSTONE_MAX_LEAVES || max_iters < 1 || max_iters > 256)
        return cst::fail(CSTONE_ERR_INVALID_ARG, "cstone_leaves_batched_workspace_size: bad argument");
    *bytes = cst::leaves_batched_ws_bytes(elem_cap, max_iters);
    return CSTONE_OK;
}

int cstone_build_leaves_batched(const uint64_t* sorted_keys, int64_t n, const int64_t* set_offsets, int32_t n_sets,
                                uint32_t ncrit, uint64_t* elements, int64_t elem_cap, int64_t* element_offsets,
                                int64_t* n_elements, uint32_t* counts, uint32_t* offsets, int32_t max_iters,
                                int32_t* iters, void* ws, size_t ws_bytes, void* stream) {
    if (n < 0 || n >= CSTONE_MAX_PARTICLES || n_sets < 1 || n_sets > (1 << 20) || !set_offsets || !elements ||
        !element_offsets || !n_elements || !counts || elem_cap < 2 * (int64_t)n_sets || elem_cap > CSTONE_MAX_LEAVES ||
        max_iters < 1 || max_iters > 256 || (n > 0 && !sorted_keys))
        return cst::fail(CSTONE_ERR_INVALID_ARG, "cstone_build_leaves_batched: bad argument");
    if (*n_elements < 0 || *n_elements > elem_cap || (*n_elements > 0 && *n_elements < 2 * (int64_t)n_sets))
        return cst::fail(CSTONE_ERR_INVALID_ARG, "cstone_build_leaves_batched: initial n_elements %lld invalid",
                         (long long)*n_elements);
    if (int rc = cst::check_ws(ws, ws_bytes, cst::leaves_batched_ws_bytes(elem_cap, max_iters),
                               "cstone_build_leaves_batched"))
        return rc;
    long long ne = *n_elements;
    int it = 0;
    int rc = cst::launch_build_leaves_batched(reinterpret_cast<const cst::u64*>(sorted_keys), n,
                                              reinterpret_cast<const long long*>(set_offsets), n_sets, ncrit,
                                              reinterpret_cast<cst::u64*>(elements), elem_cap,
                                              reinterpret_cast<long long*>(element_offsets), &ne, counts, offsets,
                                              max_iters, &it, ws, cst::as_stream(stream));
    *n_elements = ne;
    if (iters) *iters = it;
    return rc;
}

int cstone_build_leaves_batched_async(const uint64_t* sorted_keys, int64_t n, const int64_t* set_offsets,
                                      int32_t n_sets, uint32_t ncrit, uint64_t* elements, int64_t elem_cap,
                                      int64_t* element_offsets, int32_t warm, uint32_t* counts, uint32_t* offsets,
                                      int32_t max_iters, void* ws, size_t ws_bytes, void* stream) {
    if (n < 0 || n >= CSTONE_MAX_PARTICLES || n_sets < 1 || n_sets > (1 << 20) || !set_offsets || !elements ||
        !element_offsets || !counts || elem_cap < 2 * (int64_t)n_sets || elem_cap > CSTONE_MAX_LEAVES ||
        max_iters < 1 || max_iters > 256 || (n > 0 && !sorted_keys))
        return cst::fail(CSTONE_ERR_INVALID_ARG, "cstone_build_leaves_batched_async: bad argument");
    if (int rc = cst::check_ws(ws, ws_bytes, cst::leaves_batched_ws_bytes(elem_cap, max_iters),
                               "cstone_build_leaves_batched_async"))
        return rc;
    return cst::launch_build_leaves_batched_async(reinterpret_cast<const cst::u64*>(sorted_keys), n,
                                                  reinterpret_cast<const long long*>(set_offsets), n_sets, ncrit,
                                                  reinterpret_cast<cst::u64*>(elements), elem_cap,
                                                  reinterpret_cast<long long*>(element_offsets), warm ? 1 : 0, counts,
                                                  offsets, max_iters, ws, cst::as_stream(stream));
}

int cstone_leaves_result(void* ws, int64_t elem_cap, int32_t max_iters, void* stream, int64_t* n_elements,
                         int32_t* iters) {
    if (!ws || !n_elements || elem_cap < 1 || max_iters < 1 || max_iters > 256)
        return cst::fail(CSTONE_ERR_INVALID_ARG, "cstone_leaves_result: bad argument");
    long long ne = 0;
    int it = 0;
    const int rc = cst::read_leaves_result(ws, cst::as_stream(stream), elem_cap, max_iters, &ne, &it,
                                           "cstone_build_leaves_batched_async");
    *n_elements = ne;
    if (iters) *iters = it;
    return rc;
}

#endif

}  // extern "C"
