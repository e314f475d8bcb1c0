// Stable LSD radix sort_by_key of the particle keys with the identity permutation as values
// (Sec. 4 and the caption of Table 1: the particle keys are sorted with a permutation that
// records where each particle went). 63-bit keys in 64-bit words take 8 passes of 8-bit digits,
// 30-bit keys in 32-bit words take 4.
//
// Each digit pass reads a tile of keys (and values), ranks them within the tile (the lanes of a warp
// holding the same digit are found with one ballot per digit bit, which measured much cheaper than
// a warp match instruction), stages the tile in shared memory in digit order (the keys, then the
// values, through one buffer) and writes each digit's run contiguously at the tile's output
// position for that digit; the first pass generates the identity values instead of reading them.
// Ahead of every pass, a count of every tile's digits
// and a two-level scan of the counts give each tile its output positions, so no tile waits on
// another (a decoupled look-back between tiles, measured first, spent a third of the sort's time
// waiting on predecessors); the same counts give the digits' totals, whose scan over the digits
// places each digit's run, so no separate histogram pass reads the keys. A segmented sort aligns its tiles to the segments, scans the counts of all tiles
// at once, and takes a tile's position within its segment as the difference to the segment's
// first tile, added to the segment's digit offsets.
#include <mutex>

#include "common.cuh"

namespace CST_NS {
namespace {

constexpr int kRadixBits = 8;
constexpr int kRadix = 1 << kRadixBits;
constexpr int kPasses = (kKeyBits + kRadixBits - 1) / kRadixBits;  // 8 (63-bit keys) or 4 (30-bit keys)
// Tile shape (compile-time tuning knobs, set by the build from the autotuner's choice): threads per
// block, keys per thread and blocks per SM.
#ifndef CSTONE_SORT_THREADS
#define CSTONE_SORT_THREADS 256
#endif
#ifndef CSTONE_SORT_ITEMS
#define CSTONE_SORT_ITEMS 12
#endif
#ifndef CSTONE_SORT_MIN_BLOCKS
#define CSTONE_SORT_MIN_BLOCKS 4
#endif
constexpr int kThreads = CSTONE_SORT_THREADS;
constexpr int kWarps = kThreads / 32;
constexpr int kItems = CSTONE_SORT_ITEMS;
static_assert(kThreads >= 256 && kThreads % 32 == 0, "one thread per digit is needed");
static_assert(kItems % 2 == 0, "ranks are packed two per register");
constexpr int kTile = kThreads * kItems;  // keys per tile

// Segmented sorts (many independent key sets stored back to back) use tiles aligned to the
// segments: every tile holds keys of one segment only, and digits are offset per segment.
struct SegTiles {
    const u32* n_tiles;      // device scalar: tiles in use
    const u32* tile_seg;     // segment of each tile
    const u32* tile_base;    // first key (global index) of each tile
    const u32* tile_count;   // keys in each tile (<= kTile)
    const u32* seg_first;    // first tile of each segment
    const u32* seg_offsets;  // [segment][pass][digit] output position of the digit's first key
};

struct SegBuild {  // writable view of the same tables
    u32* n_tiles;
    u32* tile_seg;
    u32* tile_base;
    u32* tile_count;
    u32* seg_first;
    u32* seg_hist;
    u32* seg_offsets;
};

// Tiles per segment and their exclusive scan (one block).
__global__ void __launch_bounds__(1024) seg_setup_kernel(const long long* __restrict__ seg_offsets_in, int n_segs,
                                                         SegBuild b) {
    __shared__ u32 s_part[1024];
    const int per = (n_segs + 1023) / 1024;
    const int begin = threadIdx.x * per, end = min(begin + per, n_segs);
    u32 sum = 0;
    for (int q = begin; q < end; ++q) {
        const long long len = seg_offsets_in[q + 1] - seg_offsets_in[q];
        sum += static_cast<u32>((len + kTile - 1) / kTile);
    }
    s_part[threadIdx.x] = sum;
    __syncthreads();
    for (int st = 1; st < 1024; st <<= 1) {
        const u32 v = threadIdx.x >= (unsigned)st ? s_part[threadIdx.x - st] : 0u;
        __syncthreads();
        s_part[threadIdx.x] += v;
        __syncthreads();
    }
    u32 run = s_part[threadIdx.x] - sum;
    for (int q = begin; q < end; ++q) {
        b.seg_first[q] = run;
        const long long len = seg_offsets_in[q + 1] - seg_offsets_in[q];
        run += static_cast<u32>((len + kTile - 1) / kTile);
    }
    if (threadIdx.x == 1023) {
        b.seg_first[n_segs] = s_part[1023];
        *b.n_tiles = s_part[1023];
    }
}

// Tile table: segment, first key and key count of every tile.
__global__ void __launch_bounds__(kThreads) seg_tiles_kernel(const long long* __restrict__ seg_offsets_in, int n_segs,
                                                             u32 max_tiles, SegBuild b) {
    const u32 total = *b.n_tiles;
    for (u32 t = blockIdx.x * kThreads + threadIdx.x; t < max_tiles; t += gridDim.x * kThreads) {
        if (t >= total) {
            b.tile_count[t] = 0;
            continue;
        }
        int lo = 0, hi = n_segs;  // last segment whose first tile is <= t
        while (hi - lo > 1) {
            const int mid = (lo + hi) >> 1;
            if (b.seg_first[mid] <= t)
                lo = mid;
            else
                hi = mid;
        }
        while (lo + 1 < n_segs && b.seg_first[lo + 1] <= t) ++lo;  // skip empty segments
        const long long start = seg_offsets_in[lo] + (long long)(t - b.seg_first[lo]) * kTile;
        const long long end = seg_offsets_in[lo + 1];
        b.tile_seg[t] = static_cast<u32>(lo);
        b.tile_base[t] = static_cast<u32>(start);
        b.tile_count[t] = static_cast<u32>(min((long long)kTile, end - start));
    }
}

// Per-segment digit histograms of all 8 passes, one block per tile.
__global__ void __launch_bounds__(kThreads) seg_hist_kernel(const Key* __restrict__ keys, SegTiles st, u32* seg_hist) {
    __shared__ u32 sh[kPasses][kRadix];
    const u32 t = blockIdx.x;
    const u32 count = st.tile_count[t];
    if (count == 0) return;
    for (int i = threadIdx.x; i < kPasses * kRadix; i += kThreads) (&sh[0][0])[i] = 0;
    __syncthreads();
    const u32 base = st.tile_base[t];
    for (u32 i = threadIdx.x; i < count; i += kThreads) {
        const Key k = __ldg(keys + base + i);
#pragma unroll
        for (int p = 0; p < kPasses; ++p) atomicAdd(&sh[p][(k >> (p * kRadixBits)) & (kRadix - 1)], 1u);
    }
    __syncthreads();
    u32* dst = seg_hist + (size_t)st.tile_seg[t] * kPasses * kRadix;
    for (int i = threadIdx.x; i < kPasses * kRadix; i += kThreads) {
        const u32 v = (&sh[0][0])[i];
        if (v) atomicAdd(dst + i, v);
    }
}

// Digit offsets per segment and pass: the segment start plus the exclusive scan of its histogram.
__global__ void seg_scan_kernel(const long long* __restrict__ seg_offsets_in, const u32* __restrict__ seg_hist,
                                u32* seg_offsets) {
    const int seg = blockIdx.x;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (warp >= kPasses) return;
    const u32* h = seg_hist + ((size_t)seg * kPasses + warp) * kRadix;
    u32* o = seg_offsets + ((size_t)seg * kPasses + warp) * kRadix;
    u32 carry = static_cast<u32>(seg_offsets_in[seg]);
    for (int base = 0; base < kRadix; base += 32) {
        const u32 v = h[base + lane];
        u32 incl = v;
        for (int sft = 1; sft < 32; sft <<= 1) {
            const u32 t = __shfl_up_sync(0xffffffffu, incl, sft);
            if (lane >= sft) incl += t;
        }
        o[base + lane] = carry + incl - v;
        carry += __shfl_sync(0xffffffffu, incl, 31);
    }
}

// Lanes of the warp whose value v (9 bits: an 8-bit digit or the marker kRadix) equals this
// lane's: one ballot per bit.
__device__ __forceinline__ u32 match_digit(u32 v) {
    u32 peers = 0xffffffffu;
#pragma unroll
    for (int b = 0; b <= kRadixBits; ++b) {
        const bool bit = (v >> b) & 1u;
        const u32 bal = __ballot_sync(0xffffffffu, bit);
        peers &= bit ? bal : ~bal;
    }
    return peers;
}

struct PassSmem {
    union {  // the tile in digit order: its keys, then (once they are written out) its values
        Key keys[kTile];
        u32 vals[kTile];
    } stage;
    unsigned char dig[kTile];  // digit of every staged key
    u32 warp_hist[kWarps][kRadix];  // per-warp digit counts, then each warp's first staging slot
    u32 delta[kRadix];              // output position minus staging slot, per digit
    u32 scan_tmp[kWarps];
};

// One digit pass. tile_pos[tile][d]: for a single-set sort the output position of the tile's
// first key of digit d; for a segmented sort the keys of digit d in all tiles before this one
// (over every segment), from which the tile's segment start is subtracted.
template <bool FIRST, bool SEG>
__global__ void __launch_bounds__(kThreads, CSTONE_SORT_MIN_BLOCKS)
    sort_pass_kernel(const Key* __restrict__ kin, Key* __restrict__ kout, const u32* __restrict__ vin,
                     u32* __restrict__ vout, long long n, int pass, const u32* __restrict__ tile_pos,
                     SegTiles seg) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    PassSmem& sm = *reinterpret_cast<PassSmem*>(smem_raw);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int shift = pass * kRadixBits;

    for (int i = tid; i < kWarps * kRadix; i += kThreads) (&sm.warp_hist[0][0])[i] = 0;
    __syncthreads();
    const u32 tile = blockIdx.x;
    u32 base, count;  // first key of the tile and keys in it (n < 2^30, so 32-bit offsets)
    if (SEG) {
        if (tile >= *seg.n_tiles) return;
        base = seg.tile_base[tile];
        count = seg.tile_count[tile];
    } else {
        base = tile * static_cast<u32>(kTile);
        const long long remain = n - (long long)base;
        count = remain < kTile ? static_cast<u32>(remain) : static_cast<u32>(kTile);
    }

    // ---- load (warp-striped: warp w owns keys base + w*32*kItems + it*32 + lane)
    Key key[kItems];
    u32 val[kItems];
    const Key* tkeys = kin + base;
    const u32 woff = static_cast<u32>(warp * 32 * kItems + lane);  // offset of item 0 within the tile
#pragma unroll
    for (int it = 0; it < kItems; ++it) {
        const u32 o = woff + it * 32;
        const bool ok = o < count;
        key[it] = ok ? __ldcg(tkeys + o) : ~static_cast<Key>(0);
        if (FIRST)
            val[it] = base + o;
        else
            val[it] = ok ? __ldcg(vin + base + o) : 0u;
    }
    auto digit_of = [&](int it) -> u32 {
        return (woff + it * 32 < count) ? static_cast<u32>((key[it] >> shift) & (kRadix - 1)) : static_cast<u32>(kRadix);
    };

    // ---- rank within the warp, in memory order (stable); ranks packed two per register.
    // Items are handled in groups: all matches of a group first, then the leaders' reservations
    // (shared-memory atomics of one warp to one address take effect in program order, so earlier
    // items keep lower ranks), then the broadcasts - so the round trips of a group overlap.
    constexpr int kGroup = kItems % 8 == 0 ? 8 : (kItems % 4 == 0 ? 4 : 2);
    u32 rank2[kItems / 2];
    const u32 lt = lanemask_lt();
#pragma unroll
    for (int g0 = 0; g0 < kItems; g0 += kGroup) {
        u32 peers[kGroup], before[kGroup];
#pragma unroll
        for (int q = 0; q < kGroup; ++q) peers[q] = match_digit(digit_of(g0 + q));
#pragma unroll
        for (int q = 0; q < kGroup; ++q) {
            const u32 d = digit_of(g0 + q);
            before[q] = 0;
            if (lane == __ffs(peers[q]) - 1 && d < kRadix)
                before[q] = atomicAdd(&sm.warp_hist[warp][d], static_cast<u32>(__popc(peers[q])));
        }
#pragma unroll
        for (int q = 0; q < kGroup; ++q) {
            const u32 r = __shfl_sync(0xffffffffu, before[q], __ffs(peers[q]) - 1) + __popc(peers[q] & lt);
            const int it = g0 + q;
            if (it & 1)
                rank2[it >> 1] |= r << 16;
            else
                rank2[it >> 1] = r;
        }
    }
    __syncthreads();

    // ---- per digit: tile total and per-warp exclusive offsets (thread t < 256 owns digit t)
    const bool owner = tid < kRadix;
    const int d = owner ? tid : 0;
    u32 total = 0, incl = 0;
    if (owner) {
#pragma unroll
        for (int w = 0; w < kWarps; ++w) total += sm.warp_hist[w][d];
        // block-wide exclusive scan of the totals over digits -> staging slots
        incl = total;
        for (int s = 1; s < 32; s <<= 1) {
            const u32 t = __shfl_up_sync(0xffffffffu, incl, s);
            if (lane >= s) incl += t;
        }
        if (lane == 31) sm.scan_tmp[warp] = incl;
    }
    __syncthreads();
    if (owner) {
        u32 wpre = 0;
        for (int w = 0; w < warp; ++w) wpre += sm.scan_tmp[w];
        const u32 start = wpre + incl - total;  // first staging slot of digit d
        // staging slot of warp w's first key of digit d
        u32 run = start;
#pragma unroll
        for (int w = 0; w < kWarps; ++w) {
            const u32 c = sm.warp_hist[w][d];
            sm.warp_hist[w][d] = run;
            run += c;
        }

        // output position of the tile's first key of digit d, minus its staging slot
        if (SEG) {
            const u32 sg = seg.tile_seg[tile];
            const u32 first_tile = seg.seg_first[sg];
            const u32 seg_digit_offset = seg.seg_offsets[((size_t)sg * kPasses + pass) * kRadix + d];
            sm.delta[d] = seg_digit_offset + (tile_pos[(size_t)tile * kRadix + d] -
                                              tile_pos[(size_t)first_tile * kRadix + d]) - start;
        } else
            sm.delta[d] = tile_pos[(size_t)tile * kRadix + d] - start;
    }
    __syncthreads();

    // ---- stage the keys in digit order and write each digit's run contiguously, then the same for
    // the values in the same buffer (one staging buffer instead of two leaves more of the SM's
    // L1 for the loads in flight: about 1 % faster on clustered keys)
    u32 slot2[kItems / 2];  // staging slot of every item (0xffff: none), two per register
#pragma unroll
    for (int it = 0; it < kItems; ++it) {
        const u32 dd = digit_of(it);
        u32 slot = 0xffffu;
        if (dd < kRadix) {
            const u32 r = (rank2[it >> 1] >> ((it & 1) * 16)) & 0xffffu;
            slot = sm.warp_hist[warp][dd] + r;
            sm.stage.keys[slot] = key[it];
        }
        if (it & 1)
            slot2[it >> 1] |= slot << 16;
        else
            slot2[it >> 1] = slot;
    }
    __syncthreads();
    for (u32 s = tid; s < count; s += kThreads) {
        const Key k = sm.stage.keys[s];
        const u32 dk = static_cast<u32>(k >> shift) & (kRadix - 1);
        sm.dig[s] = static_cast<unsigned char>(dk);
        kout[sm.delta[dk] + s] = k;
    }
    __syncthreads();
#pragma unroll
    for (int it = 0; it < kItems; ++it) {
        const u32 slot = (slot2[it >> 1] >> ((it & 1) * 16)) & 0xffffu;
        if (slot != 0xffffu) sm.stage.vals[slot] = val[it];
    }
    __syncthreads();
    for (u32 s = tid; s < count; s += kThreads) vout[sm.delta[sm.dig[s]] + s] = sm.stage.vals[s];
}

// ---- output offsets of every tile, ahead of a pass (single-set sorts). A tile's output position
// for digit d is the digit's global offset plus the keys of digit d in all earlier tiles; counting
// every tile first and scanning the counts replaces the look-back (which measured a third of the
// sort's time: tiles in flight wait on their predecessors' prefixes).
constexpr int kChunkTiles = 32;  // tiles per chunk of the two-level scan

// Digit counts of every tile of the pass (the tile partition of sort_pass_kernel; unused tiles of a
// segmented sort count nothing).
template <bool SEG>
__global__ void __launch_bounds__(kThreads) tile_count_kernel(const Key* __restrict__ kin, long long n, int shift,
                                                              unsigned short* __restrict__ counts, SegTiles seg) {
    __shared__ u32 wh[kWarps][kRadix];
    const int tid = threadIdx.x, warp = tid >> 5;
    for (int i = tid; i < kWarps * kRadix; i += kThreads) (&wh[0][0])[i] = 0;
    __syncthreads();
    long long base;
    u32 count;
    if (SEG) {
        const bool used = blockIdx.x < *seg.n_tiles;
        base = used ? seg.tile_base[blockIdx.x] : 0;
        count = used ? seg.tile_count[blockIdx.x] : 0u;
    } else {
        base = (long long)blockIdx.x * kTile;
        const long long remain = n - base;
        count = remain < kTile ? static_cast<u32>(remain) : static_cast<u32>(kTile);
    }
    const Key* tkeys = kin + base;
    const u32 woff = static_cast<u32>(warp * 32 * kItems + (tid & 31));
    Key kk[kItems];
#pragma unroll
    for (int it = 0; it < kItems; ++it) {
        const u32 o = woff + it * 32;
        kk[it] = o < count ? __ldcg(tkeys + o) : ~static_cast<Key>(0);
    }
#pragma unroll
    for (int it = 0; it < kItems; ++it) {
        const u32 o = woff + it * 32;
        if (o < count) atomicAdd(&wh[warp][static_cast<u32>((kk[it] >> shift) & (kRadix - 1))], 1u);
    }
    __syncthreads();
    for (int dd = tid; dd < kRadix; dd += kThreads) {
        u32 c = 0;
#pragma unroll
        for (int w = 0; w < kWarps; ++w) c += wh[w][dd];
        counts[(size_t)blockIdx.x * kRadix + dd] = static_cast<unsigned short>(c);
    }
}

// Per chunk of kChunkTiles tiles: the keys of every digit (thread = digit).
__global__ void __launch_bounds__(kRadix) chunk_sum_kernel(const unsigned short* __restrict__ counts, long long tiles,
                                                           u32* __restrict__ chunk) {
    const int d = threadIdx.x;
    const long long t0 = (long long)blockIdx.x * kChunkTiles;
    const long long t1 = t0 + kChunkTiles < tiles ? t0 + kChunkTiles : tiles;
    u32 sum = 0;
#pragma unroll 8
    for (long long t = t0; t < t1; ++t) sum += counts[t * kRadix + d];
    chunk[(size_t)d * gridDim.x + blockIdx.x] = sum;  // digit-major
}

// Exclusive scan of the chunk sums over the chunks, per digit: one block per digit over its
// contiguous row (in place). The row's total (the keys of digit d in the whole pass) goes to
// totals[d] unless totals is NULL.
__global__ void __launch_bounds__(1024) chunk_scan_kernel(u32* __restrict__ chunk, long long nchunks,
                                                          u32* __restrict__ totals) {
    __shared__ u32 s_warp[32];
    u32* row = chunk + (size_t)blockIdx.x * nchunks;
    const long long per = (nchunks + 1023) / 1024;
    const long long c0 = threadIdx.x * per, c1 = c0 + per < nchunks ? c0 + per : nchunks;
    u32 sum = 0;
    for (long long c = c0; c < c1; ++c) sum += row[c];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    u32 incl = sum;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const u32 t = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += t;
    }
    if (lane == 31) s_warp[warp] = incl;
    __syncthreads();
    u32 before = 0;
    for (int w = 0; w < warp; ++w) before += s_warp[w];
    if (totals && threadIdx.x == 1023) totals[blockIdx.x] = before + incl;
    u32 run = before + incl - sum;
    for (long long c = c0; c < c1; ++c) {
        const u32 v = row[c];
        row[c] = run;
        run += v;
    }
}

// Output position of every tile's first key of every digit (thread = digit): the digit's first
// position in the pass (the keys of all smaller digits: an exclusive scan of totals over the digits,
// done by every block; 0 when totals is NULL) plus the digit's keys in all earlier tiles.
__global__ void __launch_bounds__(kRadix) tile_offsets_kernel(const unsigned short* __restrict__ counts, long long tiles,
                                                              const u32* __restrict__ chunk,
                                                              const u32* __restrict__ totals,
                                                              u32* __restrict__ offsets) {
    static_assert(kRadix % 32 == 0 && kRadix <= 1024, "one thread per digit");
    __shared__ u32 s_warp[kRadix / 32];
    const int d = threadIdx.x, lane = d & 31, warp = d >> 5;
    u32 digit_first = 0;
    if (totals) {
        const u32 v = totals[d];
        u32 incl = v;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const u32 t = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += t;
        }
        if (lane == 31) s_warp[warp] = incl;
        __syncthreads();
        u32 before = 0;
        for (int w = 0; w < warp; ++w) before += s_warp[w];
        digit_first = before + incl - v;
    }
    const long long t0 = (long long)blockIdx.x * kChunkTiles;
    const long long t1 = t0 + kChunkTiles < tiles ? t0 + kChunkTiles : tiles;
    u32 run = digit_first + chunk[(size_t)d * gridDim.x + blockIdx.x];
    u32 v[kChunkTiles];
#pragma unroll
    for (int k = 0; k < kChunkTiles; ++k) v[k] = t0 + k < t1 ? counts[(t0 + k) * kRadix + d] : 0u;
#pragma unroll
    for (int k = 0; k < kChunkTiles; ++k) {
        if (t0 + k < t1) offsets[(t0 + k) * kRadix + d] = run;
        run += v[k];
    }
}

struct SortLayout {
    u32* totals;   // keys of each digit in the current pass
    u32* look[2];  // per-tile digit counts and output offsets
    u32* chunk;    // per-chunk digit sums, then their scan
    Key* keys_alt;
    u32* vals_alt;
    size_t bytes;
    long long tiles;
};

SortLayout sort_layout(void* ws, long long n) {
    SortLayout l;
    Carver c(ws);
    l.tiles = (n + kTile - 1) / kTile;
    l.totals = c.take<u32>(kRadix);
    l.look[0] = c.take<u32>((size_t)l.tiles * kRadix);
    l.look[1] = c.take<u32>((size_t)l.tiles * kRadix);
    l.chunk = c.take<u32>((size_t)((l.tiles + kChunkTiles - 1) / kChunkTiles) * kRadix);
    l.keys_alt = c.take<Key>((size_t)n);
    l.vals_alt = c.take<u32>((size_t)n);
    l.bytes = c.size();
    return l;
}

}  // namespace

size_t sort_ws_bytes(long long n) { return sort_layout(nullptr, n).bytes; }

#ifndef CSTONE_KEY32  // the allocation-free sort exists for 63-bit keys only
// ---------------------------------------------------------------- sort without allocation
// Scratch of cstone_sort_static: the same layout as the caller workspace of cstone_sort, sized for
// CSTONE_SORT_STATIC_MAX_KEYS keys, held in a file-scope device array that every GPU loading the
// library keeps until the process exits.
namespace {
constexpr size_t round256(size_t b) { return (b + 255) / 256 * 256; }
constexpr long long kStaticKeys = CSTONE_SORT_STATIC_MAX_KEYS;
constexpr size_t kStaticTiles = static_cast<size_t>((kStaticKeys + kTile - 1) / kTile);
constexpr size_t kStaticBytes = sizeof(WsHeader) + round256(kRadix * 4) + 2 * round256(kStaticTiles * kRadix * 4) +
                                round256((kStaticTiles + kChunkTiles - 1) / kChunkTiles * kRadix * 4) +
                                round256(static_cast<size_t>(kStaticKeys) * 8) +
                                round256(static_cast<size_t>(kStaticKeys) * 4);

__device__ __align__(256) unsigned char g_sort_scratch[kStaticBytes];

std::mutex g_static_mutex;
constexpr int kMaxDevices = 64;
void* g_static_scratch[kMaxDevices] = {};

// Device address of g_sort_scratch on the current device, looked up once per device. In host code
// the array's name is only a host-side stand-in, never a device address. The cache is not
// invalidated by cudaDeviceReset. A stream of another device than the current one is rejected.
int static_sort_scratch(void** out, cudaStream_t st) {
    int dev = 0;
    CST_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kMaxDevices)
        return fail(CSTONE_ERR_INVALID_ARG, "cstone_sort_static: device ordinal %d not supported", dev);
    if (st != nullptr && st != cudaStreamLegacy && st != cudaStreamPerThread) {
        int sdev = -1;
        CST_CUDA(cudaStreamGetDevice(st, &sdev));
        if (sdev != dev)
            return fail(CSTONE_ERR_INVALID_ARG, "cstone_sort_static: stream of device %d, current device %d", sdev,
                        dev);
    }
    std::lock_guard<std::mutex> lock(g_static_mutex);
    if (g_static_scratch[dev] == nullptr) {
        void* p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_sort_scratch);
        if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(g_sort_scratch)");
        g_static_scratch[dev] = p;
    }
    *out = g_static_scratch[dev];
    return CSTONE_OK;
}
}  // namespace
#endif

// The digit passes (an even number). Ping-pong: odd passes (1-based) write the workspace buffers,
// even passes the output, so the last pass lands in keys_out / perm. Ahead of each pass: tile
// counts (counts), chunk sums and their scan (chunk), and the per-tile positions (tile_pos).
template <bool SEG>
int run_passes(const Key* keys_in, Key* keys_out, u32* perm, long long n, long long tiles, u32* totals,
               u32* counts, u32* chunk, u32* tile_pos, Key* keys_alt, u32* vals_alt, SegTiles seg, cudaStream_t st) {
    const int smem = static_cast<int>(sizeof(PassSmem));
    CST_CUDA(cudaFuncSetAttribute(sort_pass_kernel<true, SEG>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
    CST_CUDA(cudaFuncSetAttribute(sort_pass_kernel<false, SEG>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
    const Key* ksrc = keys_in;
    const u32* vsrc = nullptr;
    const long long nchunks = (tiles + kChunkTiles - 1) / kChunkTiles;
    // tile counts as 16-bit words (a tile holds fewer than 2^16 keys) in the counts buffer
    unsigned short* counts16 = reinterpret_cast<unsigned short*>(counts);
    static_assert(kTile < 65536, "16-bit tile counts");
    static_assert(kPasses % 2 == 0, "the last pass must write the output buffers");
    for (int p = 0; p < kPasses; ++p) {
        Key* kdst = (p % 2 == 0) ? keys_alt : keys_out;
        u32* vdst = (p % 2 == 0) ? vals_alt : perm;
        tile_count_kernel<SEG><<<(unsigned)tiles, kThreads, 0, st>>>(ksrc, n, p * kRadixBits, counts16, seg);
        CST_LAUNCHED("tile_count_kernel");
        chunk_sum_kernel<<<(unsigned)nchunks, kRadix, 0, st>>>(counts16, tiles, chunk);
        CST_LAUNCHED("chunk_sum_kernel");
        // a segmented sort scans all tiles from 0 and places the digits per segment; each tile
        // subtracts its segment's first tile
        chunk_scan_kernel<<<kRadix, 1024, 0, st>>>(chunk, nchunks, SEG ? nullptr : totals);
        CST_LAUNCHED("chunk_scan_kernel");
        tile_offsets_kernel<<<(unsigned)nchunks, kRadix, 0, st>>>(counts16, tiles, chunk, SEG ? nullptr : totals,
                                                                  tile_pos);
        CST_LAUNCHED("tile_offsets_kernel");
        if (p == 0)
            sort_pass_kernel<true, SEG><<<(unsigned)tiles, kThreads, smem, st>>>(ksrc, kdst, vsrc, vdst, n, p,
                                                                                 tile_pos, seg);
        else
            sort_pass_kernel<false, SEG><<<(unsigned)tiles, kThreads, smem, st>>>(ksrc, kdst, vsrc, vdst, n, p,
                                                                                  tile_pos, seg);
        CST_LAUNCHED("sort_pass_kernel");
        ksrc = kdst;
        vsrc = vdst;
    }
    return CSTONE_OK;
}

int launch_sort(const Key* keys_in, Key* keys_out, u32* perm, long long n, void* ws, cudaStream_t st) {
    SortLayout l = sort_layout(ws, n);
    WsHeader* hdr = reinterpret_cast<WsHeader*>(ws);
    CST_CUDA(cudaMemsetAsync(hdr, 0, sizeof(WsHeader), st));
    if (n == 0) return CSTONE_OK;
    return run_passes<false>(keys_in, keys_out, perm, n, l.tiles, l.totals, l.look[0], l.chunk, l.look[1], l.keys_alt,
                             l.vals_alt, SegTiles{}, st);
}

// ---------------------------------------------------------------- segmented sort
namespace {
struct SegLayout {
    SegBuild b;
    u32* look[2];  // per-tile digit counts and positions
    u32* chunk;
    Key* keys_alt;
    u32* vals_alt;
    size_t bytes;
    long long max_tiles;
};

SegLayout seg_layout(void* ws, long long n, int n_segs) {
    SegLayout l;
    Carver c(ws);
    l.max_tiles = (n + kTile - 1) / kTile + n_segs;
    l.b.n_tiles = c.take<u32>(1);
    l.b.tile_seg = c.take<u32>((size_t)l.max_tiles);
    l.b.tile_base = c.take<u32>((size_t)l.max_tiles);
    l.b.tile_count = c.take<u32>((size_t)l.max_tiles);
    l.b.seg_first = c.take<u32>((size_t)n_segs + 1);
    l.b.seg_hist = c.take<u32>((size_t)n_segs * kPasses * kRadix);
    l.b.seg_offsets = c.take<u32>((size_t)n_segs * kPasses * kRadix);
    l.look[0] = c.take<u32>((size_t)l.max_tiles * kRadix);
    l.look[1] = c.take<u32>((size_t)l.max_tiles * kRadix);
    l.chunk = c.take<u32>((size_t)((l.max_tiles + kChunkTiles - 1) / kChunkTiles) * kRadix);
    l.keys_alt = c.take<Key>((size_t)n);
    l.vals_alt = c.take<u32>((size_t)n);
    l.bytes = c.size();
    return l;
}

}  // namespace

size_t sort_segmented_ws_bytes(long long n, int n_segs) { return seg_layout(nullptr, n, n_segs).bytes; }

int launch_sort_segmented(const Key* keys_in, Key* keys_out, u32* perm, long long n, const long long* seg_offsets,
                          int n_segs, void* ws, cudaStream_t st) {
    SegLayout l = seg_layout(ws, n, n_segs);
    WsHeader* hdr = reinterpret_cast<WsHeader*>(ws);
    CST_CUDA(cudaMemsetAsync(hdr, 0, sizeof(WsHeader), st));
    if (n == 0) return CSTONE_OK;
    CST_CUDA(cudaMemsetAsync(l.b.seg_hist, 0, (size_t)n_segs * kPasses * kRadix * sizeof(u32), st));
    seg_setup_kernel<<<1, 1024, 0, st>>>(seg_offsets, n_segs, l.b);
    CST_LAUNCHED("seg_setup_kernel");
    const long long want = (l.max_tiles + kThreads - 1) / kThreads;
    const int tgrid = static_cast<int>(want < (long long)sm_count() * 4 ? want : (long long)sm_count() * 4);
    seg_tiles_kernel<<<tgrid, kThreads, 0, st>>>(seg_offsets, n_segs, static_cast<u32>(l.max_tiles), l.b);
    CST_LAUNCHED("seg_tiles_kernel");
    const SegTiles view{l.b.n_tiles, l.b.tile_seg, l.b.tile_base, l.b.tile_count, l.b.seg_first, l.b.seg_offsets};
    seg_hist_kernel<<<(unsigned)l.max_tiles, kThreads, 0, st>>>(keys_in, view, l.b.seg_hist);
    CST_LAUNCHED("seg_hist_kernel");
    seg_scan_kernel<<<(unsigned)n_segs, 32 * kPasses, 0, st>>>(seg_offsets, l.b.seg_hist, l.b.seg_offsets);
    CST_LAUNCHED("seg_scan_kernel");
    return run_passes<true>(keys_in, keys_out, perm, n, l.max_tiles, nullptr, l.look[0], l.chunk, l.look[1], l.keys_alt,
                            l.vals_alt, view, st);
}

}  // namespace CST_NS

extern "C" {

int CSTONE_FN(sort_workspace_size)(int64_t n, size_t* bytes) {
    if (!bytes || n < 0 || n >= CSTONE_MAX_PARTICLES)
        return cst::fail(CSTONE_ERR_INVALID_ARG, CST_STR(CSTONE_FN(sort_workspace_size)) ": bad argument (n=%lld)",
                         (long long)n);
    *bytes = CST_NS::sort_ws_bytes(n);
    return CSTONE_OK;
}

int CSTONE_FN(sort)(const CST_KEY_C* keys_in, CST_KEY_C* keys_out, uint32_t* perm, int64_t n, void* ws,
                    size_t ws_bytes, void* stream) {
    if (n < 0 || n >= CSTONE_MAX_PARTICLES || (n > 0 && (!keys_in || !keys_out || !perm)))
        return cst::fail(CSTONE_ERR_INVALID_ARG, CST_STR(CSTONE_FN(sort)) ": bad argument (n=%lld)", (long long)n);
    if (int rc = cst::check_ws(ws, ws_bytes, CST_NS::sort_ws_bytes(n), CST_STR(CSTONE_FN(sort)))) return rc;
    return CST_NS::launch_sort(reinterpret_cast<const CST_NS::Key*>(keys_in), reinterpret_cast<CST_NS::Key*>(keys_out),
                               perm, n, ws, cst::as_stream(stream));
}

#ifndef CSTONE_KEY32
int cstone_sort_static(const uint64_t* keys_in, uint64_t* keys_out, uint32_t* perm, int64_t n, void* stream) {
    if (n < 0 || (n > 0 && (!keys_in || !keys_out || !perm)))
        return cst::fail(CSTONE_ERR_INVALID_ARG, "cstone_sort_static: bad argument (n=%lld)", (long long)n);
    if (n > CSTONE_SORT_STATIC_MAX_KEYS)
        return cst::fail(CSTONE_ERR_INVALID_ARG,
                         "cstone_sort_static: n=%lld exceeds the static scratch limit of %lld keys; use cstone_sort "
                         "with a workspace",
                         (long long)n, (long long)CSTONE_SORT_STATIC_MAX_KEYS);
    if (cst::sort_ws_bytes(n) > cst::kStaticBytes)
        return cst::fail(CSTONE_ERR_INVALID_ARG, "cstone_sort_static: static scratch too small");
    void* ws = nullptr;
    if (int rc = cst::static_sort_scratch(&ws, cst::as_stream(stream))) return rc;
    return cst::launch_sort(reinterpret_cast<const cst::u64*>(keys_in), reinterpret_cast<cst::u64*>(keys_out), perm,
                            n, ws, cst::as_stream(stream));
}

int cstone_sort_segmented_workspace_size(int64_t n, int32_t n_segs, size_t* bytes) {
    if (!bytes || n < 0 || n >= CSTONE_MAX_PARTICLES || n_segs < 1 || n_segs > (1 << 20))
        return cst::fail(CSTONE_ERR_INVALID_ARG, "cstone_sort_segmented_workspace_size: bad argument");
    *bytes = cst::sort_segmented_ws_bytes(n, n_segs);
    return CSTONE_OK;
}

int cstone_sort_segmented(const uint64_t* keys_in, uint64_t* keys_out, uint32_t* perm, int64_t n,
                          const int64_t* seg_offsets, int32_t n_segs, void* ws, size_t ws_bytes, void* stream) {
    if (n < 0 || n >= CSTONE_MAX_PARTICLES || n_segs < 1 || n_segs > (1 << 20) || !seg_offsets ||
        (n > 0 && (!keys_in || !keys_out || !perm)))
        return cst::fail(CSTONE_ERR_INVALID_ARG, "cstone_sort_segmented: bad argument (n=%lld, segments=%d)",
                         (long long)n, n_segs);
    if (keys_in == keys_out && n > 0)
        return cst::fail(CSTONE_ERR_INVALID_ARG, "cstone_sort_segmented: keys_in must not alias keys_out");
    if (int rc = cst::check_ws(ws, ws_bytes, cst::sort_segmented_ws_bytes(n, n_segs), "cstone_sort_segmented"))
        return rc;
    return cst::launch_sort_segmented(reinterpret_cast<const cst::u64*>(keys_in), reinterpret_cast<cst::u64*>(keys_out),
                                      perm, n, reinterpret_cast<const long long*>(seg_offsets), n_segs, ws,
                                      cst::as_stream(stream));
}

#endif

}  // extern "C"
