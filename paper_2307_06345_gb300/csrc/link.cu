// Fully linked octree from the cornerstone array (Sec. 5, steps 1-5), breadth-first.
//
// Node keys: every leaf i gives a node at level L - log8(K_{i+1} - K_i); every adjacent pair
// (K_i, K_{i+1}) whose first differing bit is the leading bit of an octal digit (d % 3 == 0 with
// d the number of equal leading bits of the 3L-bit keys, step 2) gives the internal node at level
// d / 3 that is the lowest common ancestor of the two leaves: the pair straddles the boundary
// between its child 3 and child 4, so each internal node appears exactly once.
//
// Breadth-first order (step 3): taken in array order, leaf i followed by pair i is an in-order
// walk of the tree, so the nodes of any one level already appear in key order. A stable
// partition of that sequence by level therefore gives the breadth-first layout without sorting
// 64-bit keys, and the offsets of the partition are the level offsets LO (step 4). This replaces
// the paper's digit-weight slot mapping of step 2 followed by a radix sort of NK: the final NK
// is the same. The partition is a counting sort with L + 1 buckets: per-tile level counts, one scan
// over (level, tile), and a scatter that ranks items stably inside each tile.
//
// Step 5: the first child of an internal node. In this layout every internal node has its 8
// children together and the sibling groups follow their parents' breadth-first order, so the
// children of the g-th internal node (counting internal nodes only, in breadth-first order) are
// the nodes 8 g + 1 .. 8 g + 8: the child index that the paper's search for the key << 3 in the
// next level finds. The scatter ranks every internal node among the internal nodes with a second
// counting sort of the pairs alone and writes CO (and the parent of every sibling group) directly.
// Batched sets still search (link_b_child_kernel).
#include "common.cuh"

namespace CST_NS {
namespace {

constexpr int kThreads = 256;
constexpr int kItems = 8;
constexpr int kTile = kThreads * kItems;
constexpr int kNumLevels = kLevels + 1;  // levels 0..L

__device__ __forceinline__ int leaf_level(Key delta) {  // delta is a power of 8
    return kLevels - key_ffs(delta) / 3;
}

// Level of the internal node implied by the pair (i, i+1), or -1 when d % 3 != 0.
__device__ __forceinline__ int pair_level(Key a, Key b) {
    int d = key_clz(a ^ b) - (kWordBits - kKeyBits);  // equal leading bits of the 3L-bit keys
    return (d >= 0 && d % 3 == 0) ? d / 3 : -1;
}

__device__ __forceinline__ Key placeholder(Key key, int level) {
    return (static_cast<Key>(1) << (3 * level)) | (key >> (3 * (kLevels - level)));
}

__global__ void __launch_bounds__(kThreads) link_count_kernel(const Key* __restrict__ K, u32 nl, u32 ntiles,
                                                              u32* __restrict__ counts, u32* __restrict__ pair_counts) {
    // per-thread counts per level (own column, no conflicts): all nodes, then internal nodes
    __shared__ u32 s_c[2][kNumLevels][kThreads];
    const int tid = threadIdx.x;
#pragma unroll
    for (int l = 0; l < kNumLevels; ++l) s_c[0][l][tid] = s_c[1][l][tid] = 0;
    const u32 tile = blockIdx.x;
    const u32 i0 = tile * kTile + tid * kItems;
    for (int k = 0; k < kItems; ++k) {
        u32 i = i0 + k;
        if (i >= nl) break;
        Key a = K[i], b = K[i + 1];
        s_c[0][leaf_level(b - a)][tid] += 1;
        if (i + 1 < nl) {
            int pl = pair_level(a, b);
            if (pl >= 0) {
                s_c[0][pl][tid] += 1;
                s_c[1][pl][tid] += 1;
            }
        }
    }
    __syncthreads();
    const int lane = tid & 31, warp = tid >> 5;
    for (int r = warp; r < 2 * kNumLevels; r += kThreads / 32) {
        const u32* row = &s_c[r / kNumLevels][r % kNumLevels][0];
        u32 v = 0;
#pragma unroll
        for (int q = 0; q < kThreads / 32; ++q) v += row[q * 32 + lane];
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (lane == 0) {
            if (r < kNumLevels)
                counts[(size_t)r * ntiles + tile] = v;
            else if (pair_counts)
                pair_counts[(size_t)(r - kNumLevels) * ntiles + tile] = v;
        }
    }
}

// Exclusive scans of the level-major (level, tile) counts of all nodes (half 0) and of the internal
// nodes alone (half 1), each of `len` entries, in chunks of kScanChunk: block (c, h) sums chunk c
// of half h, then block (c, h) adds the sums of the chunks before it and scans its chunk. LO comes
// from half 0 (LO[l] = offset of (l, 0), LO[22] = total); a total of all nodes different from
// n_expected, or of internal nodes different from (n_expected - 1) / 8, means the input was not a
// cornerstone array. Without LO (the batched (set, level, tile) counts, one half) the total goes
// to the entry after the scanned ones.
constexpr u32 kScanThreads = 1024;
constexpr u32 kScanPer = 4;
constexpr u32 kScanChunk = kScanThreads * kScanPer;

__global__ void __launch_bounds__(kScanThreads) link_scan_reduce_kernel(const u32* __restrict__ counts, u32 len,
                                                                        u32* __restrict__ partial) {
    __shared__ u32 s_warp[kScanThreads / 32];
    const u32 h = blockIdx.y, c = blockIdx.x;
    const u32* a = counts + (size_t)h * len;
    u32 sum = 0;
#pragma unroll
    for (u32 j = 0; j < kScanPer; ++j) {
        const u32 i = c * kScanChunk + j * kScanThreads + threadIdx.x;  // coalesced
        if (i < len) sum += a[i];
    }
    for (int o = 16; o > 0; o >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, o);
    if ((threadIdx.x & 31) == 0) s_warp[threadIdx.x >> 5] = sum;
    __syncthreads();
    if (threadIdx.x < 32) {
        u32 v = s_warp[threadIdx.x];
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (threadIdx.x == 0) partial[h * gridDim.x + c] = v;
    }
}

__global__ void __launch_bounds__(kScanThreads) link_scan_apply_kernel(u32* __restrict__ counts, u32 len, u32 ntiles,
                                                                       const u32* __restrict__ partial,
                                                                       int* __restrict__ LO, u32 n_expected,
                                                                       WsHeader* hdr) {
    __shared__ u32 s_warp[kScanThreads / 32];
    __shared__ u32 s_carry;
    const u32 h = blockIdx.y, c = blockIdx.x, nchunks = gridDim.x;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (warp == 0) {  // sums of the chunks before this one (and of all chunks, for the total)
        u32 before = 0, all = 0;
        for (u32 k = lane; k < nchunks; k += 32) {
            const u32 v = partial[h * nchunks + k];
            all += v;
            if (k < c) before += v;
        }
        for (int o = 16; o > 0; o >>= 1) {
            before += __shfl_xor_sync(0xffffffffu, before, o);
            all += __shfl_xor_sync(0xffffffffu, all, o);
        }
        if (lane == 0) {
            s_carry = before;
            if (c == nchunks - 1) {
                if (LO) {
                    const u32 want = h == 0 ? n_expected : (n_expected - 1) / 8;
                    if (h == 0) LO[kNumLevels] = static_cast<int>(all);
                    if (all != want) raise_error(hdr, CSTONE_ERR_INVALID_ARG, all);
                } else {
                    counts[(size_t)h * len + len] = all;  // without LO (batched sets): the total after the scan
                }
            }
        }
    }
    __syncthreads();
    u32* a = counts + (size_t)h * len;
    // thread t takes the kScanPer consecutive entries c * kScanChunk + t * kScanPer + j
    const u32 i0 = c * kScanChunk + threadIdx.x * kScanPer;
    u32 v[kScanPer], sum = 0;
#pragma unroll
    for (u32 j = 0; j < kScanPer; ++j) {
        v[j] = i0 + j < len ? a[i0 + j] : 0u;
        sum += v[j];
    }
    u32 incl = sum;
    for (int o = 1; o < 32; o <<= 1) {
        const u32 t = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += t;
    }
    if (lane == 31) s_warp[warp] = incl;
    __syncthreads();
    if (warp == 0) {
        u32 w = s_warp[lane];
        for (int o = 1; o < 32; o <<= 1) {
            const u32 t = __shfl_up_sync(0xffffffffu, w, o);
            if (lane >= o) w += t;
        }
        s_warp[lane] = w;
    }
    __syncthreads();
    u32 run = s_carry + (warp > 0 ? s_warp[warp - 1] : 0u) + incl - sum;
#pragma unroll
    for (u32 j = 0; j < kScanPer; ++j) {
        const u32 i = i0 + j;
        if (i < len) {
            a[i] = run;
            if (LO && h == 0 && i % ntiles == 0) LO[i / ntiles] = static_cast<int>(run);
        }
        run += v[j];
    }
}

__global__ void __launch_bounds__(kThreads) link_scatter_kernel(const Key* __restrict__ K, u32 nl, u32 ntiles,
                                                                const u32* __restrict__ offsets,
                                                                const u32* __restrict__ pair_offsets, u32 n_nodes,
                                                                Key* __restrict__ NK, int* __restrict__ leaf_to_node,
                                                                int* __restrict__ CO, int* __restrict__ parent) {
    __shared__ u32 s_rank[kNumLevels][kThreads];   // per-thread counts, then per-thread slots
    __shared__ u32 s_prank[kNumLevels][kThreads];  // the same for internal nodes only
    const int tid = threadIdx.x;
    const u32 tile = blockIdx.x;
    const u32 i0 = tile * kTile + tid * kItems;
    const u32 n_int = (n_nodes - 1) / 8;
#pragma unroll
    for (int l = 0; l < kNumLevels; ++l) s_rank[l][tid] = s_prank[l][tid] = 0;
    // count this thread's items per level (own column, no conflicts)
    for (int k = 0; k < kItems; ++k) {
        u32 i = i0 + k;
        if (i >= nl) break;
        Key a = K[i], b = K[i + 1];
        s_rank[leaf_level(b - a)][tid] += 1;
        if (i + 1 < nl) {
            int pl = pair_level(a, b);
            if (pl >= 0) {
                s_rank[pl][tid] += 1;
                s_prank[pl][tid] += 1;
            }
        }
    }
    __syncthreads();
    // exclusive scan of every level row across the threads, plus the tile's global offset
    const int lane = tid & 31, warp = tid >> 5;
    for (int r = warp; r < 2 * kNumLevels; r += kThreads / 32) {
        const int l = r % kNumLevels;
        u32* row = r < kNumLevels ? s_rank[l] : s_prank[l];
        const u32* off = r < kNumLevels ? offsets : pair_offsets;
        u32 v[kThreads / 32];
        u32 sum = 0;
#pragma unroll
        for (int q = 0; q < kThreads / 32; ++q) {
            v[q] = row[lane * (kThreads / 32) + q];
            sum += v[q];
        }
        u32 incl = sum;
        for (int s = 1; s < 32; s <<= 1) {
            u32 t = __shfl_up_sync(0xffffffffu, incl, s);
            if (lane >= s) incl += t;
        }
        u32 run = off[(size_t)l * ntiles + tile] + incl - sum;
#pragma unroll
        for (int q = 0; q < kThreads / 32; ++q) {
            row[lane * (kThreads / 32) + q] = run;
            run += v[q];
        }
    }
    __syncthreads();
    // emit in in-order sequence: leaf i, then the internal node of pair i; the g-th internal node
    // has its children at 8 g + 1
    for (int k = 0; k < kItems; ++k) {
        u32 i = i0 + k;
        if (i >= nl) break;
        Key a = K[i], b = K[i + 1];
        int ll = leaf_level(b - a);
        u32 x = s_rank[ll][tid]++;
        if (x < n_nodes) {
            NK[x] = placeholder(a, ll);
            CO[x] = 0;
            leaf_to_node[i] = static_cast<int>(x);
        }
        if (i + 1 < nl) {
            int pl = pair_level(a, b);
            if (pl >= 0) {
                u32 y = s_rank[pl][tid]++;
                u32 g = s_prank[pl][tid]++;
                if (y < n_nodes) {
                    NK[y] = placeholder(a, pl);
                    CO[y] = g < n_int ? static_cast<int>(8u * g + 1u) : 0;
                    if (parent && g < n_int) parent[g] = static_cast<int>(y);
                }
            }
        }
    }
}

struct LinkLayout {
    u32* counts;   // [2][ntiles * 22]: all nodes, then internal nodes, per (level, tile)
    u32* partial;  // [2][chunks] chunk sums of the scans
    u32 ntiles;
    u32 chunks;    // scan chunks per half
    size_t bytes;
};

LinkLayout link_layout(void* ws, long long nl) {
    LinkLayout l;
    Carver c(ws);
    l.ntiles = static_cast<u32>((nl + kTile - 1) / kTile);
    if (l.ntiles == 0) l.ntiles = 1;
    const u32 len = l.ntiles * kNumLevels;
    l.chunks = (len + kScanChunk - 1) / kScanChunk;
    l.counts = c.take<u32>((size_t)2 * len);
    l.partial = c.take<u32>((size_t)2 * l.chunks);
    l.bytes = c.size();
    return l;
}

// ------------------------------------------------------------------ batched sets
// Several cornerstone arrays stored back to back as elements (each set's leaves followed by its end
// key 8^L). Tiles are aligned to sets, so the per-tile level counts of set s are laid out at
// [tile_first[s] * 22 + level * tiles_of_s + k]: one scan over everything then yields, set by set
// and level by level, the node positions of a concatenated node array in which every set's tree is
// one contiguous breadth-first block.
struct LinkSets {
    const long long* elem_offsets;  // [S+1] first element of each set
    u32* n_tiles;                   // device scalar
    u32* tile_first;                // [S+1] first tile of each set
    u32* tile_set;                  // [max_tiles]
    u32* tile_elem;                 // [max_tiles] first leaf element of the tile
    u32* tile_count;                // [max_tiles]
    u32* node_first;                // [S+1] expected first node of each set
    int n_sets;
};

__global__ void __launch_bounds__(1024) link_b_setup_kernel(LinkSets ls) {
    __shared__ u32 s_t[1024], s_n[1024];
    const int per = (ls.n_sets + 1023) / 1024;
    const int begin = threadIdx.x * per, end = min(begin + per, ls.n_sets);
    u32 st = 0, sn = 0;
    for (int q = begin; q < end; ++q) {
        const long long nl = ls.elem_offsets[q + 1] - ls.elem_offsets[q] - 1;
        st += static_cast<u32>((nl + kTile - 1) / kTile);
        sn += static_cast<u32>(nl + (nl - 1) / 7);
    }
    s_t[threadIdx.x] = st;
    s_n[threadIdx.x] = sn;
    __syncthreads();
    for (int o = 1; o < 1024; o <<= 1) {
        const u32 a = threadIdx.x >= (unsigned)o ? s_t[threadIdx.x - o] : 0u;
        const u32 b = threadIdx.x >= (unsigned)o ? s_n[threadIdx.x - o] : 0u;
        __syncthreads();
        s_t[threadIdx.x] += a;
        s_n[threadIdx.x] += b;
        __syncthreads();
    }
    u32 rt = s_t[threadIdx.x] - st, rn = s_n[threadIdx.x] - sn;
    for (int q = begin; q < end; ++q) {
        ls.tile_first[q] = rt;
        ls.node_first[q] = rn;
        const long long nl = ls.elem_offsets[q + 1] - ls.elem_offsets[q] - 1;
        rt += static_cast<u32>((nl + kTile - 1) / kTile);
        rn += static_cast<u32>(nl + (nl - 1) / 7);
    }
    if (threadIdx.x == 1023) {
        ls.tile_first[ls.n_sets] = s_t[1023];
        ls.node_first[ls.n_sets] = s_n[1023];
        *ls.n_tiles = s_t[1023];
    }
}

__global__ void __launch_bounds__(kThreads) link_b_tiles_kernel(LinkSets ls, u32 max_tiles, u32 elem_cap,
                                                                int* __restrict__ leaf_to_node) {
    // elements between the actual count and the capacity map to no node
    const u32 ne = static_cast<u32>(ls.elem_offsets[ls.n_sets]);
    for (u32 e = ne + blockIdx.x * kThreads + threadIdx.x; e < elem_cap; e += gridDim.x * kThreads) leaf_to_node[e] = -1;
    const u32 total = *ls.n_tiles;
    for (u32 t = blockIdx.x * kThreads + threadIdx.x; t < max_tiles; t += gridDim.x * kThreads) {
        if (t >= total) {
            ls.tile_count[t] = 0;
            continue;
        }
        int lo = 0, hi = ls.n_sets;
        while (hi - lo > 1) {
            const int mid = (lo + hi) >> 1;
            if (ls.tile_first[mid] <= t)
                lo = mid;
            else
                hi = mid;
        }
        const long long e0 = ls.elem_offsets[lo] + (long long)(t - ls.tile_first[lo]) * kTile;
        const long long last_leaf_end = ls.elem_offsets[lo + 1] - 1;  // the end key is not a leaf
        ls.tile_set[t] = static_cast<u32>(lo);
        ls.tile_elem[t] = static_cast<u32>(e0);
        ls.tile_count[t] = static_cast<u32>(min((long long)kTile, last_leaf_end - e0));
    }
}

__device__ __forceinline__ u32 count_index(const LinkSets& ls, u32 set, int level, u32 k) {
    const u32 tf = ls.tile_first[set], nt = ls.tile_first[set + 1] - tf;
    return tf * kNumLevels + static_cast<u32>(level) * nt + k;
}

__global__ void __launch_bounds__(kThreads) link_b_count_kernel(const Key* __restrict__ K, LinkSets ls,
                                                                u32* __restrict__ counts) {
    __shared__ u32 s_cnt[kNumLevels];
    const u32 tile = blockIdx.x;
    const u32 cnt = ls.tile_count[tile];
    if (cnt == 0) return;
    if (threadIdx.x < kNumLevels) s_cnt[threadIdx.x] = 0;
    __syncthreads();
    const u32 e0 = ls.tile_elem[tile];
    for (u32 q = threadIdx.x; q < cnt; q += kThreads) {
        const u32 e = e0 + q;
        const Key a = K[e], b = K[e + 1];
        atomicAdd(&s_cnt[leaf_level(b - a)], 1u);
        if (b != kKeyEnd) {
            const int pl = pair_level(a, b);
            if (pl >= 0) atomicAdd(&s_cnt[pl], 1u);
        }
    }
    __syncthreads();
    const u32 set = ls.tile_set[tile];
    if (threadIdx.x < kNumLevels)
        counts[count_index(ls, set, threadIdx.x, tile - ls.tile_first[set])] = s_cnt[threadIdx.x];
}

// Level offsets of every set (global node indices), a size check per set, and -1 for the
// leaf_to_node entries of the end keys.
__global__ void link_b_lo_kernel(const u32* __restrict__ counts, LinkSets ls, int* __restrict__ LO,
                                 int* __restrict__ leaf_to_node, WsHeader* hdr) {
    const u32 total_len = *ls.n_tiles * kNumLevels;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < ls.n_sets * (kNumLevels + 1);
         i += gridDim.x * blockDim.x) {
        const int set = i / (kNumLevels + 1), l = i % (kNumLevels + 1);
        u32 v;
        if (l < kNumLevels)
            v = counts[count_index(ls, set, l, 0)];
        else
            v = set + 1 < ls.n_sets ? counts[count_index(ls, set + 1, 0, 0)] : counts[total_len];
        LO[i] = static_cast<int>(v);
        if (l == kNumLevels) {
            const u32 first = counts[count_index(ls, set, 0, 0)];
            if (v - first != ls.node_first[set + 1] - ls.node_first[set])
                raise_error(hdr, CSTONE_ERR_INVALID_ARG, static_cast<u32>(set));
            leaf_to_node[ls.elem_offsets[set + 1] - 1] = -1;
        }
    }
}

__global__ void __launch_bounds__(kThreads) link_b_scatter_kernel(const Key* __restrict__ K, LinkSets ls,
                                                                  const u32* __restrict__ offsets, u32 n_nodes,
                                                                  Key* __restrict__ NK, int* __restrict__ leaf_to_node) {
    __shared__ u32 s_rank[kNumLevels][kThreads];
    const int tid = threadIdx.x;
    const u32 tile = blockIdx.x;
    const u32 cnt = ls.tile_count[tile];
    if (cnt == 0) return;
    const u32 e0 = ls.tile_elem[tile];
    const u32 set = ls.tile_set[tile];
    const u32 k_in_set = tile - ls.tile_first[set];
    const u32 i0 = tid * kItems;
#pragma unroll
    for (int l = 0; l < kNumLevels; ++l) s_rank[l][tid] = 0;
    for (int k = 0; k < kItems; ++k) {
        const u32 q = i0 + k;
        if (q >= cnt) break;
        const Key a = K[e0 + q], b = K[e0 + q + 1];
        s_rank[leaf_level(b - a)][tid] += 1;
        if (b != kKeyEnd) {
            const int pl = pair_level(a, b);
            if (pl >= 0) s_rank[pl][tid] += 1;
        }
    }
    __syncthreads();
    const int lane = tid & 31, warp = tid >> 5;
    for (int l = warp; l < kNumLevels; l += kThreads / 32) {
        u32 v[kThreads / 32];
        u32 sum = 0;
#pragma unroll
        for (int q = 0; q < kThreads / 32; ++q) {
            v[q] = s_rank[l][lane * (kThreads / 32) + q];
            sum += v[q];
        }
        u32 incl = sum;
        for (int o = 1; o < 32; o <<= 1) {
            const u32 t = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += t;
        }
        u32 run = offsets[count_index(ls, set, l, k_in_set)] + incl - sum;
#pragma unroll
        for (int q = 0; q < kThreads / 32; ++q) {
            s_rank[l][lane * (kThreads / 32) + q] = run;
            run += v[q];
        }
    }
    __syncthreads();
    for (int k = 0; k < kItems; ++k) {
        const u32 q = i0 + k;
        if (q >= cnt) break;
        const u32 e = e0 + q;
        const Key a = K[e], b = K[e + 1];
        const int ll = leaf_level(b - a);
        const u32 x = s_rank[ll][tid]++;
        if (x < n_nodes) {
            NK[x] = placeholder(a, ll);
            leaf_to_node[e] = static_cast<int>(x);
        }
        if (b != kKeyEnd) {
            const int pl = pair_level(a, b);
            if (pl >= 0) {
                const u32 y = s_rank[pl][tid]++;
                if (y < n_nodes) NK[y] = placeholder(a, pl);
            }
        }
    }
}

__global__ void __launch_bounds__(kThreads) link_b_child_kernel(const Key* __restrict__ NK, u32 node_cap, int n_sets,
                                                                const int* __restrict__ LO, int* __restrict__ CO) {
    const u32 last = static_cast<u32>(LO[n_sets * (kNumLevels + 1) - 1]);  // nodes of all sets
    const u32 n_nodes = last < node_cap ? last : node_cap;
    for (u32 x = blockIdx.x * kThreads + threadIdx.x; x < n_nodes; x += gridDim.x * kThreads) {
        int lo_s = 0, hi_s = n_sets;  // set whose node block contains x
        while (hi_s - lo_s > 1) {
            const int mid = (lo_s + hi_s) >> 1;
            if (static_cast<u32>(LO[mid * (kNumLevels + 1)]) <= x)
                lo_s = mid;
            else
                hi_s = mid;
        }
        const int* row = LO + lo_s * (kNumLevels + 1);
        const Key k = NK[x];
        const int level = (kWordBits - 1 - key_clz(k)) / 3;
        int c = 0;
        if (level < kLevels) {
            const Key want = k << 3;
            u32 lo = min(static_cast<u32>(row[level + 1]), n_nodes);
            u32 hi = min(static_cast<u32>(row[level + 2]), n_nodes);
            const u32 end = hi;
            while (lo < hi) {
                const u32 mid = lo + ((hi - lo) >> 1);
                if (NK[mid] < want)
                    lo = mid + 1;
                else
                    hi = mid;
            }
            if (lo < end && NK[lo] == want) c = static_cast<int>(lo);
        }
        CO[x] = c;
    }
}

struct LinkBLayout {
    LinkSets ls;
    u32* counts;   // [max_tiles * 22 + 1]: (set, level, tile) counts, their exclusive scan, the total
    u32* partial;  // [chunks] chunk sums of the scan
    u32 max_tiles;
    u32 chunks;
    size_t bytes;
};

LinkBLayout link_b_layout(void* ws, long long n_elements, int n_sets) {
    LinkBLayout l;
    Carver c(ws);
    l.max_tiles = static_cast<u32>((n_elements + kTile - 1) / kTile + n_sets);
    l.ls.n_tiles = c.take<u32>(1);
    l.ls.tile_first = c.take<u32>((size_t)n_sets + 1);
    l.ls.tile_set = c.take<u32>(l.max_tiles);
    l.ls.tile_elem = c.take<u32>(l.max_tiles);
    l.ls.tile_count = c.take<u32>(l.max_tiles);
    l.ls.node_first = c.take<u32>((size_t)n_sets + 1);
    l.ls.n_sets = n_sets;
    l.ls.elem_offsets = nullptr;
    l.counts = c.take<u32>((size_t)l.max_tiles * kNumLevels + 1);
    l.chunks = static_cast<u32>(((size_t)l.max_tiles * kNumLevels + kScanChunk - 1) / kScanChunk);
    l.partial = c.take<u32>(l.chunks);
    l.bytes = c.size();
    return l;
}

}  // namespace

size_t link_batched_ws_bytes(long long n_elements, int n_sets) { return link_b_layout(nullptr, n_elements, n_sets).bytes; }

int launch_link_batched(const Key* K, long long n_elements, const long long* elem_offsets, int n_sets, Key* NK,
                        int* CO, int* LO, int* leaf_to_node, long long n_nodes, void* ws, cudaStream_t st) {
    LinkBLayout l = link_b_layout(ws, n_elements, n_sets);
    l.ls.elem_offsets = elem_offsets;
    WsHeader* hdr = reinterpret_cast<WsHeader*>(ws);
    CST_CUDA(cudaMemsetAsync(hdr, 0, sizeof(WsHeader), st));
    CST_CUDA(cudaMemsetAsync(l.counts, 0, ((size_t)l.max_tiles * kNumLevels + 1) * sizeof(u32), st));
    link_b_setup_kernel<<<1, 1024, 0, st>>>(l.ls);
    CST_LAUNCHED("link_b_setup_kernel");
    const long long want = (l.max_tiles + kThreads - 1) / kThreads;
    const int tgrid = static_cast<int>(want < (long long)sm_count() * 4 ? want : (long long)sm_count() * 4);
    link_b_tiles_kernel<<<tgrid, kThreads, 0, st>>>(l.ls, l.max_tiles, static_cast<u32>(n_elements), leaf_to_node);
    CST_LAUNCHED("link_b_tiles_kernel");
    link_b_count_kernel<<<l.max_tiles, kThreads, 0, st>>>(K, l.ls, l.counts);
    CST_LAUNCHED("link_b_count_kernel");
    // one exclusive scan over all (set, level, tile) counts; unused tail entries are zero
    const u32 len = l.max_tiles * kNumLevels;
    link_scan_reduce_kernel<<<dim3(l.chunks, 1), kScanThreads, 0, st>>>(l.counts, len, l.partial);
    CST_LAUNCHED("link_scan_reduce_kernel");
    link_scan_apply_kernel<<<dim3(l.chunks, 1), kScanThreads, 0, st>>>(l.counts, len, 1u, l.partial, nullptr, 0u, hdr);
    CST_LAUNCHED("link_scan_apply_kernel");
    const int lo_threads = n_sets * (kNumLevels + 1);
    link_b_lo_kernel<<<(lo_threads + 255) / 256, 256, 0, st>>>(l.counts, l.ls, LO, leaf_to_node, hdr);
    CST_LAUNCHED("link_b_lo_kernel");
    link_b_scatter_kernel<<<l.max_tiles, kThreads, 0, st>>>(K, l.ls, l.counts, static_cast<u32>(n_nodes), NK,
                                                            leaf_to_node);
    CST_LAUNCHED("link_b_scatter_kernel");
    const long long wantc = (n_nodes + kThreads - 1) / kThreads;
    const int cgrid = static_cast<int>(wantc < (long long)sm_count() * 8 ? (wantc > 0 ? wantc : 1) : (long long)sm_count() * 8);
    link_b_child_kernel<<<cgrid, kThreads, 0, st>>>(NK, static_cast<u32>(n_nodes), n_sets, LO, CO);
    CST_LAUNCHED("link_b_child_kernel");
    return CSTONE_OK;
}

namespace {
}  // namespace

size_t link_ws_bytes(long long nl) { return link_layout(nullptr, nl).bytes; }

int launch_link(const Key* K, long long nl, Key* NK, int* CO, int* LO, int* leaf_to_node, int* parent, void* ws,
                cudaStream_t st) {
    LinkLayout l = link_layout(ws, nl);
    WsHeader* hdr = reinterpret_cast<WsHeader*>(ws);
    CST_CUDA(cudaMemsetAsync(hdr, 0, sizeof(WsHeader), st));
    const u32 n_nodes = static_cast<u32>(nl + (nl - 1) / 7);
    const u32 len = l.ntiles * kNumLevels;
    u32* pair_counts = l.counts + len;
    link_count_kernel<<<l.ntiles, kThreads, 0, st>>>(K, static_cast<u32>(nl), l.ntiles, l.counts, pair_counts);
    CST_LAUNCHED("link_count_kernel");
    link_scan_reduce_kernel<<<dim3(l.chunks, 2), kScanThreads, 0, st>>>(l.counts, len, l.partial);
    CST_LAUNCHED("link_scan_reduce_kernel");
    link_scan_apply_kernel<<<dim3(l.chunks, 2), kScanThreads, 0, st>>>(l.counts, len, l.ntiles, l.partial, LO, n_nodes,
                                                                        hdr);
    CST_LAUNCHED("link_scan_apply_kernel");
    link_scatter_kernel<<<l.ntiles, kThreads, 0, st>>>(K, static_cast<u32>(nl), l.ntiles, l.counts, pair_counts,
                                                       n_nodes, NK, leaf_to_node, CO, parent);
    CST_LAUNCHED("link_scatter_kernel");
    return CSTONE_OK;
}

}  // namespace CST_NS

extern "C" {

int CSTONE_FN(link_workspace_size)(int64_t n_leaves, size_t* bytes) {
    if (!bytes || n_leaves < 1 || n_leaves > CSTONE_MAX_LEAVES)
        return cst::fail(CSTONE_ERR_INVALID_ARG, CST_STR(CSTONE_FN(link_workspace_size)) ": bad argument");
    *bytes = CST_NS::link_ws_bytes(n_leaves);
    return CSTONE_OK;
}

int CSTONE_FN(link_tree)(const CST_KEY_C* leaves, int64_t n_leaves, CST_KEY_C* node_keys, int32_t* child,
                         int32_t* level_offsets, int32_t* leaf_to_node, int32_t* parent, void* ws, size_t ws_bytes,
                         void* stream) {
    if (n_leaves < 1 || n_leaves > CSTONE_MAX_LEAVES || (n_leaves - 1) % 7 != 0 || !leaves || !node_keys || !child ||
        !level_offsets || !leaf_to_node)
        return cst::fail(CSTONE_ERR_INVALID_ARG,
                         CST_STR(CSTONE_FN(link_tree)) ": bad argument (n_leaves=%lld must be 1 + 7k, arrays non-NULL)",
                         (long long)n_leaves);
    if (int rc = cst::check_ws(ws, ws_bytes, CST_NS::link_ws_bytes(n_leaves), CST_STR(CSTONE_FN(link_tree))))
        return rc;
    return CST_NS::launch_link(reinterpret_cast<const CST_NS::Key*>(leaves), n_leaves,
                               reinterpret_cast<CST_NS::Key*>(node_keys), child, level_offsets, leaf_to_node, parent,
                               ws, cst::as_stream(stream));
}

#ifndef CSTONE_KEY32  // batched builds exist for 63-bit keys only
int cstone_link_batched_workspace_size(int64_t n_elements, int32_t n_sets, size_t* bytes) {
    if (!bytes || n_sets < 1 || n_sets > (1 << 20) || n_elements < 2 * (int64_t)n_sets ||
        n_elements > CSTONE_MAX_LEAVES)
        return cst::fail(CSTONE_ERR_INVALID_ARG, "cstone_link_batched_workspace_size: bad argument");
    *bytes = cst::link_batched_ws_bytes(n_elements, n_sets);
    return CSTONE_OK;
}

int cstone_link_tree_batched(const uint64_t* elements, int64_t n_elements, const int64_t* element_offsets,
                             int32_t n_sets, int64_t n_nodes, uint64_t* node_keys, int32_t* child,
                             int32_t* level_offsets, int32_t* leaf_to_node, void* ws, size_t ws_bytes, void* stream) {
    if (n_sets < 1 || n_sets > (1 << 20) || n_elements < 2 * (int64_t)n_sets || n_elements > CSTONE_MAX_LEAVES ||
        n_nodes < n_sets || n_nodes > 2 * (int64_t)CSTONE_MAX_LEAVES || !elements || !element_offsets ||
        !node_keys || !child || !level_offsets || !leaf_to_node)
        return cst::fail(CSTONE_ERR_INVALID_ARG, "cstone_link_tree_batched: bad argument");
    if (int rc = cst::check_ws(ws, ws_bytes, cst::link_batched_ws_bytes(n_elements, n_sets),
                               "cstone_link_tree_batched"))
        return rc;
    return cst::launch_link_batched(reinterpret_cast<const cst::u64*>(elements), n_elements,
                                    reinterpret_cast<const long long*>(element_offsets), n_sets,
                                    reinterpret_cast<cst::u64*>(node_keys), child, level_offsets, leaf_to_node,
                                    n_nodes, ws, cst::as_stream(stream));
}

#endif

}  // extern "C"
