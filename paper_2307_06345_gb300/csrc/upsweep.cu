// Upsweeps over the linked octree (Sec. 5 node properties; Sec. 7 computes them bottom-up: a leaf
// from its particles, an internal node from its eight children).
//
// Both upsweeps walk the levels of the breadth-first tree from the deepest up in one cooperative
// launch: the leaves' values are written first, then every internal node of a level combines its 8
// children (in child order, so results do not depend on timing), with a bounded grid barrier
// between levels. Level l occupies nodes [LO[l], LO[l+1]); a level whose next level is empty has no
// internal node and is skipped.
//
// Multipoles (four launches: pack, leaf sums, sums of the few leaves too large for one group of
// lanes, level-by-level combination; the pack is skipped when the key pass wrote the records):
// FP32 accumulation with compensation. Each sum is a pair (sum, compensation) updated with an exact
// two-sum step (Neumaier), and the pairs of mass and second moments are carried up the tree in
// scratch so the compensation survives all L levels. Positions are held in 64-bit fixed point
// (records.cuh), so coordinate differences are exact and are rounded to FP32 once; the expansion
// centre (centre of mass) is kept in fixed point and written out in FP64.
// A leaf takes its first particle as the anchor for the differences, an internal node its first
// non-empty child's centre. The stored centre c' is the centre of mass rounded (the FP32 quotient
// of the first moments, on the fixed-point grid), and every second moment is taken about c'. Each
// node also carries its residual first moment r = sum m (x - c') (zero for the exact centre; the
// rounding of c' makes it about -M (c' - c)), so that an internal node combines its children with
// the exact parallel-axis shift about its own c':
//   Q = sum_k [Q_k + M_k e_k e_k^T + r_k e_k^T + e_k r_k^T],  r = sum_k [r_k + M_k e_k],
// with e_k = c'_k - c' (exact in fixed point). Dropping the r_k terms would leave an error of
// order |c'_k - c_k| |e_k| M_k, which is not small against Q when the first moments were taken
// about an anchor far from a tight concentration of the node's mass.
#include "common.cuh"
#include "records.cuh"

namespace CST_NS {
namespace {

constexpr int kThreads = 256;
// Levels with at most this many internal nodes are combined by one block (see the level loops).
constexpr u32 kSmallLevel = 2 * kThreads;

// ---------------------------------------------------------------------------- counts
constexpr int kNumLevels = kLevels + 1;

// The internal nodes in breadth-first order of their children. Every node but the root is a child,
// and siblings are stored together in parent order, so the children of internal node x start at
// child[x] = 8 g + 1 for the g-th internal node in that order, and the internal nodes of level l are
// g in [(LO[l + 1] - 1) / 8, (LO[l + 2] - 1) / 8). internal[g] = x lets a level's threads take only
// its internal nodes instead of all its nodes (most of which are leaves). A child index off that
// pattern is recorded in the error word and skipped.
__device__ __forceinline__ void list_internal(const int* __restrict__ child, u32 n_nodes, u32 n_int, int* internal,
                                              u32 gtid, u32 gthreads, WsHeader* hdr) {
    for (u32 x = gtid; x < n_nodes; x += gthreads) {
        const int c = child[x];
        if (c == 0) continue;
        const u32 g = static_cast<u32>(c - 1) >> 3;
        if (c < 1 || ((static_cast<u32>(c) - 1u) & 7u) != 0u || g >= n_int) {
            raise_error(hdr, CSTONE_ERR_INVALID_ARG, 0x74000u);
            continue;
        }
        internal[g] = static_cast<int>(x);
    }
}

// Range [g0, g1) of the internal nodes of level l (empty for a malformed level table).
__device__ __forceinline__ void internal_range(const int* s_lo, int l, u32 n_int, u32& g0, u32& g1) {
    g0 = static_cast<u32>(s_lo[l + 1] - 1) >> 3;
    g1 = min(static_cast<u32>(s_lo[l + 2] - 1) >> 3, n_int);
}

__global__ void __launch_bounds__(kThreads) upsweep_counts_kernel(const u32* __restrict__ leaf_counts, u32 nl,
                                                                  const int* __restrict__ leaf_to_node,
                                                                  const int* __restrict__ child,
                                                                  const int* __restrict__ level_offsets,
                                                                  u32* __restrict__ node_counts, int* internal,
                                                                  GridBarrier* bar, WsHeader* hdr) {
    __shared__ int s_lo[kNumLevels + 1];
    if (threadIdx.x <= kNumLevels) s_lo[threadIdx.x] = level_offsets[threadIdx.x];
    __syncthreads();
    const u32 gtid = blockIdx.x * kThreads + threadIdx.x, gthreads = gridDim.x * kThreads;
    const u32 n_int = (nl - 1) / 7;
    const u32 n_nodes = nl + n_int;  // an index outside is recorded in the error word and skipped
    for (u32 i = gtid; i < nl; i += gthreads) {
        const int v = leaf_to_node[i];
        if (v >= 0 && static_cast<u32>(v) < n_nodes)
            node_counts[v] = leaf_counts[i];
        else
            raise_error(hdr, CSTONE_ERR_INVALID_ARG, 0x71000u);
    }
    list_internal(child, n_nodes, n_int, internal, gtid, gthreads, hdr);
    grid_barrier(bar, hdr);
    auto combine = [&](u32 g) {
        const u32 c = 8u * g + 1u;  // c + 7 <= 8 n_int = n_nodes - 1
        const int x = internal[g];
        u32 sum = 0;
#pragma unroll
        for (int k = 0; k < 8; ++k) sum += __ldcg(node_counts + c + k);
        if (x < 0 || static_cast<u32>(x) >= n_nodes || static_cast<u32>(child[x]) != c) {
            raise_error(hdr, CSTONE_ERR_INVALID_ARG, 0x73000u);
            return;
        }
        node_counts[x] = sum;
    };
    // A level of at most kSmallLevel internal nodes is summed by block 0 alone, followed by a block
    // barrier instead of a grid barrier (the top levels and the deepest levels of a clustered tree
    // are small); a grid barrier precedes the next level that the whole grid sums.
    bool pending = false;  // block 0 wrote levels since the last grid barrier (the same in every block)
    for (int l = kLevels - 1; l >= 0; --l) {
        if (s_lo[l + 2] == s_lo[l + 1]) continue;  // no internal node at level l
        u32 g0, g1;
        internal_range(s_lo, l, n_int, g0, g1);
        if (g1 <= g0 + kSmallLevel) {
            if (blockIdx.x == 0) {
                for (u32 g = g0 + threadIdx.x; g < g1; g += kThreads) combine(g);
                __syncthreads();
            }
            pending = true;
            continue;
        }
        if (pending) grid_barrier(bar, hdr);
        for (u32 g = g0 + gtid; g < g1; g += gthreads) combine(g);
        grid_barrier(bar, hdr);
        pending = false;
    }
}

// Batched sets: the trees of all sets in one concatenated node array, level offsets per set
// ([set][23], global node indices). Each level is processed for all sets at once: every block
// scans the sets' level sizes in shared memory and maps a flat item index to (set, node).
constexpr int kMaxBatchSets = 4096;

__global__ void __launch_bounds__(kThreads) upsweep_counts_batched_kernel(
    const u32* __restrict__ elem_counts, u32 n_elements, const int* __restrict__ leaf_to_node,
    const int* __restrict__ child, const int* __restrict__ level_offsets, int n_sets, u32* __restrict__ node_counts,
    GridBarrier* bar, WsHeader* hdr) {
    __shared__ u32 s_prefix[kMaxBatchSets + 1];
    __shared__ u32 s_warp[kThreads / 32];
    const u32 gtid = blockIdx.x * kThreads + threadIdx.x, gthreads = gridDim.x * kThreads;
    constexpr int kRow = kNumLevels + 1;
    // nodes of all sets (the node arrays hold at least this many); an index outside is recorded
    // in the error word and skipped
    const u32 n_nodes = static_cast<u32>(level_offsets[n_sets * kRow - 1]);
    for (u32 e = gtid; e < n_elements; e += gthreads) {
        const int v = leaf_to_node[e];
        if (v >= 0) {
            if (static_cast<u32>(v) < n_nodes)
                node_counts[v] = elem_counts[e];
            else
                raise_error(hdr, CSTONE_ERR_INVALID_ARG, 0x71000u);
        }
    }
    grid_barrier(bar, hdr);
    for (int l = kLevels - 1; l >= 0; --l) {
        // exclusive prefix over sets of the number of level-l nodes that can have children
        const int per = (n_sets + kThreads - 1) / kThreads;
        const int b0 = threadIdx.x * per, b1 = min(b0 + per, n_sets);
        u32 sum = 0;
        for (int q = b0; q < b1; ++q) {
            const int* row = level_offsets + q * kRow;
            sum += (row[l + 2] > row[l + 1]) ? static_cast<u32>(row[l + 1] - row[l]) : 0u;
        }
        u32 incl = sum;
        const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
        for (int o = 1; o < 32; o <<= 1) {
            const u32 t = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += t;
        }
        if (lane == 31) s_warp[warp] = incl;
        __syncthreads();
        u32 wpre = 0, total = 0;
        for (int w = 0; w < kThreads / 32; ++w) {
            if (w < warp) wpre += s_warp[w];
            total += s_warp[w];
        }
        u32 run = wpre + incl - sum;
        for (int q = b0; q < b1; ++q) {
            s_prefix[q] = run;
            const int* row = level_offsets + q * kRow;
            run += (row[l + 2] > row[l + 1]) ? static_cast<u32>(row[l + 1] - row[l]) : 0u;
        }
        if (threadIdx.x == 0) s_prefix[n_sets] = total;
        __syncthreads();
        if (total == 0) continue;  // no internal node at level l in any set (uniform across blocks)
        for (u32 k = gtid; k < total; k += gthreads) {
            int a = 0, c = n_sets;  // last set whose prefix is <= k
            while (c - a > 1) {
                const int mid = (a + c) >> 1;
                if (s_prefix[mid] <= k)
                    a = mid;
                else
                    c = mid;
            }
            while (a + 1 < n_sets && s_prefix[a + 1] <= k) ++a;
            const u32 x = static_cast<u32>(level_offsets[a * kRow + l]) + (k - s_prefix[a]);
            if (x >= n_nodes) {
                raise_error(hdr, CSTONE_ERR_INVALID_ARG, 0x72000u);
                continue;
            }
            const int cc = child[x];
            if (cc == 0) continue;
            if (cc < 0 || static_cast<u32>(cc) + 8u > n_nodes) {
                raise_error(hdr, CSTONE_ERR_INVALID_ARG, 0x73000u);
                continue;
            }
            u32 sm = 0;
#pragma unroll
            for (int q = 0; q < 8; ++q) sm += __ldcg(node_counts + cc + q);
            node_counts[x] = sm;
        }
        grid_barrier(bar, hdr);
    }
}

// ---------------------------------------------------------------------------- compensated sums
// A running FP32 sum with Neumaier's compensation term (s, c): s + c tracks the exact sum with an
// error independent of the number of terms. Explicit rounding intrinsics keep the compiler from
// fusing or reassociating the compensation.
struct __align__(8) ff {
    float hi, lo;  // sum and compensation
};

__device__ __forceinline__ ff ff_zero() { return {0.f, 0.f}; }

__device__ __forceinline__ ff ff_add(ff a, float x) {
    const float t = __fadd_rn(a.hi, x);
    const float e = fabsf(a.hi) >= fabsf(x) ? __fadd_rn(__fsub_rn(a.hi, t), x) : __fadd_rn(__fsub_rn(x, t), a.hi);
    return {t, __fadd_rn(a.lo, e)};
}

__device__ __forceinline__ ff ff_add(ff a, ff b) {
    ff r = ff_add(a, b.hi);
    r.lo = __fadd_rn(r.lo, b.lo);
    return r;
}

__device__ __forceinline__ float ff_val(ff a) { return __fadd_rn(a.hi, a.lo); }

struct MpScratch {  // per node: compensated sums and the fixed-point centre carried up the tree
    ff* mass;           // [n]
    ff* quad;           // [6 n], component-major
    ff* res;            // [3 n], component-major: residual first moment about the stored centre
    long long* cfix;    // [3 n], component-major
    Record* rec;        // [n_particles]
    u32* big;           // [n_leaves] leaves handed to the block-per-leaf kernel
    u32* n_big;         // their number
    int* internal;      // [n_internal] internal nodes in breadth-first order of their children
};

__device__ __forceinline__ void store_node(int v, u32 n_nodes, ff M, const long long c[3], const ff q[6],
                                           const ff r[3], MpScratch s, const FixedFrame& f, float* __restrict__ mass,
                                           double* __restrict__ com, float* __restrict__ quad) {
    s.mass[v] = M;
#pragma unroll
    for (int d = 0; d < 3; ++d) s.res[(size_t)d * n_nodes + v] = r[d];
    mass[v] = ff_val(M);
    const bool empty = M.hi == 0.f && M.lo == 0.f;
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        s.cfix[(size_t)d * n_nodes + v] = c[d];
        com[(size_t)d * n_nodes + v] = empty ? 0.0 : fixed_to_double(c[d], f);
    }
#pragma unroll
    for (int k = 0; k < 6; ++k) {
        s.quad[(size_t)k * n_nodes + v] = q[k];
        quad[(size_t)k * n_nodes + v] = ff_val(q[k]);
    }
}

// Coordinates and masses packed into 32-byte fixed-point records, in input order (coalesced).
// A coordinate outside the fixed-point range raises CSTONE_ERR_INVALID_ARG.
__global__ void __launch_bounds__(kThreads) multipole_pack_kernel(const double* __restrict__ x,
                                                                  const double* __restrict__ y,
                                                                  const double* __restrict__ z,
                                                                  const float* __restrict__ m, u32 n,
                                                                  const double* __restrict__ box, Record* rec,
                                                                  WsHeader* hdr) {
    __shared__ FixedFrame s_f;
    if (threadIdx.x == 0) s_f = make_frame(box);
    __syncthreads();
    const FixedFrame f = s_f;
    auto pack = [&](double px, double py, double pz, float pm, u32 p) {
        if (!store_record(rec, p, px, py, pz, pm, f)) raise_error(hdr, CSTONE_ERR_INVALID_ARG, p);
    };
    // one particle per thread and step: 8-byte coalesced loads, and a warp's two 16-byte stores
    // cover 1 KB of records contiguously
    for (u32 p = blockIdx.x * kThreads + threadIdx.x; p < n; p += gridDim.x * kThreads)
        pack(__ldcg(x + p), __ldcg(y + p), __ldcg(z + p), __ldcg(m + p), p);
}

// Leaf moments. A leaf is handled by a group of kGroupLanes lanes (8, or 4 or 2 where leaves are
// small), each lane taking every kGroupLanes-th particle and loading its 32-byte record through
// perm (the one random access of the upsweep), with the group's partial sums combined by
// shuffles: the centre of mass from fixed-point differences to the leaf's first particle, then the
// second moments about it. A lane issues the perm loads of its first kHeld particles together,
// then their record loads together, and keeps those records in registers for the second pass, so
// a leaf of up to kGroupLanes * kHeld particles costs two round trips to memory instead of two per
// particle; records beyond that are read again for the second pass. Narrower groups put more
// leaves, and so more record loads, in flight per warp: with 4.6 particles per leaf (2^27 clumps
// at N_crit 16) two lanes per leaf take the whole multipole upsweep from 10.9 to 6.5 ms.
constexpr int kLeafThreads = 256;
constexpr u32 kBigLeaf = 512;   // larger leaves are summed by a whole block
#ifndef CSTONE_MP_HELD
#define CSTONE_MP_HELD 4
#endif
constexpr int kHeld = CSTONE_MP_HELD;  // records per lane held between the two passes

template <int G>
__device__ __forceinline__ ff group_sum(ff v) {
#pragma unroll
    for (int s = G / 2; s >= 1; s >>= 1) {
        ff o;
        o.hi = __shfl_xor_sync(0xffffffffu, v.hi, s, G);
        o.lo = __shfl_xor_sync(0xffffffffu, v.lo, s, G);
        v = ff_add(v, o);
    }
    return v;
}

__device__ __forceinline__ Record load_record(const Record* rec, u32 p) {
    const longlong2* src = reinterpret_cast<const longlong2*>(rec + p);
    const longlong2 a = __ldg(src), b = __ldg(src + 1);
    Record r;
    r.x = a.x;
    r.y = a.y;
    r.z = b.x;
    r.m = __uint_as_float(static_cast<u32>(b.y));
    r.pad = 0u;
    return r;
}

template <int kGroupLanes>
__global__ void __launch_bounds__(kLeafThreads, 4) multipole_leaf_kernel(const u32* __restrict__ offsets, u32 nl,
                                                                      const u32* __restrict__ perm,
                                                                      const int* __restrict__ leaf_to_node,
                                                                      u32 n_nodes, MpScratch s,
                                                                      const double* __restrict__ box,
                                                                      float* __restrict__ mass,
                                                                      double* __restrict__ com,
                                                                      float* __restrict__ quad) {
    __shared__ FixedFrame s_f;
    if (threadIdx.x == 0) s_f = make_frame(box);
    __syncthreads();
    const FixedFrame f = s_f;
    const u32 gl = threadIdx.x % kGroupLanes;
    const u32 i = (blockIdx.x * kLeafThreads + threadIdx.x) / kGroupLanes;
    bool active = i < nl;
    u32 a = active ? offsets[i] : 0u, b = active ? offsets[i + 1] : 0u;
    if (b - a > kBigLeaf) {  // a whole block sums this leaf later (multipole_bigleaf_kernel)
        if (gl == 0) s.big[atomicAdd(s.n_big, 1u)] = i;
        active = false;
        a = b = 0u;
    }
    u32 trips = (b - a + kGroupLanes - 1) / kGroupLanes;
    for (int o = 16; o > 0; o >>= 1) trips = max(trips, __shfl_xor_sync(0xffffffffu, trips, o));
    // the held records: all perm loads first, then all record loads
    u32 p[kHeld];
#pragma unroll
    for (int t = 0; t < kHeld; ++t) {
        const u32 j = a + t * kGroupLanes + gl;
        p[t] = j < b ? __ldg(perm + j) : 0u;
    }
    Record held[kHeld];
#pragma unroll
    for (int t = 0; t < kHeld; ++t) {
        const u32 j = a + t * kGroupLanes + gl;
        if (j < b) held[t] = load_record(s.rec, p[t]);
        else held[t] = Record{};
    }
    Record r0;  // the leaf's first particle (lane 0 of the group holds it)
    r0.x = __shfl_sync(0xffffffffu, held[0].x, 0, kGroupLanes);
    r0.y = __shfl_sync(0xffffffffu, held[0].y, 0, kGroupLanes);
    r0.z = __shfl_sync(0xffffffffu, held[0].z, 0, kGroupLanes);
    r0.m = __shfl_sync(0xffffffffu, held[0].m, 0, kGroupLanes);
    r0.pad = 0u;
    ff M = ff_zero(), S[3] = {ff_zero(), ff_zero(), ff_zero()}, Q[6];
#pragma unroll
    for (int k = 0; k < 6; ++k) Q[k] = ff_zero();
    auto acc = [](ff& sum, float v) { sum = ff_add(sum, v); };
    auto first_moments = [&](const Record& r) {
        acc(M, r.m);
        acc(S[0], __fmul_rn(r.m, fixed_diff(r.x, r0.x, f)));
        acc(S[1], __fmul_rn(r.m, fixed_diff(r.y, r0.y, f)));
        acc(S[2], __fmul_rn(r.m, fixed_diff(r.z, r0.z, f)));
    };
#pragma unroll
    for (int t = 0; t < kHeld; ++t)
        if (a + t * kGroupLanes + gl < b) first_moments(held[t]);
    for (u32 t = kHeld; t < trips; ++t) {
        const u32 j = a + t * kGroupLanes + gl;
        if (j < b) first_moments(load_record(s.rec, __ldg(perm + j)));
    }
    M = group_sum<kGroupLanes>(M);
#pragma unroll
    for (int d = 0; d < 3; ++d) S[d] = group_sum<kGroupLanes>(S[d]);
    long long c[3] = {0, 0, 0};
    if (b > a) {  // centre = anchor + S / M, rounded to the fixed-point grid
        const float Mv = ff_val(M);
        const long long r0c[3] = {r0.x, r0.y, r0.z};
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            const float off = __fdiv_rn(ff_val(S[d]), Mv);
            c[d] = r0c[d] + float_to_int64(__fmul_rn(__fmul_rn(off, 1.0f / f.s1), 1.0f / f.s2));
        }
    }
    ff R[3] = {ff_zero(), ff_zero(), ff_zero()};  // residual first moment about c
    auto second_moments = [&](const Record& r) {
        const float e0 = fixed_diff(r.x, c[0], f);
        const float e1 = fixed_diff(r.y, c[1], f);
        const float e2 = fixed_diff(r.z, c[2], f);
        const float me0 = __fmul_rn(r.m, e0), me1 = __fmul_rn(r.m, e1), me2 = __fmul_rn(r.m, e2);
        acc(R[0], me0);
        acc(R[1], me1);
        acc(R[2], me2);
        acc(Q[0], __fmul_rn(me0, e0));
        acc(Q[1], __fmul_rn(me0, e1));
        acc(Q[2], __fmul_rn(me0, e2));
        acc(Q[3], __fmul_rn(me1, e1));
        acc(Q[4], __fmul_rn(me1, e2));
        acc(Q[5], __fmul_rn(me2, e2));
    };
#pragma unroll
    for (int t = 0; t < kHeld; ++t)
        if (a + t * kGroupLanes + gl < b) second_moments(held[t]);
    for (u32 t = kHeld; t < trips; ++t) {
        const u32 j = a + t * kGroupLanes + gl;
        if (j < b) second_moments(load_record(s.rec, __ldg(perm + j)));
    }
#pragma unroll
    for (int k = 0; k < 6; ++k) Q[k] = group_sum<kGroupLanes>(Q[k]);
#pragma unroll
    for (int d = 0; d < 3; ++d) R[d] = group_sum<kGroupLanes>(R[d]);
    if (active && gl == 0) store_node(leaf_to_node[i], n_nodes, M, c, Q, R, s, f, mass, com, quad);
}

// Sum of a compensated pair over the block (every thread gets the total); red holds kThreads / 32
// pairs of scratch.
__device__ __forceinline__ ff block_sum(ff v, ff* red) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        ff w;
        w.hi = __shfl_xor_sync(0xffffffffu, v.hi, o);
        w.lo = __shfl_xor_sync(0xffffffffu, v.lo, o);
        v = ff_add(v, w);
    }
    __syncthreads();  // red may still be read by the previous call
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    ff t = red[0];
#pragma unroll
    for (int w = 1; w < kLeafThreads / 32; ++w) t = ff_add(t, red[w]);
    return t;
}

// Leaves of more than kBigLeaf particles (full-depth cells of dense data, which are never split),
// one block per leaf: the same two passes (first moments about the first particle, then second
// moments about the centre), each thread taking every kLeafThreads-th particle.
__global__ void __launch_bounds__(kLeafThreads) multipole_bigleaf_kernel(const u32* __restrict__ offsets,
                                                                         const u32* __restrict__ perm,
                                                                         const int* __restrict__ leaf_to_node,
                                                                         u32 n_nodes, MpScratch s,
                                                                         const double* __restrict__ box,
                                                                         float* __restrict__ mass,
                                                                         double* __restrict__ com,
                                                                         float* __restrict__ quad) {
    __shared__ FixedFrame s_f;
    __shared__ ff s_red[kLeafThreads / 32];
    if (threadIdx.x == 0) s_f = make_frame(box);
    __syncthreads();
    const FixedFrame f = s_f;
    const u32 nbig = *s.n_big;
    for (u32 q = blockIdx.x; q < nbig; q += gridDim.x) {
        const u32 i = s.big[q];
        const u32 a = offsets[i], b = offsets[i + 1];
        const Record r0 = s.rec[__ldg(perm + a)];
        ff M = ff_zero(), S[3] = {ff_zero(), ff_zero(), ff_zero()}, Q[6];
#pragma unroll
        for (int k = 0; k < 6; ++k) Q[k] = ff_zero();
        for (u32 j = a + threadIdx.x; j < b; j += kLeafThreads) {
            const Record r = s.rec[__ldg(perm + j)];
            M = ff_add(M, r.m);
            S[0] = ff_add(S[0], __fmul_rn(r.m, fixed_diff(r.x, r0.x, f)));
            S[1] = ff_add(S[1], __fmul_rn(r.m, fixed_diff(r.y, r0.y, f)));
            S[2] = ff_add(S[2], __fmul_rn(r.m, fixed_diff(r.z, r0.z, f)));
        }
        M = block_sum(M, s_red);
#pragma unroll
        for (int d = 0; d < 3; ++d) S[d] = block_sum(S[d], s_red);
        long long c[3];
        const float Mv = ff_val(M);
        const long long r0c[3] = {r0.x, r0.y, r0.z};
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            const float off = Mv != 0.f ? __fdiv_rn(ff_val(S[d]), Mv) : 0.f;
            c[d] = r0c[d] + float_to_int64(__fmul_rn(__fmul_rn(off, 1.0f / f.s1), 1.0f / f.s2));
        }
        ff R[3] = {ff_zero(), ff_zero(), ff_zero()};  // residual first moment about c
        for (u32 j = a + threadIdx.x; j < b; j += kLeafThreads) {
            const Record r = s.rec[__ldg(perm + j)];
            const float e0 = fixed_diff(r.x, c[0], f);
            const float e1 = fixed_diff(r.y, c[1], f);
            const float e2 = fixed_diff(r.z, c[2], f);
            const float me0 = __fmul_rn(r.m, e0), me1 = __fmul_rn(r.m, e1), me2 = __fmul_rn(r.m, e2);
            R[0] = ff_add(R[0], me0);
            R[1] = ff_add(R[1], me1);
            R[2] = ff_add(R[2], me2);
            Q[0] = ff_add(Q[0], __fmul_rn(me0, e0));
            Q[1] = ff_add(Q[1], __fmul_rn(me0, e1));
            Q[2] = ff_add(Q[2], __fmul_rn(me0, e2));
            Q[3] = ff_add(Q[3], __fmul_rn(me1, e1));
            Q[4] = ff_add(Q[4], __fmul_rn(me1, e2));
            Q[5] = ff_add(Q[5], __fmul_rn(me2, e2));
        }
#pragma unroll
        for (int k = 0; k < 6; ++k) Q[k] = block_sum(Q[k], s_red);
#pragma unroll
        for (int d = 0; d < 3; ++d) R[d] = block_sum(R[d], s_red);
        if (threadIdx.x == 0) store_node(leaf_to_node[i], n_nodes, M, c, Q, R, s, f, mass, com, quad);
        __syncthreads();
    }
}

// Internal nodes, level by level from the deepest: every internal node of a level combines its 8
// children (in child order) with the parallel-axis shift; a grid barrier separates the levels.
__global__ void __launch_bounds__(kThreads, 4) multipole_level_kernel(const int* __restrict__ child,
                                                                   const int* __restrict__ level_offsets, u32 n_nodes,
                                                                   MpScratch s, const double* __restrict__ box,
                                                                   float* __restrict__ mass, double* __restrict__ com,
                                                                   float* __restrict__ quad, GridBarrier* bar,
                                                                   WsHeader* hdr) {
    __shared__ int s_lo[kNumLevels + 1];
    __shared__ FixedFrame s_f;
    if (threadIdx.x <= kNumLevels) s_lo[threadIdx.x] = level_offsets[threadIdx.x];
    if (threadIdx.x == 0) s_f = make_frame(box);
    __syncthreads();
    const FixedFrame f = s_f;
    const u32 gtid = blockIdx.x * kThreads + threadIdx.x, gthreads = gridDim.x * kThreads;
    const u32 n_int = (n_nodes - 1) / 8;
    list_internal(child, n_nodes, n_int, s.internal, gtid, gthreads, hdr);
    grid_barrier(bar, hdr);
    // One internal node per group of 8 lanes, lane k taking child k: the node's sums are shuffle
    // reductions over the group (compensated adds, pairwise order).
    auto group_ff = [](ff v) {
#pragma unroll
        for (int s_ = 4; s_ >= 1; s_ >>= 1) {
            ff o;
            o.hi = __shfl_xor_sync(0xffffffffu, v.hi, s_, 8);
            o.lo = __shfl_xor_sync(0xffffffffu, v.lo, s_, 8);
            v = ff_add(v, o);
        }
        return v;
    };
    auto combine8 = [&](u32 g, bool active) {  // every lane of the warp calls it (shuffles)
        const int lane8 = threadIdx.x & 7;
        const int gbase = (threadIdx.x & 31) & ~7;
        const int c0 = static_cast<int>(8u * (active ? g : 0u) + 1u);
        const int ck = c0 + lane8;
        ff Mk = ff_zero();
        long long cc[3] = {0, 0, 0};
        ff rk[3] = {ff_zero(), ff_zero(), ff_zero()}, qk[6];
#pragma unroll
        for (int q = 0; q < 6; ++q) qk[q] = ff_zero();
        if (active) {
            const float2 mm = __ldcg(reinterpret_cast<const float2*>(s.mass) + ck);
            Mk = {mm.x, mm.y};
#pragma unroll
            for (int d = 0; d < 3; ++d) {
                cc[d] = __ldcg(s.cfix + (size_t)d * n_nodes + ck);
                const float2 rr = __ldcg(reinterpret_cast<const float2*>(s.res + (size_t)d * n_nodes) + ck);
                rk[d] = ff{rr.x, rr.y};
            }
#pragma unroll
            for (int q = 0; q < 6; ++q) {
                const float2 qq = __ldcg(reinterpret_cast<const float2*>(s.quad + (size_t)q * n_nodes) + ck);
                qk[q] = ff{qq.x, qq.y};
            }
        }
        const u32 nz = (__ballot_sync(0xffffffffu, active && (Mk.hi != 0.f || Mk.lo != 0.f)) >> gbase) & 0xffu;
        const int anchor = nz ? __ffs(nz) - 1 : 0;
        long long ca[3], cp[3] = {0, 0, 0};
#pragma unroll
        for (int d = 0; d < 3; ++d) ca[d] = __shfl_sync(0xffffffffu, cc[d], anchor, 8);
        ff Mp = group_ff(Mk), Qp[6], Rp[3];
        const float mk = ff_val(Mk);
        ff Sp[3];
#pragma unroll
        for (int d = 0; d < 3; ++d) Sp[d] = group_ff(ff{nz ? __fmul_rn(mk, fixed_diff(cc[d], ca[d], f)) : 0.f, 0.f});
        if (nz) {
            const float Mv = ff_val(Mp);
#pragma unroll
            for (int d = 0; d < 3; ++d) {
                const float off = __fdiv_rn(ff_val(Sp[d]), Mv);
                cp[d] = ca[d] + float_to_int64(__fmul_rn(__fmul_rn(off, 1.0f / f.s1), 1.0f / f.s2));
            }
        }
        float e[3];
#pragma unroll
        for (int d = 0; d < 3; ++d) e[d] = nz ? fixed_diff(cc[d], cp[d], f) : 0.f;
        const float me0 = __fmul_rn(mk, e[0]), me1 = __fmul_rn(mk, e[1]), me2 = __fmul_rn(mk, e[2]);
        const float shift[6] = {__fmul_rn(me0, e[0]), __fmul_rn(me0, e[1]), __fmul_rn(me0, e[2]),
                                __fmul_rn(me1, e[1]), __fmul_rn(me1, e[2]), __fmul_rn(me2, e[2])};
        float rv[3];
#pragma unroll
        for (int d = 0; d < 3; ++d) rv[d] = ff_val(rk[d]);
        const float cross[6] = {
            __fmul_rn(2.0f, __fmul_rn(rv[0], e[0])), __fadd_rn(__fmul_rn(rv[0], e[1]), __fmul_rn(rv[1], e[0])),
            __fadd_rn(__fmul_rn(rv[0], e[2]), __fmul_rn(rv[2], e[0])), __fmul_rn(2.0f, __fmul_rn(rv[1], e[1])),
            __fadd_rn(__fmul_rn(rv[1], e[2]), __fmul_rn(rv[2], e[1])), __fmul_rn(2.0f, __fmul_rn(rv[2], e[2]))};
#pragma unroll
        for (int q = 0; q < 6; ++q) {
            ff t = ff_add(qk[q], shift[q]);
            t = ff_add(t, cross[q]);
            Qp[q] = group_ff(nz ? t : ff_zero());
        }
        const float me[3] = {me0, me1, me2};
#pragma unroll
        for (int d = 0; d < 3; ++d) Rp[d] = group_ff(nz ? ff_add(rk[d], me[d]) : ff_zero());
        if (!active || lane8 != 0) return;
        const int x = s.internal[g];
        if (x < 0 || static_cast<u32>(x) >= n_nodes || child[x] != c0) {
            raise_error(hdr, CSTONE_ERR_INVALID_ARG, 0x75000u);
            return;
        }
        store_node(x, n_nodes, Mp, cp, Qp, Rp, s, f, mass, com, quad);
    };
    // small levels by block 0 alone, as in the count upsweep; 8 lanes per node, the loop bounds
    // the same in every lane of a warp
    constexpr u32 kGroups = kThreads / 8;
    const u32 gw = (blockIdx.x * kThreads + threadIdx.x) / 32, nw = gridDim.x * (kThreads / 32);
    bool pending = false;
    for (int l = kLevels - 1; l >= 0; --l) {
        if (s_lo[l + 2] == s_lo[l + 1]) continue;  // no internal node at level l
        u32 g0, g1;
        internal_range(s_lo, l, n_int, g0, g1);
        if (g1 <= g0 + kSmallLevel) {
            if (blockIdx.x == 0) {
                for (u32 b0 = g0; b0 < g1; b0 += kGroups) {  // uniform trip count in the block
                    const u32 g = b0 + threadIdx.x / 8;
                    combine8(g, g < g1);
                }
                __syncthreads();
            }
            pending = true;
            continue;
        }
        if (pending) grid_barrier(bar, hdr);
        for (u32 b0 = g0 + 4 * gw; b0 < g1; b0 += 4 * nw) {  // a warp takes 4 nodes, b0 the same in its lanes
            const u32 g = b0 + (threadIdx.x & 31) / 8;
            combine8(g, g < g1);
        }
        grid_barrier(bar, hdr);
        pending = false;
    }
}

struct UpLayout {
    GridBarrier* bar;
    int* internal;  // [n_internal]
    MpScratch mp;
    size_t bytes;
};

UpLayout up_layout(void* ws, long long nl, long long n_particles, bool multipoles) {
    UpLayout l;
    Carver c(ws);
    const long long nn = nl + (nl - 1) / 7;
    l.bar = c.take<GridBarrier>(1);
    l.internal = c.take<int>((size_t)((nl - 1) / 7));
    l.mp = MpScratch{};
    l.mp.internal = l.internal;
    if (multipoles) {
        l.mp.mass = c.take<ff>((size_t)nn);
        l.mp.quad = c.take<ff>((size_t)nn * 6);
        l.mp.res = c.take<ff>((size_t)nn * 3);
        l.mp.cfix = c.take<long long>((size_t)nn * 3);
        l.mp.rec = c.take<Record>((size_t)(n_particles > 0 ? n_particles : 1));
        l.mp.big = c.take<u32>((size_t)nl);
        l.mp.n_big = c.take<u32>(1);
    }
    l.bytes = c.size();
    return l;
}

}  // namespace

size_t upsweep_ws_bytes(long long nl) { return up_layout(nullptr, nl, 0, false).bytes; }
size_t multipole_ws_bytes(long long nl, long long n) { return up_layout(nullptr, nl, n, true).bytes; }

int launch_upsweep_counts(const u32* leaf_counts, long long nl, const int* leaf_to_node, const int* child,
                          const int* level_offsets, u32* node_counts, void* ws, cudaStream_t st) {
    UpLayout l = up_layout(ws, nl, 0, false);
    WsHeader* hdr = reinterpret_cast<WsHeader*>(ws);
    CST_CUDA(cudaMemsetAsync(hdr, 0, sizeof(WsHeader), st));
    CST_CUDA(cudaMemsetAsync(l.bar, 0, sizeof(GridBarrier), st));
    u32 nl_ = static_cast<u32>(nl);
    GridBarrier* bar = l.bar;
    int* internal = l.internal;
    void* args[] = {&leaf_counts, &nl_, &leaf_to_node, &child, &level_offsets, &node_counts, &internal, &bar, &hdr};
    const int grid = cooperative_grid(reinterpret_cast<const void*>(upsweep_counts_kernel), kThreads, 0, 4);
    CST_COOP(cudaLaunchCooperativeKernel(reinterpret_cast<void*>(upsweep_counts_kernel), dim3(grid), dim3(kThreads),
                                         args, 0, st));
    return CSTONE_OK;
}

int launch_upsweep_counts_batched(const u32* elem_counts, long long n_elements, const int* leaf_to_node,
                                  const int* child, const int* level_offsets, int n_sets, u32* node_counts, void* ws,
                                  cudaStream_t st) {
    UpLayout l = up_layout(ws, 1, 0, false);
    WsHeader* hdr = reinterpret_cast<WsHeader*>(ws);
    CST_CUDA(cudaMemsetAsync(hdr, 0, sizeof(WsHeader), st));
    CST_CUDA(cudaMemsetAsync(l.bar, 0, sizeof(GridBarrier), st));
    u32 ne = static_cast<u32>(n_elements);
    GridBarrier* bar = l.bar;
    void* args[] = {&elem_counts, &ne, &leaf_to_node, &child, &level_offsets, &n_sets, &node_counts, &bar, &hdr};
    const int grid = cooperative_grid(reinterpret_cast<const void*>(upsweep_counts_batched_kernel), kThreads, 0, 4);
    CST_COOP(cudaLaunchCooperativeKernel(reinterpret_cast<void*>(upsweep_counts_batched_kernel), dim3(grid),
                                         dim3(kThreads), args, 0, st));
    return CSTONE_OK;
}

// records == NULL: pack them from x, y, z, m into the workspace first; otherwise they were written
// by the record-writing key kernel (and the workspace has no record area).
int launch_upsweep_multipoles(const double* x, const double* y, const double* z, const float* m, const u32* perm,
                              long long n, const u32* offsets, long long nl, const int* leaf_to_node, const int* child,
                              const int* level_offsets, const double* box, float* mass, double* com, float* quad,
                              void* ws, cudaStream_t st, const Record* records = nullptr) {
    UpLayout l = up_layout(ws, nl, records ? 0 : n, true);
    if (records) l.mp.rec = const_cast<Record*>(records);
    WsHeader* hdr = reinterpret_cast<WsHeader*>(ws);
    CST_CUDA(cudaMemsetAsync(hdr, 0, sizeof(WsHeader), st));
    CST_CUDA(cudaMemsetAsync(l.bar, 0, sizeof(GridBarrier), st));
    const u32 nn = static_cast<u32>(nl + (nl - 1) / 7);
    if (n > 0 && !records) {
        long long want = (n + kThreads - 1) / kThreads;
        int pgrid = static_cast<int>(want < (long long)sm_count() * 8 ? want : (long long)sm_count() * 8);
        multipole_pack_kernel<<<pgrid, kThreads, 0, st>>>(x, y, z, m, static_cast<u32>(n), box, l.mp.rec, hdr);
        CST_LAUNCHED("multipole_pack_kernel");
    }
    CST_CUDA(cudaMemsetAsync(l.mp.n_big, 0, sizeof(u32), st));
    // lanes per leaf from the mean leaf size (measured: 2 at 4.6 particles per leaf, 8 at 17.5)
    const int G = n < 8 * nl ? 2 : (n < 12 * nl ? 4 : 8);
    const long long groups_per_block = kLeafThreads / G;
    const unsigned lgrid = static_cast<unsigned>((nl + groups_per_block - 1) / groups_per_block);
    if (G == 2)
        multipole_leaf_kernel<2><<<lgrid, kLeafThreads, 0, st>>>(offsets, static_cast<u32>(nl), perm, leaf_to_node, nn,
                                                                 l.mp, box, mass, com, quad);
    else if (G == 4)
        multipole_leaf_kernel<4><<<lgrid, kLeafThreads, 0, st>>>(offsets, static_cast<u32>(nl), perm, leaf_to_node, nn,
                                                                 l.mp, box, mass, com, quad);
    else
        multipole_leaf_kernel<8><<<lgrid, kLeafThreads, 0, st>>>(offsets, static_cast<u32>(nl), perm, leaf_to_node, nn,
                                                                 l.mp, box, mass, com, quad);
    CST_LAUNCHED("multipole_leaf_kernel");
    multipole_bigleaf_kernel<<<sm_count() * 4, kLeafThreads, 0, st>>>(offsets, perm, leaf_to_node, nn, l.mp, box, mass,
                                                                     com, quad);
    CST_LAUNCHED("multipole_bigleaf_kernel");
    if (nl > 1) {
        u32 nn_ = nn;
        MpScratch mp = l.mp;
        GridBarrier* bar = l.bar;
        void* args[] = {&child, &level_offsets, &nn_, &mp, &box, &mass, &com, &quad, &bar, &hdr};
        const int grid = cooperative_grid(reinterpret_cast<const void*>(multipole_level_kernel), kThreads, 0, 4);
        CST_COOP(cudaLaunchCooperativeKernel(reinterpret_cast<void*>(multipole_level_kernel), dim3(grid),
                                             dim3(kThreads), args, 0, st));
    }
    return CSTONE_OK;
}

}  // namespace CST_NS

extern "C" {

int CSTONE_FN(upsweep_workspace_size)(int64_t n_leaves, size_t* bytes) {
    if (!bytes || n_leaves < 1 || n_leaves > CSTONE_MAX_LEAVES)
        return cst::fail(CSTONE_ERR_INVALID_ARG, CST_STR(CSTONE_FN(upsweep_workspace_size)) ": bad argument");
    *bytes = CST_NS::upsweep_ws_bytes(n_leaves);
    return CSTONE_OK;
}

int CSTONE_FN(upsweep_counts)(const uint32_t* leaf_counts, int64_t n_leaves, const int32_t* leaf_to_node,
                          const int32_t* child, const int32_t* level_offsets, uint32_t* node_counts, void* ws,
                          size_t ws_bytes, void* stream) {
    if (n_leaves < 1 || n_leaves > CSTONE_MAX_LEAVES || (n_leaves - 1) % 7 != 0 || !leaf_counts || !leaf_to_node ||
        !child || !level_offsets || !node_counts)
        return cst::fail(CSTONE_ERR_INVALID_ARG, CST_STR(CSTONE_FN(upsweep_counts)) ": bad argument");
    if (int rc = cst::check_ws(ws, ws_bytes, CST_NS::upsweep_ws_bytes(n_leaves), CST_STR(CSTONE_FN(upsweep_counts))))
        return rc;
    return CST_NS::launch_upsweep_counts(leaf_counts, n_leaves, leaf_to_node, child, level_offsets, node_counts, ws,
                                      cst::as_stream(stream));
}

int CSTONE_FN(multipole_workspace_size)(int64_t n, int64_t n_leaves, size_t* bytes) {
    if (!bytes || n < 0 || n >= CSTONE_MAX_PARTICLES || n_leaves < 1 || n_leaves > CSTONE_MAX_LEAVES)
        return cst::fail(CSTONE_ERR_INVALID_ARG, CST_STR(CSTONE_FN(multipole_workspace_size)) ": bad argument");
    *bytes = CST_NS::multipole_ws_bytes(n_leaves, n);
    return CSTONE_OK;
}

int CSTONE_FN(upsweep_multipoles_records)(const void* records, const uint32_t* perm, int64_t n,
                                          const uint32_t* offsets, int64_t n_leaves, const int32_t* leaf_to_node,
                                          const int32_t* child, const int32_t* level_offsets, const double* box,
                                          float* mass, double* com, float* quad, void* ws, size_t ws_bytes,
                                          void* stream) {
    if (n < 0 || n >= CSTONE_MAX_PARTICLES || n_leaves < 1 || n_leaves > CSTONE_MAX_LEAVES ||
        (n_leaves - 1) % 7 != 0 || !offsets || !leaf_to_node || !child || !level_offsets || !mass || !com || !quad ||
        !box || (n > 0 && (!records || !perm)) || (reinterpret_cast<uintptr_t>(records) & 15u) != 0)
        return cst::fail(CSTONE_ERR_INVALID_ARG, CST_STR(CSTONE_FN(upsweep_multipoles_records)) ": bad argument");
    if (int rc = cst::check_ws(ws, ws_bytes, CST_NS::multipole_ws_bytes(n_leaves, 0),
                               CST_STR(CSTONE_FN(upsweep_multipoles_records))))
        return rc;
    return CST_NS::launch_upsweep_multipoles(nullptr, nullptr, nullptr, nullptr, perm, n, offsets, n_leaves,
                                             leaf_to_node, child, level_offsets, box, mass, com, quad, ws,
                                             cst::as_stream(stream), static_cast<const cst::Record*>(records));
}

int CSTONE_FN(upsweep_multipoles)(const double* x, const double* y, const double* z, const float* m,
                              const uint32_t* perm, int64_t n, const uint32_t* offsets, int64_t n_leaves,
                              const int32_t* leaf_to_node, const int32_t* child, const int32_t* level_offsets,
                              const double* box, float* mass, double* com, float* quad, void* ws, size_t ws_bytes,
                              void* stream) {
    if (n < 0 || n >= CSTONE_MAX_PARTICLES || n_leaves < 1 || n_leaves > CSTONE_MAX_LEAVES ||
        (n_leaves - 1) % 7 != 0 || !offsets || !leaf_to_node || !child || !level_offsets || !mass || !com || !quad ||
        !box || (n > 0 && (!x || !y || !z || !m || !perm)))
        return cst::fail(CSTONE_ERR_INVALID_ARG, CST_STR(CSTONE_FN(upsweep_multipoles)) ": bad argument");
    if (int rc = cst::check_ws(ws, ws_bytes, CST_NS::multipole_ws_bytes(n_leaves, n),
                               CST_STR(CSTONE_FN(upsweep_multipoles))))
        return rc;
    return CST_NS::launch_upsweep_multipoles(x, y, z, m, perm, n, offsets, n_leaves, leaf_to_node, child, level_offsets,
                                          box, mass, com, quad, ws, cst::as_stream(stream));
}

#ifndef CSTONE_KEY32  // batched builds exist for 63-bit keys only
int cstone_upsweep_counts_batched(const uint32_t* elem_counts, int64_t n_elements, const int32_t* leaf_to_node,
                                  const int32_t* child, const int32_t* level_offsets, int32_t n_sets,
                                  uint32_t* node_counts, void* ws, size_t ws_bytes, void* stream) {
    if (n_sets < 1 || n_sets > cst::kMaxBatchSets || n_elements < 2 * (int64_t)n_sets ||
        n_elements > CSTONE_MAX_LEAVES || !elem_counts || !leaf_to_node || !child || !level_offsets || !node_counts)
        return cst::fail(CSTONE_ERR_INVALID_ARG, "cstone_upsweep_counts_batched: bad argument (at most %d sets)",
                         cst::kMaxBatchSets);
    if (int rc = cst::check_ws(ws, ws_bytes, cst::upsweep_ws_bytes(1), "cstone_upsweep_counts_batched")) return rc;
    return cst::launch_upsweep_counts_batched(elem_counts, n_elements, leaf_to_node, child, level_offsets, n_sets,
                                              node_counts, ws, cst::as_stream(stream));
}

#endif

}  // extern "C"
