// Upsweeps over the linked octree (Sec. 5 node properties; Sec. 7 computes node properties "by an
// upward pass" where leaves depend on their particles and internal nodes on their children).
//
// Both upsweeps are single launches: one thread per leaf writes the leaf's value and climbs. At
// every sibling group it increments the group's arrival counter; the eighth arrival computes the
// parent from its 8 children (always in child order, so results do not depend on timing) and
// continues upwards, the others stop. Breadth-first layout puts the 8 children of a node in one
// aligned group, group g = nodes 1 + 8g .. 8 + 8g, whose parent is parent[g].
//
// Multipoles (three launches: gather into sorted order, leaf sums, climb): FP32 accumulation with
// compensation. Each sum is a pair (sum, compensation) updated with an exact two-sum step
// (Neumaier), and the pairs of mass and second moments are carried up the tree in scratch so the
// compensation survives all 21 levels. Coordinate differences are rounded to FP32 once from their
// exact value; the expansion centre (centre of mass) is kept in FP64.
// A leaf takes its first particle as the anchor for the differences, an internal node its first
// non-empty child's centre; second moments of an internal node use the parallel-axis shift
// Q = sum_c [Q_c + M_c (c_c - c)(c_c - c)^T].
#include "common.cuh"

namespace cst {
namespace {

constexpr int kThreads = 256;

// ---------------------------------------------------------------------------- counts
__global__ void __launch_bounds__(kThreads) upsweep_counts_kernel(const u32* __restrict__ leaf_counts, u32 nl,
                                                                  const int* __restrict__ leaf_to_node,
                                                                  const int* __restrict__ parent,
                                                                  u32* __restrict__ node_counts,
                                                                  u32* __restrict__ arrive) {
    u32 i = blockIdx.x * kThreads + threadIdx.x;
    if (i >= nl) return;
    int v = leaf_to_node[i];
    node_counts[v] = leaf_counts[i];
    while (v != 0) {
        u32 g = static_cast<u32>(v - 1) >> 3;
        __threadfence();
        if (atomicAdd(&arrive[g], 1u) != 7u) return;
        __threadfence();
        const u32* kids = node_counts + 1 + 8 * g;
        u32 s = 0;
#pragma unroll
        for (int c = 0; c < 8; ++c) s += __ldcg(kids + c);
        v = parent[g];
        node_counts[v] = s;
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

// x - a rounded once to FP32. The exact difference is formed from the two 53-bit significands in
// 64-bit integer arithmetic (aligned by the exponent gap, at most 9 bits here) and converted with
// one rounding; the power-of-two scale is exact. Zero, subnormal or far-apart operands and
// magnitudes outside the FP32 range of the scale take the FP64 path.
__device__ __forceinline__ float diff_f32(double x, double a) {
    const u64 bx = static_cast<u64>(__double_as_longlong(x));
    const u64 ba = static_cast<u64>(__double_as_longlong(a));
    const int ex = static_cast<int>((bx >> 52) & 0x7ffu), ea = static_cast<int>((ba >> 52) & 0x7ffu);
    const int emin = min(ex, ea);
    if (ex == 0 || ea == 0 || abs(ex - ea) > 9 || emin < 975 || max(ex, ea) > 1130)
        return __double2float_rn(__dsub_rn(x, a));
    constexpr u64 kMant = (1ULL << 52) - 1;
    long long X = static_cast<long long>(((bx & kMant) | (1ULL << 52)) << (ex - emin));
    long long A = static_cast<long long>(((ba & kMant) | (1ULL << 52)) << (ea - emin));
    if (bx >> 63) X = -X;
    if (ba >> 63) A = -A;
    const float f = __ll2float_rn(X - A);
    return __fmul_rn(f, __int_as_float((emin - 1075 + 127) << 23));
}

struct MpScratch {  // per node: compensated sums carried up the tree
    ff* mass;       // [n]
    ff* quad;       // [6 n], component-major
    double* xs;     // [n_particles] coordinates and masses in sorted order
    double* ys;
    double* zs;
    float* ms;
};

__device__ __forceinline__ void store_node(int v, u32 n_nodes, ff M, const double c[3], const ff q[6], MpScratch s,
                                           float* __restrict__ mass, double* __restrict__ com,
                                           float* __restrict__ quad) {
    s.mass[v] = M;
    mass[v] = ff_val(M);
#pragma unroll
    for (int d = 0; d < 3; ++d) com[(size_t)d * n_nodes + v] = c[d];
#pragma unroll
    for (int k = 0; k < 6; ++k) {
        s.quad[(size_t)k * n_nodes + v] = q[k];
        quad[(size_t)k * n_nodes + v] = ff_val(q[k]);
    }
}

// The one random access of the upsweep: coordinates and masses gathered into sorted order,
// several independent gathers in flight per thread.
constexpr int kGather = 4;

__global__ void __launch_bounds__(kThreads) multipole_gather_kernel(const double* __restrict__ x,
                                                                    const double* __restrict__ y,
                                                                    const double* __restrict__ z,
                                                                    const float* __restrict__ m,
                                                                    const u32* __restrict__ perm, u32 n, MpScratch s) {
    const u32 stride = gridDim.x * kThreads * kGather;
    for (u32 j0 = (blockIdx.x * kThreads) * kGather + threadIdx.x; j0 < n; j0 += stride) {
        u32 p[kGather];
#pragma unroll
        for (int q = 0; q < kGather; ++q) {
            const u32 j = j0 + q * kThreads;
            p[q] = j < n ? __ldcs(perm + j) : 0u;
        }
        double px[kGather], py[kGather], pz[kGather];
        float pm[kGather];
#pragma unroll
        for (int q = 0; q < kGather; ++q) {
            px[q] = __ldg(x + p[q]);
            py[q] = __ldg(y + p[q]);
            pz[q] = __ldg(z + p[q]);
            pm[q] = __ldg(m + p[q]);
        }
#pragma unroll
        for (int q = 0; q < kGather; ++q) {
            const u32 j = j0 + q * kThreads;
            if (j < n) {
                s.xs[j] = px[q];
                s.ys[j] = py[q];
                s.zs[j] = pz[q];
                s.ms[j] = pm[q];
            }
        }
    }
}

// Leaf moments, one thread per leaf over its contiguous run of gathered particles: the centre of
// mass from differences to the first particle, then the second moments about it.
__global__ void __launch_bounds__(kThreads) multipole_leaf_kernel(const u32* __restrict__ offsets, u32 nl,
                                                                  const int* __restrict__ leaf_to_node, u32 n_nodes,
                                                                  MpScratch s, float* __restrict__ mass,
                                                                  double* __restrict__ com,
                                                                  float* __restrict__ quad) {
    const u32 i = blockIdx.x * kThreads + threadIdx.x;
    if (i >= nl) return;
    const int v = leaf_to_node[i];
    const u32 a = offsets[i], b = offsets[i + 1];
    ff M = ff_zero(), S[3] = {ff_zero(), ff_zero(), ff_zero()}, Q[6];
#pragma unroll
    for (int k = 0; k < 6; ++k) Q[k] = ff_zero();
    double c[3] = {0.0, 0.0, 0.0};
    if (b > a) {
        const double ax = s.xs[a], ay = s.ys[a], az = s.zs[a];
        for (u32 j = a; j < b; ++j) {
            const float mj = s.ms[j];
            M = ff_add(M, mj);
            S[0] = ff_add(S[0], __fmul_rn(mj, diff_f32(s.xs[j], ax)));
            S[1] = ff_add(S[1], __fmul_rn(mj, diff_f32(s.ys[j], ay)));
            S[2] = ff_add(S[2], __fmul_rn(mj, diff_f32(s.zs[j], az)));
        }
        const float Mv = ff_val(M);
        c[0] = __dadd_rn(ax, (double)__fdiv_rn(ff_val(S[0]), Mv));
        c[1] = __dadd_rn(ay, (double)__fdiv_rn(ff_val(S[1]), Mv));
        c[2] = __dadd_rn(az, (double)__fdiv_rn(ff_val(S[2]), Mv));
        for (u32 j = a; j < b; ++j) {
            const float mj = s.ms[j];
            const float e0 = diff_f32(s.xs[j], c[0]);
            const float e1 = diff_f32(s.ys[j], c[1]);
            const float e2 = diff_f32(s.zs[j], c[2]);
            const float me0 = __fmul_rn(mj, e0), me1 = __fmul_rn(mj, e1), me2 = __fmul_rn(mj, e2);
            Q[0] = ff_add(Q[0], __fmul_rn(me0, e0));
            Q[1] = ff_add(Q[1], __fmul_rn(me0, e1));
            Q[2] = ff_add(Q[2], __fmul_rn(me0, e2));
            Q[3] = ff_add(Q[3], __fmul_rn(me1, e1));
            Q[4] = ff_add(Q[4], __fmul_rn(me1, e2));
            Q[5] = ff_add(Q[5], __fmul_rn(me2, e2));
        }
    }
    store_node(v, n_nodes, M, c, Q, s, mass, com, quad);
}

// Internal nodes: one thread per leaf climbs; the eighth arrival at a sibling group combines the
// 8 children (in child order) into the parent with the parallel-axis shift.
__global__ void __launch_bounds__(kThreads) multipole_climb_kernel(u32 nl, const int* __restrict__ leaf_to_node,
                                                                   const int* __restrict__ parent, u32 n_nodes,
                                                                   MpScratch s, float* __restrict__ mass,
                                                                   double* __restrict__ com, float* __restrict__ quad,
                                                                   u32* __restrict__ arrive) {
    const u32 i = blockIdx.x * kThreads + threadIdx.x;
    if (i >= nl) return;
    int v = leaf_to_node[i];
    while (v != 0) {
        const u32 g = static_cast<u32>(v - 1) >> 3;
        __threadfence();
        if (atomicAdd(&arrive[g], 1u) != 7u) return;
        __threadfence();
        const int c0 = 1 + 8 * static_cast<int>(g);
        ff Mc[8];
        int anchor = -1;
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            const float2 mm = __ldcg(reinterpret_cast<const float2*>(s.mass) + c0 + k);
            Mc[k] = {mm.x, mm.y};
            if (anchor < 0 && (mm.x != 0.f || mm.y != 0.f)) anchor = k;
        }
        ff Mp = ff_zero(), Sp[3] = {ff_zero(), ff_zero(), ff_zero()}, Qp[6];
#pragma unroll
        for (int k = 0; k < 6; ++k) Qp[k] = ff_zero();
        double cp[3] = {0.0, 0.0, 0.0};
        if (anchor >= 0) {
            double cc[8][3];
#pragma unroll
            for (int k = 0; k < 8; ++k)
#pragma unroll
                for (int d = 0; d < 3; ++d) cc[k][d] = __ldcg(com + (size_t)d * n_nodes + c0 + k);
            double ca[3];
#pragma unroll
            for (int d = 0; d < 3; ++d) {
                ca[d] = cc[0][d];
#pragma unroll
                for (int k = 1; k < 8; ++k)
                    if (k == anchor) ca[d] = cc[k][d];
            }
#pragma unroll
            for (int k = 0; k < 8; ++k) {
                Mp = ff_add(Mp, Mc[k]);
                const float mk = ff_val(Mc[k]);
#pragma unroll
                for (int d = 0; d < 3; ++d) Sp[d] = ff_add(Sp[d], __fmul_rn(mk, diff_f32(cc[k][d], ca[d])));
            }
            const float Mv = ff_val(Mp);
#pragma unroll
            for (int d = 0; d < 3; ++d) cp[d] = __dadd_rn(ca[d], (double)__fdiv_rn(ff_val(Sp[d]), Mv));
#pragma unroll
            for (int k = 0; k < 8; ++k) {
                float e[3];
#pragma unroll
                for (int d = 0; d < 3; ++d) e[d] = diff_f32(cc[k][d], cp[d]);
                const float mk = ff_val(Mc[k]);
                const float me0 = __fmul_rn(mk, e[0]), me1 = __fmul_rn(mk, e[1]), me2 = __fmul_rn(mk, e[2]);
                const float shift[6] = {__fmul_rn(me0, e[0]), __fmul_rn(me0, e[1]), __fmul_rn(me0, e[2]),
                                        __fmul_rn(me1, e[1]), __fmul_rn(me1, e[2]), __fmul_rn(me2, e[2])};
#pragma unroll
                for (int q = 0; q < 6; ++q) {
                    const float2 qq = __ldcg(reinterpret_cast<const float2*>(s.quad + (size_t)q * n_nodes) + c0 + k);
                    Qp[q] = ff_add(Qp[q], ff{qq.x, qq.y});
                    Qp[q] = ff_add(Qp[q], shift[q]);
                }
            }
        }
        v = parent[g];
        store_node(v, n_nodes, Mp, cp, Qp, s, mass, com, quad);
    }
}

struct UpLayout {
    u32* arrive;
    MpScratch mp;
    size_t bytes;
};

UpLayout up_layout(void* ws, long long nl, long long n_particles, bool multipoles) {
    UpLayout l;
    Carver c(ws);
    long long ni = (nl - 1) / 7;
    long long nn = nl + ni;
    l.arrive = c.take<u32>((size_t)(ni > 0 ? ni : 1));
    l.mp = MpScratch{};
    if (multipoles) {
        l.mp.mass = c.take<ff>((size_t)nn);
        l.mp.quad = c.take<ff>((size_t)nn * 6);
        l.mp.xs = c.take<double>((size_t)n_particles);
        l.mp.ys = c.take<double>((size_t)n_particles);
        l.mp.zs = c.take<double>((size_t)n_particles);
        l.mp.ms = c.take<float>((size_t)n_particles);
    }
    l.bytes = c.size();
    return l;
}

}  // namespace

size_t upsweep_ws_bytes(long long nl) { return up_layout(nullptr, nl, 0, false).bytes; }
size_t multipole_ws_bytes(long long nl, long long n) { return up_layout(nullptr, nl, n, true).bytes; }

int launch_upsweep_counts(const u32* leaf_counts, long long nl, const int* leaf_to_node, const int* parent,
                          u32* node_counts, void* ws, cudaStream_t st) {
    UpLayout l = up_layout(ws, nl, 0, false);
    long long ni = (nl - 1) / 7;
    CST_CUDA(cudaMemsetAsync(ws, 0, sizeof(WsHeader), st));
    if (ni > 0) CST_CUDA(cudaMemsetAsync(l.arrive, 0, (size_t)ni * sizeof(u32), st));
    unsigned grid = static_cast<unsigned>((nl + kThreads - 1) / kThreads);
    upsweep_counts_kernel<<<grid, kThreads, 0, st>>>(leaf_counts, static_cast<u32>(nl), leaf_to_node, parent,
                                                     node_counts, l.arrive);
    CST_LAUNCHED("upsweep_counts_kernel");
    return CSTONE_OK;
}

int launch_upsweep_multipoles(const double* x, const double* y, const double* z, const float* m, const u32* perm,
                              long long n, const u32* offsets, long long nl, const int* leaf_to_node, const int* parent,
                              float* mass, double* com, float* quad, void* ws, cudaStream_t st) {
    UpLayout l = up_layout(ws, nl, n, true);
    long long ni = (nl - 1) / 7;
    CST_CUDA(cudaMemsetAsync(ws, 0, sizeof(WsHeader), st));
    if (ni > 0) CST_CUDA(cudaMemsetAsync(l.arrive, 0, (size_t)ni * sizeof(u32), st));
    unsigned grid = static_cast<unsigned>((nl + kThreads - 1) / kThreads);
    const u32 nn = static_cast<u32>(nl + ni);
    if (n > 0) {
        long long want = (n + (long long)kThreads * kGather - 1) / ((long long)kThreads * kGather);
        int ggrid = static_cast<int>(want < (long long)sm_count() * 16 ? want : (long long)sm_count() * 16);
        multipole_gather_kernel<<<ggrid, kThreads, 0, st>>>(x, y, z, m, perm, static_cast<u32>(n), l.mp);
        CST_LAUNCHED("multipole_gather_kernel");
    }
    multipole_leaf_kernel<<<grid, kThreads, 0, st>>>(offsets, static_cast<u32>(nl), leaf_to_node, nn, l.mp, mass, com,
                                                     quad);
    CST_LAUNCHED("multipole_leaf_kernel");
    if (ni > 0) {
        multipole_climb_kernel<<<grid, kThreads, 0, st>>>(static_cast<u32>(nl), leaf_to_node, parent, nn, l.mp, mass,
                                                          com, quad, l.arrive);
        CST_LAUNCHED("multipole_climb_kernel");
    }
    return CSTONE_OK;
}

}  // namespace cst

extern "C" {

int cstone_upsweep_workspace_size(int64_t n_leaves, size_t* bytes) {
    if (!bytes || n_leaves < 1 || n_leaves > CSTONE_MAX_LEAVES)
        return cst::fail(CSTONE_ERR_INVALID_ARG, "cstone_upsweep_workspace_size: bad argument");
    *bytes = cst::upsweep_ws_bytes(n_leaves);
    return CSTONE_OK;
}

int cstone_upsweep_counts(const uint32_t* leaf_counts, int64_t n_leaves, const int32_t* leaf_to_node,
                          const int32_t* parent, uint32_t* node_counts, void* ws, size_t ws_bytes, void* stream) {
    if (n_leaves < 1 || n_leaves > CSTONE_MAX_LEAVES || (n_leaves - 1) % 7 != 0 || !leaf_counts || !leaf_to_node ||
        !node_counts || (n_leaves > 1 && !parent))
        return cst::fail(CSTONE_ERR_INVALID_ARG, "cstone_upsweep_counts: bad argument");
    if (int rc = cst::check_ws(ws, ws_bytes, cst::upsweep_ws_bytes(n_leaves), "cstone_upsweep_counts")) return rc;
    return cst::launch_upsweep_counts(leaf_counts, n_leaves, leaf_to_node, parent, node_counts, ws,
                                      cst::as_stream(stream));
}

int cstone_multipole_workspace_size(int64_t n, int64_t n_leaves, size_t* bytes) {
    if (!bytes || n < 0 || n >= CSTONE_MAX_PARTICLES || n_leaves < 1 || n_leaves > CSTONE_MAX_LEAVES)
        return cst::fail(CSTONE_ERR_INVALID_ARG, "cstone_multipole_workspace_size: bad argument");
    *bytes = cst::multipole_ws_bytes(n_leaves, n);
    return CSTONE_OK;
}

int cstone_upsweep_multipoles(const double* x, const double* y, const double* z, const float* m,
                              const uint32_t* perm, int64_t n, const uint32_t* offsets, int64_t n_leaves,
                              const int32_t* leaf_to_node, const int32_t* parent, const int32_t* child,
                              float* mass, double* com, float* quad, void* ws, size_t ws_bytes, void* stream) {
    (void)child;
    if (n < 0 || n >= CSTONE_MAX_PARTICLES || n_leaves < 1 || n_leaves > CSTONE_MAX_LEAVES ||
        (n_leaves - 1) % 7 != 0 || !offsets || !leaf_to_node || !mass || !com || !quad ||
        (n > 0 && (!x || !y || !z || !m || !perm)) || (n_leaves > 1 && !parent))
        return cst::fail(CSTONE_ERR_INVALID_ARG, "cstone_upsweep_multipoles: bad argument");
    if (int rc = cst::check_ws(ws, ws_bytes, cst::multipole_ws_bytes(n_leaves, n), "cstone_upsweep_multipoles"))
        return rc;
    return cst::launch_upsweep_multipoles(x, y, z, m, perm, n, offsets, n_leaves, leaf_to_node, parent, mass, com, quad,
                                          ws, cst::as_stream(stream));
}

}  // extern "C"
