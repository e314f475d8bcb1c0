// Bounding cube and space-filling-curve keys (Sec. 3).
//
// Keys are streaming work: 24 bytes of coordinates in, 8 bytes of key out per particle. The
// kernel reads the three coordinate arrays with 16-byte vector loads (two particles per thread
// per step), computes the grid cell with the result of IEEE double precision with explicitly
// rounded operations (an integer fixed-point evaluation where its error bound proves the same
// cell; no FMA contraction, so the cell matches any IEEE host bit for bit) and encodes it. With
// masses, a second kernel also writes each particle's multipole record from the same read.
//
// Hilbert encoding uses a finite-state machine equivalent to J. Skilling's transpose formulation
// of the Hilbert curve: walking the bit levels from the top, Skilling's per-level inversions and
// exchanges act on all lower bits as a signed permutation of the axes, and the final Gray-code
// flip of a level is the parity of the Gray-coded third axis above it. Tracking (permutation,
// flips, parity) as a state gives 48 reachable states. The host builds the one-level table
// (state, octant) -> (digit, next state) once and passes it to the kernels as a by-value
// parameter (no device memory or symbol upload); each block composes it into a three-level table
// in shared memory, so a 21-level key takes 7 lookups.
#include <mutex>

#include <cooperative_groups.h>

#include "common.cuh"
#include "records.cuh"

namespace cg = cooperative_groups;

namespace CST_NS {

// ---------------------------------------------------------------------------------- bounding cube
namespace {

// A double as a signed 64-bit integer of the same order: the magnitude bits of a negative value
// are flipped, so that a more negative double is a smaller integer (the sign bit is kept, which
// makes the map its own inverse). Minima and maxima then take integer min / max: on this part the
// FP64 min / max and the unsigned 64-bit compare-and-select both cost more than the HBM stream.
__device__ __forceinline__ long long ordered_bits(double v) {
    const long long b = __double_as_longlong(v);
    return b ^ static_cast<long long>(static_cast<u64>(b >> 63) >> 1);
}

__device__ __forceinline__ double from_ordered(long long o) {
    return __longlong_as_double(o ^ static_cast<long long>(static_cast<u64>(o >> 63) >> 1));
}

constexpr long long kOrderedMax = 0x7fffffffffffffffLL;
constexpr long long kOrderedMin = -kOrderedMax - 1;

struct BoxAcc {
    long long lo[3];  // ordered bits of the per-axis minimum
    long long hi[3];  // ordered bits of the per-axis maximum
};

__global__ void bbox_init_kernel(BoxAcc* acc) {
    int t = threadIdx.x;
    if (t < 3) {
        acc->lo[t] = kOrderedMax;
        acc->hi[t] = kOrderedMin;
    }
}

__global__ void __launch_bounds__(256) bbox_reduce_kernel(const double* __restrict__ x, const double* __restrict__ y,
                                                          const double* __restrict__ z, long long n, BoxAcc* acc) {
    long long lo[3] = {kOrderedMax, kOrderedMax, kOrderedMax}, hi[3] = {kOrderedMin, kOrderedMin, kOrderedMin};
    const double* c[3] = {x, y, z};
    auto take = [&](int d, double v) {
        const long long o = ordered_bits(v);
        lo[d] = min(lo[d], o);
        hi[d] = max(hi[d], o);
    };
    const bool vec = ((reinterpret_cast<uintptr_t>(x) | reinterpret_cast<uintptr_t>(y) | reinterpret_cast<uintptr_t>(z)) &
                      15u) == 0;
    const long long stride = (long long)gridDim.x * blockDim.x;
    long long done = 0;
    if (vec) {  // two 16-byte loads per array and thread per step: 6 loads in flight
        const long long quads = n >> 2;
        for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < quads; q += stride) {
            double2 v[3][2];
#pragma unroll
            for (int d = 0; d < 3; ++d) {
                const double2* p = reinterpret_cast<const double2*>(c[d]) + 2 * q;
                v[d][0] = __ldcg(p);
                v[d][1] = __ldcg(p + 1);
            }
#pragma unroll
            for (int d = 0; d < 3; ++d) {
                take(d, v[d][0].x);
                take(d, v[d][0].y);
                take(d, v[d][1].x);
                take(d, v[d][1].y);
            }
        }
        done = quads << 2;
    }
    for (long long i = done + blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += stride) {
#pragma unroll
        for (int d = 0; d < 3; ++d) take(d, __ldg(c[d] + i));
    }
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        for (int s = 16; s > 0; s >>= 1) {
            lo[d] = min(lo[d], __shfl_xor_sync(0xffffffffu, lo[d], s));
            hi[d] = max(hi[d], __shfl_xor_sync(0xffffffffu, hi[d], s));
        }
    }
    // the block's warps through shared memory, then one update of the global bounds per block
    // (all blocks update the same six words)
    __shared__ long long s_lo[8][3], s_hi[8][3];
    const int warp = threadIdx.x >> 5;
    if ((threadIdx.x & 31) == 0)
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            s_lo[warp][d] = lo[d];
            s_hi[warp][d] = hi[d];
        }
    __syncthreads();
    if (threadIdx.x < 3) {
        const int d = threadIdx.x;
        long long l = s_lo[0][d], h = s_hi[0][d];
        for (int w = 1; w < static_cast<int>(blockDim.x >> 5); ++w) {
            l = min(l, s_lo[w][d]);
            h = max(h, s_hi[w][d]);
        }
        atomicMin(&acc->lo[d], l);
        atomicMax(&acc->hi[d], h);
    }
}

// Per-axis minima and maxima {min x, min y, min z, max x, max y, max z}; with no points the
// minima are +inf and the maxima -inf, so that a reduction over several sets ignores an empty one.
__global__ void bounds_finalize_kernel(const BoxAcc* acc, long long n, double* bounds) {
    if (threadIdx.x >= 3) return;
    const int d = threadIdx.x;
    bounds[d] = n > 0 ? from_ordered(acc->lo[d]) : __longlong_as_double(0x7ff0000000000000LL);
    bounds[3 + d] = n > 0 ? from_ordered(acc->hi[d]) : __longlong_as_double(static_cast<long long>(0xfff0000000000000ULL));
}

__global__ void bbox_finalize_kernel(const BoxAcc* acc, long long n, double* box) {
    if (threadIdx.x != 0) return;
    if (n == 0) {
        box[0] = box[1] = box[2] = 0.0;
        box[3] = 1.0;
        return;
    }
    double side = 0.0;
    for (int d = 0; d < 3; ++d) {
        double lo = from_ordered(acc->lo[d]);
        double hi = from_ordered(acc->hi[d]);
        box[d] = lo;
        double ext = __dsub_rn(hi, lo);
        side = ext > side ? ext : side;
    }
    box[3] = side > 0.0 ? side : 1.0;
}

// ---------------------------------------------------------------------------------- grid + keys
struct HilbertTable {
    unsigned short one[kHilbertStates * 8];  // (state, 1 octant) -> 3 digit bits | next << 3
};

// Cell index of one coordinate: floor((x - lo) * scale) clamped to [0, 2^21 - 1], with the
// subtraction and the product rounded once each (explicit round-to-nearest intrinsics keep the
// compiler from fusing them into an FMA).
__device__ __forceinline__ u32 grid_cell(double x, double lo, double scale) {
    double u = __dmul_rn(__dsub_rn(x, lo), scale);
    if (!(u > 0.0)) return 0u;
    if (u >= 2097152.0) return 2097151u;
    return __double2uint_rz(u);
}

// Integer evaluation of grid_cell. Double-precision throughput is a small fraction of the integer
// throughput on this GPU, so the cell is first computed in 64-bit fixed point:
//   X = trunc(x * 2^F), LO = trunc(lo * 2^F), u * 2^R ~= ((X - LO) * S) >> 64, S = scale * 2^G,
// with F chosen so |X| < 2^61 on [lo, lo + 2 side) and S holding scale's 53-bit mantissa at the
// top of 64 bits. The truncations, the product and the two IEEE roundings of the reference
// together move u by far less than 2^-24 cells, so whenever the fixed-point u is at least 2^-20
// away from an integer its floor is the floor of the IEEE result. The remaining ~2^-19 of
// coordinates, and boxes where the error bound does not hold, take the IEEE path.
struct FixedGrid {
    long long lo_fixed;   // LO
    u64 scale_fixed;      // S
    u64 lo_ord, hi_ord;   // order-preserving bits of lo and of lo + 2 side
    double lo, scale;
    int F, R;
    int fast;
};

__device__ __forceinline__ u64 order_bits(double v) {
    u64 b = static_cast<u64>(__double_as_longlong(v));
    return (b >> 63) ? ~b : (b | (1ULL << 63));
}

__device__ __forceinline__ int exponent_of(double v) {  // unbiased exponent field (0 for zero/subnormal)
    return static_cast<int>((static_cast<u64>(__double_as_longlong(v)) >> 52) & 0x7ffu);
}

// trunc(x * 2^F) for |x| * 2^F < 2^62
__device__ __forceinline__ long long to_fixed(double x, int F) {
    u64 b = static_cast<u64>(__double_as_longlong(x));
    int e = static_cast<int>((b >> 52) & 0x7ffu);
    u64 mant = b & ((1ULL << 52) - 1);
    if (e != 0) mant |= (1ULL << 52);
    int sh = (e == 0 ? 1 : e) - 1075 + F;
    u64 mag = sh >= 0 ? (mant << sh) : (sh > -64 ? (mant >> (-sh)) : 0ULL);
    return (b >> 63) ? -static_cast<long long>(mag) : static_cast<long long>(mag);
}

// F_frame != 0: take that fixed-point exponent (a frame shared with other arrays) instead of the
// axis' own; the fast path is then enabled only where its error bound holds for it.
__device__ FixedGrid make_fixed_grid(double lo, double side, int F_frame = 0) {
    FixedGrid f;
    f.lo = lo;
    f.scale = __ddiv_rn(2097152.0, side);
    const double hi = __dadd_rn(lo, __dmul_rn(2.0, side));
    f.lo_ord = order_bits(lo);
    f.hi_ord = order_bits(hi);
    // 2^E > max(|lo|, |hi|)
    const int e_max = max(exponent_of(lo), exponent_of(hi)) - 1023 + 1;
    f.F = F_frame != 0 && F_frame <= 61 - e_max ? F_frame : 61 - e_max;
    const int es = exponent_of(f.scale) - 1023 - 52;  // scale = mantissa * 2^es
    const int G = 11 - es;
    f.R = f.F + G - 64;
    u64 sb = static_cast<u64>(__double_as_longlong(f.scale));
    f.scale_fixed = ((sb & ((1ULL << 52) - 1)) | (1ULL << 52)) << 11;
    f.fast = (f.R >= 26 && f.R <= 62 && es + 78 <= f.F && f.F <= 1074 && exponent_of(f.scale) != 0 &&
              exponent_of(f.scale) != 0x7ff && !(hi <= lo));
    f.lo_fixed = f.fast ? to_fixed(lo, f.F) : 0;
    return f;
}

// X: trunc(x * 2^F) when already known (the record-writing pass shares it with the record), or
// computed here (only for x inside the box, where it cannot overflow).
template <bool HAVE_X = false>
__device__ __forceinline__ u32 grid_cell_fixed(double x, const FixedGrid& f, long long X = 0) {
    const u64 o = order_bits(x);
    if (o <= f.lo_ord) return 0u;
    if (o >= f.hi_ord) return 2097151u;
    const u64 d = static_cast<u64>((HAVE_X ? X : to_fixed(x, f.F)) - f.lo_fixed);
    const u64 u = __umul64hi(d, f.scale_fixed);
    const u32 frac20 = static_cast<u32>(u >> (f.R - 20)) & 0xfffffu;
    if (frac20 == 0u || frac20 == 0xfffffu) return grid_cell(x, f.lo, f.scale);
    const u64 g = u >> f.R;
    return g > 2097151ULL ? 2097151u : static_cast<u32>(g);
}

// Spread the 21 bits of v to every third bit position (bit b -> bit 3b).
__device__ __forceinline__ u64 spread3(u32 v) {
    u64 x = v & 0x1fffffu;
    x = (x | (x << 32)) & 0x001f00000000ffffULL;
    x = (x | (x << 16)) & 0x001f0000ff0000ffULL;
    x = (x | (x << 8)) & 0x100f00f00f00f00fULL;
    x = (x | (x << 4)) & 0x10c30c30c30c30c3ULL;
    x = (x | (x << 2)) & 0x1249249249249249ULL;
    return x;
}

__device__ __forceinline__ u64 morton_of(u32 gx, u32 gy, u32 gz) {
    return (spread3(gx) << 2) | (spread3(gy) << 1) | spread3(gz);
}

// Key of this build's length from a 63-bit key: the cell of a coarser grid is the top 3L bits of
// the 21-level key (octree prefix of both curves, and floor(cell_21 / 2^(21-L)) = cell_L exactly
// because the grid scales differ by a power of two).
__device__ __forceinline__ Key to_key(u64 k63) { return static_cast<Key>(k63 >> (63 - kKeyBits)); }

// The three fixed-point grids of the box and the one-level Hilbert table in shared memory (both
// key kernels); Hilbert keys also use a three-level table in dynamic shared memory, indexed by the
// state and 3 bits of each coordinate's cell (3 levels, x bits above y bits above z bits), so a key
// takes 7 lookups and no Morton interleave. Each block builds it from the one-level table.
struct KeySmem {
    unsigned short t1[kHilbertStates * 8];
    FixedGrid grid[3];
};
constexpr int kHilbert3Entries = kHilbertStates * 512;
constexpr size_t kHilbert3Bytes = kHilbert3Entries * sizeof(unsigned short);  // 48 KB

template <int CURVE>
__device__ __forceinline__ void load_key_smem(KeySmem& sm, unsigned short* t3, const HilbertTable& table,
                                              const double* box, bool record_frame = false, bool grids = true) {
    if (CURVE == CSTONE_HILBERT)
        for (int i = threadIdx.x; i < kHilbertStates * 8; i += blockDim.x) sm.t1[i] = table.one[i];
    if (grids && threadIdx.x < 3)
        sm.grid[threadIdx.x] = make_fixed_grid(box[threadIdx.x], box[3], record_frame ? make_frame(box).F : 0);
    if (CURVE == CSTONE_HILBERT) {
        __syncthreads();
        // entry (state, x3 y3 z3): three one-level steps, the octant of each level taken from the
        // top remaining bit of x3, y3, z3 (x most significant, as in the Morton interleave)
        for (int e = threadIdx.x; e < kHilbert3Entries; e += blockDim.x) {
            const int idx = e & 511;
            u32 state = static_cast<u32>(e >> 9), digits = 0;
#pragma unroll
            for (int lv = 2; lv >= 0; --lv) {
                const u32 o = (((idx >> (6 + lv)) & 1u) << 2) | (((idx >> (3 + lv)) & 1u) << 1) | ((idx >> lv) & 1u);
                const u32 v = sm.t1[state * 8u + o];
                digits = (digits << 3) | (v & 7u);
                state = v >> 3;
            }
            t3[e] = static_cast<unsigned short>(digits | (state << 9));
        }
    }
}

// 63-bit Hilbert key of a cell from the three-level table: 7 steps of 3 levels.
__device__ __forceinline__ u64 hilbert_of_cell(u32 gx, u32 gy, u32 gz, const unsigned short* t3) {
    u64 key = 0;
    u32 state = 0;
#pragma unroll
    for (int sh = 18; sh >= 0; sh -= 3) {
        const u32 idx = (((gx >> sh) & 7u) << 6) | (((gy >> sh) & 7u) << 3) | ((gz >> sh) & 7u);
        const u32 v = t3[state * 512u + idx];
        key = (key << 9) | (v & 511u);
        state = v >> 9;
    }
    return key;
}

template <int CURVE, bool HAVE_X = false>
__device__ __forceinline__ Key encode_key(const KeySmem& sm, const unsigned short* t3, bool fast, double px,
                                          double py, double pz, long long X = 0, long long Y = 0, long long Z = 0) {
    u32 gx, gy, gz;
    if (fast) {
        gx = grid_cell_fixed<HAVE_X>(px, sm.grid[0], X);
        gy = grid_cell_fixed<HAVE_X>(py, sm.grid[1], Y);
        gz = grid_cell_fixed<HAVE_X>(pz, sm.grid[2], Z);
    } else {
        gx = grid_cell(px, sm.grid[0].lo, sm.grid[0].scale);
        gy = grid_cell(py, sm.grid[1].lo, sm.grid[1].scale);
        gz = grid_cell(pz, sm.grid[2].lo, sm.grid[2].scale);
    }
    if (CURVE == CSTONE_HILBERT) return to_key(hilbert_of_cell(gx, gy, gz, t3));
    return to_key(morton_of(gx, gy, gz));
}

template <int CURVE, bool VEC>
__global__ void __launch_bounds__(256) keys_kernel(const double* __restrict__ x, const double* __restrict__ y,
                                                   const double* __restrict__ z, long long n,
                                                   const double* __restrict__ box, Key* __restrict__ keys,
                                                   const __grid_constant__ HilbertTable table) {
    __shared__ KeySmem sm;
    extern __shared__ unsigned short t3[];  // kHilbert3Bytes for Hilbert keys
    load_key_smem<CURVE>(sm, t3, table, box);
    __syncthreads();
    const bool fast = sm.grid[0].fast && sm.grid[1].fast && sm.grid[2].fast;
    auto encode = [&](double px, double py, double pz) -> Key { return encode_key<CURVE>(sm, t3, fast, px, py, pz); };

    if (!VEC) {
        for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
            keys[i] = encode(__ldcg(x + i), __ldcg(y + i), __ldcg(z + i));
        return;
    }
    const long long pairs = n >> 1;
    const double2* x2 = reinterpret_cast<const double2*>(x);
    const double2* y2 = reinterpret_cast<const double2*>(y);
    const double2* z2 = reinterpret_cast<const double2*>(z);
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < pairs; i += (long long)gridDim.x * blockDim.x) {
        double2 a = __ldcg(x2 + i), b = __ldcg(y2 + i), c = __ldcg(z2 + i);
        const Key k0 = encode(a.x, b.x, c.x), k1 = encode(a.y, b.y, c.y);
        if constexpr (sizeof(Key) == 8)
            __stcs(reinterpret_cast<ulonglong2*>(keys) + i, make_ulonglong2(k0, k1));
        else
            __stcs(reinterpret_cast<uint2*>(keys) + i, make_uint2(k0, k1));
    }
    if ((n & 1) && blockIdx.x == 0 && threadIdx.x == 0) {
        long long i = n - 1;
        keys[i] = encode(x[i], y[i], z[i]);
    }
}

// Keys and each particle's multipole record (fixed-point position and mass, records.cuh) from
// the same read of the coordinates. A warp takes 64 consecutive particles, lane l the particles
// l and l + 32: both halves keep the warp's loads and stores contiguous (a warp's two 16-byte
// record stores cover 1 KB), and the two encodings interleave.
#ifndef CSTONE_KEYS_REC_MIN_BLOCKS
#define CSTONE_KEYS_REC_MIN_BLOCKS 3
#endif
template <int CURVE>
__global__ void __launch_bounds__(256, CSTONE_KEYS_REC_MIN_BLOCKS)
    keys_records_kernel(const double* __restrict__ x, const double* __restrict__ y, const double* __restrict__ z,
                        const float* __restrict__ m, long long n, const double* __restrict__ box,
                        Key* __restrict__ keys, Record* __restrict__ rec, WsHeader* hdr,
                        const __grid_constant__ HilbertTable table) {
    __shared__ KeySmem sm;
    __shared__ FixedFrame s_frame;
    extern __shared__ unsigned short t3[];  // kHilbert3Bytes for Hilbert keys
    load_key_smem<CURVE>(sm, t3, table, box, true);  // the grids take the records' fixed-point frame
    if (threadIdx.x == 32) s_frame = make_frame(box);
    __syncthreads();
    // the fixed-point coordinate serves the record and, where the fast path is on, the grid cell
    const bool fast = sm.grid[0].fast && sm.grid[1].fast && sm.grid[2].fast && sm.grid[0].F == s_frame.F &&
                      sm.grid[1].F == s_frame.F && sm.grid[2].F == s_frame.F;
    const FixedFrame fr = s_frame;
    const long long lane = threadIdx.x & 31;
    const long long warps = (long long)gridDim.x * (blockDim.x >> 5);
    auto fixed = [&](double v, bool& in) -> long long {
        const bool ok = static_cast<int>((static_cast<u64>(__double_as_longlong(v)) >> 52) & 0x7ffu) < fr.e_lim;
        in = in && ok;
        return ok ? fixed_of(v, fr.F) : 0;
    };
    auto one = [&](long long i, double px, double py, double pz, float pm) -> Key {
        bool in = true;
        const long long X = fixed(px, in), Y = fixed(py, in), Z = fixed(pz, in);
        const Key k = fast ? encode_key<CURVE, true>(sm, t3, true, px, py, pz, X, Y, Z)
                           : encode_key<CURVE>(sm, t3, false, px, py, pz);
        longlong2* dst = reinterpret_cast<longlong2*>(rec + i);
        __stcs(dst, make_longlong2(in ? X : 0, in ? Y : 0));
        __stcs(dst + 1, make_longlong2(in ? Z : 0, static_cast<long long>(__float_as_uint(pm))));
        if (!in) raise_error(hdr, CSTONE_ERR_INVALID_ARG, static_cast<u32>(i));
        return k;
    };
    for (long long base = ((long long)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5)) * 64; base < n;
         base += warps * 64) {
        const long long i0 = base + lane, i1 = base + 32 + lane;
        if (i0 >= n) break;
        const bool ok1 = i1 < n;
        const double ax = __ldcg(x + i0), ay = __ldcg(y + i0), az = __ldcg(z + i0);
        const float am = __ldcg(m + i0);
        double bx = 0.0, by = 0.0, bz = 0.0;
        float bm = 0.f;
        if (ok1) {
            bx = __ldcg(x + i1);
            by = __ldcg(y + i1);
            bz = __ldcg(z + i1);
            bm = __ldcg(m + i1);
        }
        keys[i0] = one(i0, ax, ay, az, am);
        if (ok1) keys[i1] = one(i1, bx, by, bz, bm);
    }
}

// ------------------------------------------------------------------ host: Hilbert state machine
// State of Skilling's walk seen from one bit level: perm[i] = input axis currently feeding
// transposed axis i, flip[i] = inversion of that axis, gray = parity of the Gray-coded third
// axis over the levels above (the final per-level flip of Skilling's algorithm).
struct WalkState {
    int perm[3];
    int flip[3];
    int gray;
    bool operator==(const WalkState& o) const {
        for (int i = 0; i < 3; ++i)
            if (perm[i] != o.perm[i] || flip[i] != o.flip[i]) return false;
        return gray == o.gray;
    }
};

// One bit level: input octant bits (x high) -> output digit, state updated for the next level.
int walk_level(WalkState& s, int octant) {
    int in[3] = {(octant >> 2) & 1, (octant >> 1) & 1, octant & 1};
    int e[3];
    for (int i = 0; i < 3; ++i) e[i] = in[s.perm[i]] ^ s.flip[i];
    for (int i = 0; i < 3; ++i) {
        if (e[i]) {
            s.flip[0] ^= 1;  // inversion of the first axis' lower bits
        } else {             // exchange of the lower bits of the first axis and axis i
            int tp = s.perm[0], tf = s.flip[0];
            s.perm[0] = s.perm[i];
            s.flip[0] = s.flip[i];
            s.perm[i] = tp;
            s.flip[i] = tf;
        }
    }
    int g0 = e[0], g1 = e[1] ^ e[0], g2 = e[2] ^ g1;
    int digit = ((g0 ^ s.gray) << 2) | ((g1 ^ s.gray) << 1) | (g2 ^ s.gray);
    s.gray ^= g2;
    return digit;
}

const HilbertTable& hilbert_table() {
    static HilbertTable table;
    static std::once_flag once;
    std::call_once(once, [] {
        WalkState states[kHilbertStates];
        int count = 1;
        states[0] = WalkState{{0, 1, 2}, {0, 0, 0}, 0};
        int next1[kHilbertStates][8], digit1[kHilbertStates][8];
        for (int s = 0; s < count; ++s) {
            for (int o = 0; o < 8; ++o) {
                WalkState w = states[s];
                digit1[s][o] = walk_level(w, o);
                int id = -1;
                for (int k = 0; k < count; ++k)
                    if (states[k] == w) id = k;
                if (id < 0) {
                    id = count;
                    if (count < kHilbertStates) states[count++] = w;
                }
                next1[s][o] = id;
            }
        }
        for (int s = 0; s < kHilbertStates; ++s) {
            for (int o = 0; o < 8; ++o)
                table.one[s * 8 + o] = static_cast<unsigned short>(digit1[s][o] | (next1[s][o] << 3));
        }
    });
    return table;
}

// ------------------------------------------------------------------ batched sets
// Set of particle p: the last set whose first particle is <= p (sets are stored back to back).
__device__ __forceinline__ int set_of(const long long* __restrict__ set_offsets, int n_sets, long long p) {
    int lo = 0, hi = n_sets;
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (__ldg(set_offsets + mid) <= p)
            lo = mid;
        else
            hi = mid;
    }
    while (lo + 1 < n_sets && __ldg(set_offsets + lo + 1) <= p) ++lo;  // skip empty sets
    return lo;
}

// Bounding cube of every set: one cluster of kBoxCluster blocks per set (a large set is read by
// kBoxCluster SMs, not one); each block reduces its share of the set, and the cluster's first block
// combines the blocks' results from their shared memory (distributed shared memory of the cluster).
constexpr int kBoxCluster = 16;  // a non-portable cluster size, allowed per kernel at launch
constexpr int kBoxThreads = 256;

__global__ void __cluster_dims__(kBoxCluster, 1, 1) __launch_bounds__(kBoxThreads)
    bbox_batched_kernel(const double* __restrict__ x, const double* __restrict__ y, const double* __restrict__ z,
                        const long long* __restrict__ set_offsets, double* __restrict__ boxes) {
    __shared__ long long s_lo[kBoxThreads / 32][3], s_hi[kBoxThreads / 32][3];
    __shared__ long long s_blo[3], s_bhi[3];  // this block's result, read by the cluster's first block
    cg::cluster_group cluster = cg::this_cluster();
    const unsigned rank = cluster.block_rank();
    const int set = static_cast<int>(blockIdx.x / kBoxCluster);
    const long long a = set_offsets[set], b = set_offsets[set + 1];
    long long lo[3] = {kOrderedMax, kOrderedMax, kOrderedMax}, hi[3] = {kOrderedMin, kOrderedMin, kOrderedMin};
    const double* c[3] = {x, y, z};
    for (long long i = a + static_cast<long long>(rank) * kBoxThreads + threadIdx.x; i < b;
         i += static_cast<long long>(kBoxCluster) * kBoxThreads) {
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            const long long o = ordered_bits(__ldg(c[d] + i));
            lo[d] = min(lo[d], o);
            hi[d] = max(hi[d], o);
        }
    }
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        for (int sft = 16; sft > 0; sft >>= 1) {
            lo[d] = min(lo[d], __shfl_xor_sync(0xffffffffu, lo[d], sft));
            hi[d] = max(hi[d], __shfl_xor_sync(0xffffffffu, hi[d], sft));
        }
    }
    const int warp = threadIdx.x >> 5;
    if ((threadIdx.x & 31) == 0)
        for (int d = 0; d < 3; ++d) {
            s_lo[warp][d] = lo[d];
            s_hi[warp][d] = hi[d];
        }
    __syncthreads();
    if (threadIdx.x < 3) {
        const int d = threadIdx.x;
        long long l = s_lo[0][d], h = s_hi[0][d];
        for (int w = 1; w < kBoxThreads / 32; ++w) {
            l = min(l, s_lo[w][d]);
            h = max(h, s_hi[w][d]);
        }
        s_blo[d] = l;
        s_bhi[d] = h;
    }
    cluster.sync();  // every block's result is in its shared memory
    if (rank == 0 && threadIdx.x == 0) {
        double* box = boxes + 4 * set;
        if (b <= a) {
            box[0] = box[1] = box[2] = 0.0;
            box[3] = 1.0;
        } else {
            double side = 0.0;
            for (int d = 0; d < 3; ++d) {
                long long l = s_blo[d], h = s_bhi[d];
                for (unsigned r = 1; r < kBoxCluster; ++r) {
                    l = min(l, cluster.map_shared_rank(s_blo, r)[d]);
                    h = max(h, cluster.map_shared_rank(s_bhi, r)[d]);
                }
                const double lod = from_ordered(l), hid = from_ordered(h);
                box[d] = lod;
                const double ext = __dsub_rn(hid, lod);
                side = ext > side ? ext : side;
            }
            box[3] = side > 0.0 ? side : 1.0;
        }
    }
    cluster.sync();  // the other blocks keep their shared memory until it has been read
}

__global__ void keys_batched_setup_kernel(const double* __restrict__ boxes, int n_sets, FixedGrid* grids) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < 3 * n_sets; i += gridDim.x * blockDim.x) {
        const int sidx = i / 3, d = i % 3;
        grids[i] = make_fixed_grid(boxes[4 * sidx + d], boxes[4 * sidx + 3]);
    }
}

template <int CURVE>
__global__ void __launch_bounds__(256) keys_batched_kernel(const double* __restrict__ x, const double* __restrict__ y,
                                                           const double* __restrict__ z,
                                                           const long long* __restrict__ set_offsets, int n_sets,
                                                           long long n, const FixedGrid* __restrict__ grids,
                                                           Key* __restrict__ keys,
                                                           const __grid_constant__ HilbertTable table) {
    __shared__ KeySmem sm;  // only its one-level table is used here (the grids are per set)
    extern __shared__ unsigned short t3[];  // kHilbert3Bytes for Hilbert keys
    if (CURVE == CSTONE_HILBERT) load_key_smem<CURVE>(sm, t3, table, nullptr, false, false);
    __syncthreads();
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const int sidx = set_of(set_offsets, n_sets, i);
        const FixedGrid* g = grids + 3 * sidx;
        const double px = __ldcg(x + i), py = __ldcg(y + i), pz = __ldcg(z + i);
        u32 c[3];
        const double pc[3] = {px, py, pz};
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            const FixedGrid f = g[d];
            c[d] = f.fast ? grid_cell_fixed(pc[d], f) : grid_cell(pc[d], f.lo, f.scale);
        }
        keys[i] = to_key(CURVE == CSTONE_HILBERT ? hilbert_of_cell(c[0], c[1], c[2], t3) : morton_of(c[0], c[1], c[2]));
    }
}

}  // namespace

const HilbertDecodeTable& hilbert_decode_table() {
    static HilbertDecodeTable dec;
    static std::once_flag once;
    std::call_once(once, [] {
        const HilbertTable& t = hilbert_table();
        for (int s = 0; s < kHilbertStates; ++s)
            for (int o = 0; o < 8; ++o) {
                const int e = t.one[s * 8 + o];
                dec.one[s * 8 + (e & 7)] = static_cast<unsigned short>(o | ((e >> 3) << 3));
            }
    });
    return dec;
}

size_t keys_batched_ws_bytes(int n_sets) {
    Carver c(nullptr);
    c.take<FixedGrid>((size_t)n_sets * 3);
    return c.size();
}

int launch_bbox_batched(const double* x, const double* y, const double* z, const long long* set_offsets, int n_sets,
                        double* boxes, cudaStream_t st) {
    CST_CUDA(cudaFuncSetAttribute(bbox_batched_kernel, cudaFuncAttributeNonPortableClusterSizeAllowed, 1));
    bbox_batched_kernel<<<n_sets * kBoxCluster, kBoxThreads, 0, st>>>(x, y, z, set_offsets, boxes);
    CST_LAUNCHED("bbox_batched_kernel");
    return CSTONE_OK;
}

int launch_keys_batched(const double* x, const double* y, const double* z, const long long* set_offsets, int n_sets,
                        long long n, const double* boxes, int curve, Key* keys, void* ws, cudaStream_t st) {
    Carver c(ws);
    FixedGrid* grids = c.take<FixedGrid>((size_t)n_sets * 3);
    keys_batched_setup_kernel<<<(3 * n_sets + 127) / 128, 128, 0, st>>>(boxes, n_sets, grids);
    CST_LAUNCHED("keys_batched_setup_kernel");
    if (n == 0) return CSTONE_OK;
    const HilbertTable& tab = hilbert_table();
    const long long want = (n + 255) / 256;
    const int grid = static_cast<int>(want < (long long)sm_count() * 8 ? want : (long long)sm_count() * 8);
    if (curve == CSTONE_HILBERT) {  // the three-level table takes 48 KB of dynamic shared memory
        CST_CUDA(cudaFuncSetAttribute(keys_batched_kernel<CSTONE_HILBERT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      static_cast<int>(kHilbert3Bytes)));
        keys_batched_kernel<CSTONE_HILBERT><<<grid, 256, kHilbert3Bytes, st>>>(x, y, z, set_offsets, n_sets, n, grids,
                                                                               keys, tab);
    }
    else
        keys_batched_kernel<CSTONE_MORTON><<<grid, 256, 0, st>>>(x, y, z, set_offsets, n_sets, n, grids, keys, tab);
    CST_LAUNCHED("keys_batched_kernel");
    return CSTONE_OK;
}

int launch_keys(const double* x, const double* y, const double* z, long long n, const double* box, int curve,
                Key* keys, cudaStream_t st) {
    if (n == 0) return CSTONE_OK;
    const HilbertTable& tab = hilbert_table();
    long long pairs = (n + 1) / 2;
    long long want = (pairs + 255) / 256;
    int grid = static_cast<int>(want < (long long)sm_count() * 8 ? (want > 0 ? want : 1) : (long long)sm_count() * 8);
    bool vec = ((reinterpret_cast<uintptr_t>(x) | reinterpret_cast<uintptr_t>(y) | reinterpret_cast<uintptr_t>(z) |
                 reinterpret_cast<uintptr_t>(keys)) & 15u) == 0;
    if (curve == CSTONE_HILBERT) {  // the three-level table takes 48 KB of dynamic shared memory
        CST_CUDA(cudaFuncSetAttribute(keys_kernel<CSTONE_HILBERT, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      static_cast<int>(kHilbert3Bytes)));
        CST_CUDA(cudaFuncSetAttribute(keys_kernel<CSTONE_HILBERT, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      static_cast<int>(kHilbert3Bytes)));
        if (vec)
            keys_kernel<CSTONE_HILBERT, true><<<grid, 256, kHilbert3Bytes, st>>>(x, y, z, n, box, keys, tab);
        else
            keys_kernel<CSTONE_HILBERT, false><<<grid, 256, kHilbert3Bytes, st>>>(x, y, z, n, box, keys, tab);
    } else {
        if (vec)
            keys_kernel<CSTONE_MORTON, true><<<grid, 256, 0, st>>>(x, y, z, n, box, keys, tab);
        else
            keys_kernel<CSTONE_MORTON, false><<<grid, 256, 0, st>>>(x, y, z, n, box, keys, tab);
    }
    CST_LAUNCHED("keys_kernel");
    return CSTONE_OK;
}

// Keys and multipole records in one pass; ws holds only the header (error word).
int launch_keys_records(const double* x, const double* y, const double* z, const float* m, long long n,
                        const double* box, int curve, Key* keys, Record* rec, void* ws, cudaStream_t st) {
    WsHeader* hdr = reinterpret_cast<WsHeader*>(ws);
    CST_CUDA(cudaMemsetAsync(hdr, 0, sizeof(WsHeader), st));
    if (n == 0) return CSTONE_OK;
    const HilbertTable& tab = hilbert_table();
    long long want = (n + 511) / 512;  // 64 particles per warp and step
    int grid = static_cast<int>(want < (long long)sm_count() * 8 ? (want > 0 ? want : 1) : (long long)sm_count() * 8);
    if (curve == CSTONE_HILBERT)
        CST_CUDA(cudaFuncSetAttribute(keys_records_kernel<CSTONE_HILBERT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      static_cast<int>(kHilbert3Bytes)));
    if (curve == CSTONE_HILBERT)
        keys_records_kernel<CSTONE_HILBERT><<<grid, 256, kHilbert3Bytes, st>>>(x, y, z, m, n, box, keys, rec, hdr, tab);
    else
        keys_records_kernel<CSTONE_MORTON><<<grid, 256, 0, st>>>(x, y, z, m, n, box, keys, rec, hdr, tab);
    CST_LAUNCHED("keys_records_kernel");
    return CSTONE_OK;
}

// bounding cube (bounds == false: box = {lo, side}) or per-axis bounds (bounds == true)
int launch_bbox(const double* x, const double* y, const double* z, long long n, double* box, void* ws,
                cudaStream_t st, bool bounds = false) {
    Carver c(ws);
    BoxAcc* acc = c.take<BoxAcc>(1);
    bbox_init_kernel<<<1, 32, 0, st>>>(acc);
    CST_LAUNCHED("bbox_init_kernel");
    if (n > 0) {
        long long want = (n + 1023) / 1024;  // 16 blocks per SM measured best (two waves of 8)
        int grid = static_cast<int>(want < (long long)sm_count() * 16 ? want : (long long)sm_count() * 16);
        bbox_reduce_kernel<<<grid, 256, 0, st>>>(x, y, z, n, acc);
        CST_LAUNCHED("bbox_reduce_kernel");
    }
    if (bounds) {
        bounds_finalize_kernel<<<1, 32, 0, st>>>(acc, n, box);
        CST_LAUNCHED("bounds_finalize_kernel");
    } else {
        bbox_finalize_kernel<<<1, 32, 0, st>>>(acc, n, box);
        CST_LAUNCHED("bbox_finalize_kernel");
    }
    return CSTONE_OK;
}

size_t bbox_ws_bytes() {
    Carver c(nullptr);
    c.take<BoxAcc>(1);
    return c.size();
}

}  // namespace CST_NS

extern "C" {

int CSTONE_FN(keys)(const double* x, const double* y, const double* z, int64_t n, const double* box, int curve,
                    CST_KEY_C* keys, void* stream) {
    if (n < 0 || n >= CSTONE_MAX_PARTICLES || !box || (n > 0 && (!x || !y || !z || !keys)))
        return cst::fail(CSTONE_ERR_INVALID_ARG, CST_STR(CSTONE_FN(keys)) ": bad argument (n=%lld)", (long long)n);
    if (curve != CSTONE_MORTON && curve != CSTONE_HILBERT)
        return cst::fail(CSTONE_ERR_INVALID_ARG, CST_STR(CSTONE_FN(keys)) ": unknown curve %d", curve);
    if (((reinterpret_cast<uintptr_t>(x) | reinterpret_cast<uintptr_t>(y) | reinterpret_cast<uintptr_t>(z)) & 7u) != 0 ||
        (reinterpret_cast<uintptr_t>(keys) & (sizeof(CST_KEY_C) - 1)) != 0)
        return cst::fail(CSTONE_ERR_INVALID_ARG, CST_STR(CSTONE_FN(keys)) ": arrays must be aligned to their element size");
    return CST_NS::launch_keys(x, y, z, n, box, curve, reinterpret_cast<CST_NS::Key*>(keys), cst::as_stream(stream));
}

int CSTONE_FN(keys_records)(const double* x, const double* y, const double* z, const float* m, int64_t n,
                            const double* box, int curve, CST_KEY_C* keys, void* records, void* ws, size_t ws_bytes,
                            void* stream) {
    if (n < 0 || n >= CSTONE_MAX_PARTICLES || !box || (n > 0 && (!x || !y || !z || !m || !keys || !records)))
        return cst::fail(CSTONE_ERR_INVALID_ARG, CST_STR(CSTONE_FN(keys_records)) ": bad argument (n=%lld)",
                         (long long)n);
    if (curve != CSTONE_MORTON && curve != CSTONE_HILBERT)
        return cst::fail(CSTONE_ERR_INVALID_ARG, CST_STR(CSTONE_FN(keys_records)) ": unknown curve %d", curve);
    if (((reinterpret_cast<uintptr_t>(x) | reinterpret_cast<uintptr_t>(y) | reinterpret_cast<uintptr_t>(z)) & 7u) != 0 ||
        (reinterpret_cast<uintptr_t>(m) & 3u) != 0 || (reinterpret_cast<uintptr_t>(records) & 15u) != 0 ||
        (reinterpret_cast<uintptr_t>(keys) & (sizeof(CST_KEY_C) - 1)) != 0)
        return cst::fail(CSTONE_ERR_INVALID_ARG,
                         CST_STR(CSTONE_FN(keys_records)) ": arrays must be aligned (records to 16 bytes)");
    if (int rc = cst::check_ws(ws, ws_bytes, sizeof(cst::WsHeader), CST_STR(CSTONE_FN(keys_records)))) return rc;
    return CST_NS::launch_keys_records(x, y, z, m, n, box, curve, reinterpret_cast<CST_NS::Key*>(keys),
                                       static_cast<cst::Record*>(records), ws, cst::as_stream(stream));
}

#ifndef CSTONE_KEY32  // the bounding cube and the batched entry points exist once, for 63-bit keys
int cstone_records_size(int64_t n, size_t* bytes) {
    if (!bytes || n < 0 || n >= CSTONE_MAX_PARTICLES)
        return cst::fail(CSTONE_ERR_INVALID_ARG, "cstone_records_size: bad argument");
    *bytes = static_cast<size_t>(n > 0 ? n : 1) * sizeof(cst::Record);
    return CSTONE_OK;
}

int cstone_keys_records_workspace_size(size_t* bytes) {
    if (!bytes) return cst::fail(CSTONE_ERR_INVALID_ARG, "cstone_keys_records_workspace_size: bad argument");
    *bytes = sizeof(cst::WsHeader);
    return CSTONE_OK;
}

int cstone_bbox_workspace_size(int64_t n, size_t* bytes) {
    if (!bytes || n < 0) return cst::fail(CSTONE_ERR_INVALID_ARG, "cstone_bbox_workspace_size: bad argument");
    *bytes = cst::bbox_ws_bytes();
    return CSTONE_OK;
}

int cstone_bbox(const double* x, const double* y, const double* z, int64_t n, double* box, void* ws, size_t ws_bytes,
                void* stream) {
    if (n < 0 || n >= CSTONE_MAX_PARTICLES || !box || (n > 0 && (!x || !y || !z)))
        return cst::fail(CSTONE_ERR_INVALID_ARG, "cstone_bbox: bad argument (n=%lld)", (long long)n);
    if (int rc = cst::check_ws(ws, ws_bytes, cst::bbox_ws_bytes(), "cstone_bbox")) return rc;
    return cst::launch_bbox(x, y, z, n, box, ws, cst::as_stream(stream));
}

int cstone_bounds(const double* x, const double* y, const double* z, int64_t n, double* bounds, void* ws,
                  size_t ws_bytes, void* stream) {
    if (n < 0 || n >= CSTONE_MAX_PARTICLES || !bounds || (n > 0 && (!x || !y || !z)))
        return cst::fail(CSTONE_ERR_INVALID_ARG, "cstone_bounds: bad argument (n=%lld)", (long long)n);
    if (int rc = cst::check_ws(ws, ws_bytes, cst::bbox_ws_bytes(), "cstone_bounds")) return rc;
    return cst::launch_bbox(x, y, z, n, bounds, ws, cst::as_stream(stream), true);
}

int cstone_bbox_batched(const double* x, const double* y, const double* z, const int64_t* set_offsets, int32_t n_sets,
                        double* boxes, void* stream) {
    if (n_sets < 1 || n_sets > (1 << 20) || !set_offsets || !boxes || !x || !y || !z)
        return cst::fail(CSTONE_ERR_INVALID_ARG, "cstone_bbox_batched: bad argument");
    return cst::launch_bbox_batched(x, y, z, reinterpret_cast<const long long*>(set_offsets), n_sets, boxes,
                                    cst::as_stream(stream));
}

int cstone_keys_batched_workspace_size(int32_t n_sets, size_t* bytes) {
    if (!bytes || n_sets < 1 || n_sets > (1 << 20))
        return cst::fail(CSTONE_ERR_INVALID_ARG, "cstone_keys_batched_workspace_size: bad argument");
    *bytes = cst::keys_batched_ws_bytes(n_sets);
    return CSTONE_OK;
}

int cstone_keys_batched(const double* x, const double* y, const double* z, int64_t n, const int64_t* set_offsets,
                        int32_t n_sets, const double* boxes, int curve, uint64_t* keys, void* ws, size_t ws_bytes,
                        void* stream) {
    if (n < 0 || n >= CSTONE_MAX_PARTICLES || n_sets < 1 || n_sets > (1 << 20) || !set_offsets || !boxes ||
        (n > 0 && (!x || !y || !z || !keys)))
        return cst::fail(CSTONE_ERR_INVALID_ARG, "cstone_keys_batched: bad argument");
    if (curve != CSTONE_MORTON && curve != CSTONE_HILBERT)
        return cst::fail(CSTONE_ERR_INVALID_ARG, "cstone_keys_batched: unknown curve %d", curve);
    if (int rc = cst::check_ws(ws, ws_bytes, cst::keys_batched_ws_bytes(n_sets), "cstone_keys_batched")) return rc;
    return cst::launch_keys_batched(x, y, z, reinterpret_cast<const long long*>(set_offsets), n_sets, n, boxes, curve,
                                    reinterpret_cast<cst::u64*>(keys), ws, cst::as_stream(stream));
}
#endif

}  // extern "C"
