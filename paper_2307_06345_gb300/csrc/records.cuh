// Particle records of the multipole upsweep: coordinates in 64-bit fixed point and the mass,
// 32 bytes per particle in input order. Written by the pack step of the upsweep, or together with
// the keys by the record-writing key kernel (one read of the coordinates for both); read by the
// leaf sums through the sort permutation. Independent of the key length.
#pragma once

#include "common.cuh"

namespace cst {

// Coordinates in 64-bit fixed point: X = trunc(x * 2^F) with F chosen from the box so that
// |X| < 2^61 for |x| < 2^E >= max(|lo|, |lo + 2 side|). Differences of fixed-point values are
// exact; one conversion rounds them to FP32 and a power-of-two scale (split in two factors so
// that each is a normal float) restores physical units.
struct FixedFrame {
    int F;
    float s1, s2;  // 2^-F = s1 * s2
    int e_lim;     // biased exponent bound: |x| < 2^(e_lim - 1023)
};

__device__ __forceinline__ float pow2f(int k) { return __int_as_float((k + 127) << 23); }

__device__ inline FixedFrame make_frame(const double* box) {
    FixedFrame f;
    const double lo0 = fmin(fmin(box[0], box[1]), box[2]);
    const double lo1 = fmax(fmax(box[0], box[1]), box[2]);
    const double hi = __dadd_rn(lo1, __dmul_rn(2.0, box[3]));
    const double big = fmax(fabs(lo0), fmax(fabs(lo1), fabs(hi)));
    const int e = static_cast<int>((static_cast<u64>(__double_as_longlong(big)) >> 52) & 0x7ffu);
    const int E = e - 1023 + 1;  // 2^E > big
    f.F = 61 - E;
    f.e_lim = E + 1023;
    const int h = f.F / 2;
    f.s1 = pow2f(-h);
    f.s2 = pow2f(-(f.F - h));
    return f;
}

__device__ __forceinline__ long long fixed_of(double x, int F) {
    const u64 b = static_cast<u64>(__double_as_longlong(x));
    const int e = static_cast<int>((b >> 52) & 0x7ffu);
    u64 mant = b & ((1ULL << 52) - 1);
    if (e != 0) mant |= (1ULL << 52);
    const int sh = (e == 0 ? 1 : e) - 1075 + F;
    const u64 mag = sh >= 0 ? (mant << sh) : (sh > -64 ? (mant >> (-sh)) : 0ULL);
    return (b >> 63) ? -static_cast<long long>(mag) : static_cast<long long>(mag);
}

__device__ __forceinline__ float fixed_diff(long long a, long long b, const FixedFrame& f) {
    return __fmul_rn(__fmul_rn(__ll2float_rn(a - b), f.s1), f.s2);
}

__device__ __forceinline__ double fixed_to_double(long long a, const FixedFrame& f) {
    // exact power-of-two scaling of the (rounded) conversion
    return __dmul_rn(__dmul_rn(__ll2double_rn(a), (double)f.s1), (double)f.s2);
}

struct __align__(16) Record {  // one particle, original order
    long long x, y, z;
    float m;
    u32 pad;
};


// The record of one particle, written as two 16-byte streaming stores. A coordinate outside the
// fixed-point range of the frame gives a zero position and false (the caller records the error).
__device__ __forceinline__ bool store_record(Record* rec, u32 p, double px, double py, double pz, float pm,
                                             const FixedFrame& f) {
    const int ex = static_cast<int>((static_cast<u64>(__double_as_longlong(px)) >> 52) & 0x7ffu);
    const int ey = static_cast<int>((static_cast<u64>(__double_as_longlong(py)) >> 52) & 0x7ffu);
    const int ez = static_cast<int>((static_cast<u64>(__double_as_longlong(pz)) >> 52) & 0x7ffu);
    const bool ok = max(ex, max(ey, ez)) < f.e_lim;
    const long long X = ok ? fixed_of(px, f.F) : 0, Y = ok ? fixed_of(py, f.F) : 0, Z = ok ? fixed_of(pz, f.F) : 0;
    longlong2* dst = reinterpret_cast<longlong2*>(rec + p);
    __stcs(dst, make_longlong2(X, Y));
    __stcs(dst + 1, make_longlong2(Z, static_cast<long long>(__float_as_uint(pm))));
    return ok;
}

}  // namespace cst
