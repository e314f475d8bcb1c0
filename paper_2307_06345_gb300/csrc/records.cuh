// Particle records of the multipole upsweep: coordinates in 64-bit fixed point and the mass,
// 32 bytes per particle in input order. Written by the pack step of the upsweep, or together with
// the keys by the record-writing key kernel (one read of the coordinates for both); read by the
// leaf sums through the sort permutation. Independent of the key length.
#pragma once

#include "common.cuh"

namespace cst {

// Coordinates in 64-bit fixed point: X = trunc(x * 2^F) with F chosen from the box so that
// |X| < 2^61 for |x| < 2^E >= max(|lo|, |lo + 2 side|). Differences of fixed-point values are
// exact; one conversion takes them to FP32 (int64_to_float below) and a power-of-two scale (split
// in two factors so that each is a normal float) restores physical units.
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

// FP32 value of a 64-bit integer. The direct 64-bit conversion runs at the FP64 rate on GB300
// (measured about 2 per SM and clock, against 30 for a 32-bit one), so the value is taken in its two
// 32-bit halves: exactly rounded where it fits 32 bits, otherwise hi * 2^32 + lo with one fused
// multiply-add, within 0.75 units in the last place for |d| < 2^56 and 1 unit above (where hi itself
// rounds).
__device__ __forceinline__ float int64_to_float(long long d) {
    const u32 lo = static_cast<u32>(static_cast<u64>(d));
    const int hi = static_cast<int>(d >> 32);
    const float wide = __fmaf_rn(__int2float_rn(hi), 4294967296.0f, __uint2float_rn(lo));
    return hi == (static_cast<int>(lo) >> 31) ? __int2float_rn(static_cast<int>(lo)) : wide;
}

// Nearest 64-bit integer of a float with |x| < 2^62, without the 64-bit conversion (the same
// result there): below 2^31 the 32-bit rounding; above, x is an integer, mantissa *
// 2^(exponent - 23). 0 for NaN and for |x| >= 2^62 (a zero-mass leaf's centre offset is NaN).
__device__ __forceinline__ long long float_to_int64(float x) {
    if (fabsf(x) < 2147483648.0f) return __float2int_rn(x);
    const u32 b = __float_as_uint(x);
    const int sh = static_cast<int>((b >> 23) & 0xffu) - 150;  // 8 <= sh <= 38 for 2^31 <= |x| < 2^62
    if (sh > 38) return 0;
    const long long mag = static_cast<long long>((b & 0x7fffffu) | 0x800000u) << sh;
    return (b >> 31) ? -mag : mag;
}

__device__ __forceinline__ float fixed_diff(long long a, long long b, const FixedFrame& f) {
    return __fmul_rn(__fmul_rn(int64_to_float(a - b), f.s1), f.s2);
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
