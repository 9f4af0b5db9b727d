// Compensated float32 ("double-float") helpers for the float64 parts of the
// refinement.  GB300 runs FP64 arithmetic, and conversions between float
// and double, at about 1/64 of its FP32 rate (measured: one warp
// instruction per 64-82 cycles per warp), so float64 values are split into
// float pairs by integer operations on their bit patterns and products are
// summed with error-free transformations in float32:
//   a = a_hi + a_lo (+ |d| <= 2^-47 |a|), a_hi and a_lo truncations
//   a b ~ a_hi b_hi + (a_hi b_lo + a_lo b_hi), a_hi b_hi = p + e exactly (FMA)
//   (s, c) <- TwoSum(s, p) with the error, e and the cross terms into c.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace lobpcg {

// Exact float -> double on the bit pattern (float32 zeros and denormals,
// below 2^-126, give 0).
__device__ __forceinline__ double df_to_f64(float f) {
    const unsigned u = __float_as_uint(f);
    const unsigned e = (u >> 23) & 0xffu;
    if (e == 0) return 0.0;
    const unsigned hi = (u & 0x80000000u) | ((e - 127u + 1023u) << 20) | ((u & 0x7fffffu) >> 3);
    return __hiloint2double(static_cast<int>(hi), static_cast<int>((u & 7u) << 29));
}

// z = hi + lo + d, |d| < 2^-47 |z|: hi = z with its significand cut to 24
// bits, lo = the rest cut to 24 bits.  |z| below 2^-126 gives 0 (and its
// lo part below 2^-126 is dropped); |z| of 2^128 or more takes the slow
// conversion (not met by the blocks this is used on).
__device__ __forceinline__ void df_split(double z, float &hi, float &lo) {
    const unsigned long long b = static_cast<unsigned long long>(__double_as_longlong(z));
    const int E = static_cast<int>((b >> 52) & 0x7ff) - 1023;
    const unsigned sgn = static_cast<unsigned>(b >> 32) & 0x80000000u;
    if (E < -126) {
        hi = lo = 0.f;
        return;
    }
    if (E > 127) {
        hi = __double2float_rn(z);
        lo = 0.f;
        return;
    }
    const unsigned long long m = b & 0xFFFFFFFFFFFFFull;   // 52 fraction bits
    hi = __uint_as_float(sgn | (static_cast<unsigned>(E + 127) << 23) | static_cast<unsigned>(m >> 29));
    const unsigned long long L = m & ((1ull << 29) - 1);   // the rest: L 2^(E - 52)
    const int p = 63 - __clzll(static_cast<long long>(L));  // leading one of L (L = 0: -1)
    const int El = E - 52 + p;
    if (L == 0 || El < -126) {
        lo = 0.f;
        return;
    }
    const unsigned mant = (p >= 23) ? static_cast<unsigned>(L >> (p - 23)) : static_cast<unsigned>(L << (23 - p));
    lo = __uint_as_float(sgn | (static_cast<unsigned>(El + 127) << 23) | (mant & 0x7fffffu));
}

// (s, c) += (ah + al)(bh + bl); the intrinsics keep the compiler from
// contracting or reassociating the error-free steps
__device__ __forceinline__ void df_mac(float ah, float al, float bh, float bl, float &s, float &c) {
    const float p = __fmul_rn(ah, bh);
    const float e = __fmaf_rn(ah, bh, -p);
    const float x = __fmaf_rn(ah, bl, __fmul_rn(al, bh));
    const float sn = __fadd_rn(s, p);
    const float bp = __fsub_rn(sn, s);
    const float t = __fadd_rn(__fsub_rn(s, __fsub_rn(sn, bp)), __fsub_rn(p, bp));
    s = sn;
    c = __fadd_rn(c, __fadd_rn(t, __fadd_rn(e, x)));
}

// Packed pairs (f32x2 instructions; each half rounds to nearest as its
// scalar counterpart, and the explicit rounding mode keeps the compiler from
// contracting them).
#define LOBPCG_DF2_OP(name, op)                                                       \
    __device__ __forceinline__ float2 name(float2 a, float2 b) {                      \
        float2 r;                                                                     \
        asm("{\n\t.reg .b64 ra, rb, rd;\n\t"                                          \
            "mov.b64 ra, {%2, %3};\n\t"                                               \
            "mov.b64 rb, {%4, %5};\n\t" op " rd, ra, rb;\n\t"                        \
            "mov.b64 {%0, %1}, rd;\n\t}"                                              \
            : "=f"(r.x), "=f"(r.y)                                                    \
            : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));                                \
        return r;                                                                     \
    }
LOBPCG_DF2_OP(df2_add, "add.rn.f32x2")
LOBPCG_DF2_OP(df2_sub, "sub.rn.f32x2")
LOBPCG_DF2_OP(df2_mul, "mul.rn.f32x2")
#undef LOBPCG_DF2_OP
__device__ __forceinline__ float2 df2_fma(float2 a, float2 b, float2 c) {
    float2 r;
    asm("{\n\t.reg .b64 ra, rb, rc;\n\t"
        "mov.b64 ra, {%2, %3};\n\t"
        "mov.b64 rb, {%4, %5};\n\t"
        "mov.b64 rc, {%6, %7};\n\t"
        "fma.rn.f32x2 rc, ra, rb, rc;\n\t"
        "mov.b64 {%0, %1}, rc;\n\t}"
        : "=f"(r.x), "=f"(r.y)
        : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y), "f"(c.x), "f"(c.y));
    return r;
}

// df_mac on two independent pairs at once: (s, c) += (ah + al)(bh + bl)
// per half, nbh = -bh.  Same steps as df_mac with q = -p: e = ah bh + q
// exactly, TwoSum(s, -q) = (s - q, (s - (sn - bp)) - (q + bp)); each half
// gives the bits df_mac gives.
__device__ __forceinline__ void df_mac2(float2 ah, float2 al, float2 bh, float2 nbh, float2 bl, float2 &s,
                                        float2 &c) {
    const float2 q = df2_mul(ah, nbh);
    const float2 e = df2_fma(ah, bh, q);
    const float2 x = df2_fma(ah, bl, df2_mul(al, bh));
    const float2 sn = df2_sub(s, q);
    const float2 bp = df2_sub(sn, s);
    const float2 t = df2_sub(df2_sub(s, df2_sub(sn, bp)), df2_add(q, bp));
    s = sn;
    c = df2_add(c, df2_add(t, df2_add(e, x)));
}

}  // namespace lobpcg
