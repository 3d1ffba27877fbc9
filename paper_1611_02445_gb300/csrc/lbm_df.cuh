// lbm_df.cuh -- double-float arithmetic: a value is the unevaluated sum hi + lo of two
// FP32 numbers (about 48 significant bits).
//
// The error-free transformations are Knuth's TwoSum and Dekker's FastTwoSum for sums and
// the FMA form of Dekker's TwoProduct (Dekker, "A floating-point technique for extending
// the available precision", Numer. Math. 18, 1971; Knuth, TAOCP vol. 2, 4.2.2). Every
// FP32 operation here is written with an explicit round-to-nearest intrinsic, so the
// compiler cannot contract or reassociate it.
//
// Pairs need not be normalised (|lo| may exceed half an ulp of hi): the step uses them
// for quantities bounded by the lattice weights, where an absolute error of about
// 2^-48 is what matters.
#pragma once
#include <stdint.h>

#if defined(__CUDA_ARCH__)
#define LBM_DF_HD __device__ __forceinline__
#define LBM_FADD(a, b) __fadd_rn((a), (b))
#define LBM_FSUB(a, b) __fsub_rn((a), (b))
#define LBM_FMUL(a, b) __fmul_rn((a), (b))
#define LBM_FFMA(a, b, c) __fmaf_rn((a), (b), (c))
#else
#include <cmath>
#include <cstring>
#define LBM_DF_HD static inline
#define LBM_FADD(a, b) ((a) + (b))
#define LBM_FSUB(a, b) ((a) - (b))
#define LBM_FMUL(a, b) ((a) * (b))
#define LBM_FFMA(a, b, c) std::fma((float)(a), (float)(b), (float)(c))
#endif

namespace lbm {

struct dfl {
    float h, l;
};

LBM_DF_HD dfl df_make(float h, float l) {
    dfl r;
    r.h = h;
    r.l = l;
    return r;
}

// a + b = s + e exactly (6 operations)
LBM_DF_HD dfl two_sum(float a, float b) {
    const float s = LBM_FADD(a, b);
    const float bb = LBM_FSUB(s, a);
    const float e = LBM_FADD(LBM_FSUB(a, LBM_FSUB(s, bb)), LBM_FSUB(b, bb));
    return df_make(s, e);
}
// a * b = p + e exactly (2 operations)
LBM_DF_HD dfl two_prod(float a, float b) {
    const float p = LBM_FMUL(a, b);
    return df_make(p, LBM_FFMA(a, b, -p));
}
LBM_DF_HD dfl df_neg(dfl x) { return df_make(-x.h, -x.l); }
LBM_DF_HD dfl df_add(dfl x, dfl y) {
    const dfl s = two_sum(x.h, y.h);
    return df_make(s.h, LBM_FADD(s.l, LBM_FADD(x.l, y.l)));
}
// a + b = s + e exactly when |a| >= |b| (Dekker's FastTwoSum, 3 operations)
LBM_DF_HD dfl fast_two_sum(float a, float b) {
    const float s = LBM_FADD(a, b);
    return df_make(s, LBM_FSUB(b, LBM_FSUB(s, a)));
}
// x + y for |x.h| >= |y.h|: the same result as df_add at 5 operations instead of 8
LBM_DF_HD dfl df_add_dom(dfl x, dfl y) {
    const dfl s = fast_two_sum(x.h, y.h);
    return df_make(s.h, LBM_FADD(s.l, LBM_FADD(x.l, y.l)));
}
LBM_DF_HD dfl df_sub_dom(dfl x, dfl y) { return df_add_dom(x, df_neg(y)); }
LBM_DF_HD dfl df_sub(dfl x, dfl y) { return df_add(x, df_neg(y)); }
// The lo * lo term is kept: dropping it biases products of correlated operands.
LBM_DF_HD dfl df_mul(dfl x, dfl y) {
    dfl p = two_prod(x.h, y.h);
    p.l = LBM_FFMA(x.h, y.l, LBM_FFMA(x.l, y.h, LBM_FFMA(x.l, y.l, p.l)));
    return p;
}
// product with an FP32 number
LBM_DF_HD dfl df_mulf(dfl x, float y) {
    dfl p = two_prod(x.h, y);
    p.l = LBM_FFMA(x.l, y, p.l);
    return p;
}
// product with a power of two: exact
LBM_DF_HD dfl df_scale2(dfl x, float pow2) { return df_make(LBM_FMUL(x.h, pow2), LBM_FMUL(x.l, pow2)); }
LBM_DF_HD dfl df_norm(dfl x) { return two_sum(x.h, x.l); }

// 1/x for x near 1 (a density): FP32 reciprocal, then one Newton step in double-float.
LBM_DF_HD dfl df_recip(dfl x) {
#if defined(__CUDA_ARCH__)
    const float r0 = __frcp_rn(x.h);
#else
    const float r0 = 1.0f / x.h;
#endif
    // e = 1 - x r0, formed from the exact product x.h r0 = p + pe (p close to 1)
    const dfl p = two_prod(x.h, r0);
    const float e = LBM_FSUB(LBM_FSUB(LBM_FSUB(1.0f, p.h), p.l), LBM_FMUL(x.l, r0));
    // r = r0 / (1 - e) = r0 (1 + e + e^2 + ...); the e^2 term is kept because it is
    // always positive and would otherwise bias every reciprocal low
    return df_make(r0, LBM_FMUL(r0, LBM_FFMA(e, e, e)));
}

// ------------------------------------------------------------------ FP64 <-> pairs
// Bit-level conversions that use no FP64 instruction.
LBM_DF_HD uint64_t bits_of(double d) {
#if defined(__CUDA_ARCH__)
    return (uint64_t)__double_as_longlong(d);
#else
    uint64_t u;
    std::memcpy(&u, &d, 8);
    return u;
#endif
}
LBM_DF_HD double double_of(uint64_t u) {
#if defined(__CUDA_ARCH__)
    return __longlong_as_double((long long)u);
#else
    double d;
    std::memcpy(&d, &u, 8);
    return d;
#endif
}
LBM_DF_HD float float_of(uint32_t u) {
#if defined(__CUDA_ARCH__)
    return __uint_as_float(u);
#else
    float f;
    std::memcpy(&f, &u, 4);
    return f;
#endif
}
LBM_DF_HD uint32_t fbits_of(float f) {
#if defined(__CUDA_ARCH__)
    return __float_as_uint(f);
#else
    uint32_t u;
    std::memcpy(&u, &f, 4);
    return u;
#endif
}

// d = hi + lo with hi the truncation of d to FP32 and lo the rest rounded to FP32;
// |d - hi - lo| <= 2^-48 |d|. Valid for 2^-60 <= |d| < 2; smaller values become 0.
LBM_DF_HD dfl df_from_double(double d) {
    const uint64_t b = bits_of(d);
    const uint32_t H = (uint32_t)(b >> 32), L = (uint32_t)b;
    if ((H & 0x7ff00000u) < (963u << 20)) return df_make(0.0f, 0.0f);   // |d| < 2^-60
    // (H << 3 | L >> 29) holds the low 9 exponent bits and the top 23 fraction bits;
    // rebias the exponent from 1023 to 127 (for |d| < 2 the 9-bit field is E - 512)
    const uint32_t a = (H << 3) | (L >> 29);
    const uint32_t hb = (a - (384u << 23)) | (H & 0x80000000u);
    // remaining 29 fraction bits, scaled by 2^(E - 1075) = 2^(E_f - 52 - 127) with sign
    const uint32_t sb = (hb & 0xff800000u) - (52u << 23);
    const float lo = LBM_FMUL((float)(L & 0x1fffffffu), float_of(sb));
    return df_make(float_of(hb), lo);
}

// Nearest double to hi + lo for a positive value in [2^-40, 2) (the pair need not be
// normalised, but |lo| must stay below hi/2^20): normalise with FastTwoSum, widen hi
// exactly, count lo in units of the double's last place and add the count to hi's bit
// pattern. When lo is negative the count is taken in the last place of the float just
// below hi, which differs from hi's own only when hi is a power of two and the result
// lies in the binade below, where the last place is half as large.
LBM_DF_HD double df_to_double_pos(dfl x) {
    const float s = LBM_FADD(x.h, x.l);
    const float l = LBM_FSUB(x.l, LBM_FSUB(s, x.h));
    const uint32_t hb = fbits_of(s);
    const uint64_t hi64 = ((uint64_t)((hb >> 3) + (896u << 20)) << 32) | (uint64_t)(hb << 29);
    // ulp of the double = 2^(E_f - 127 - 52); scale lo by its inverse 2^(179 - E_f), with
    // E_f the exponent of s, or of the float below s when lo is negative
    const uint32_t sb = (306u << 23) - ((hb - (fbits_of(l) >> 31)) & 0x7f800000u);
    const float q = LBM_FMUL(l, float_of(sb));
#if defined(__CUDA_ARCH__)
    const int k = __float2int_rn(q);
#else
    const int k = (int)std::nearbyint(q);
#endif
    return double_of(hi64 + (uint64_t)(int64_t)k);
}

// ------------------------------------------------------------ 64-bit fixed point
// Populations as integers in units of 2^-58 (|d| < 32): sums of them are exact.
constexpr int FIX_SHIFT = 58;

// d * 2^58 rounded to nearest (ties away from zero), from the bit pattern (no FP64
// instruction). Rounding, not truncation, keeps sums of many conversions unbiased.
LBM_DF_HD int64_t fix_from_double(double d) {
    const uint64_t b = bits_of(d);
    const int E = (int)((b >> 52) & 0x7ffu);
    const uint64_t m = (b & 0x000fffffffffffffull) | 0x0010000000000000ull;
    const int s = E - (1075 - FIX_SHIFT);            // value = m * 2^(E - 1075)
    uint64_t v;
    if (s >= 0) {
        v = m << (s > 10 ? 10 : s);                  // |d| < 32 keeps s <= 9
    } else {
        const int r = s < -62 ? 62 : -s;
        v = (m + (1ull << (r - 1))) >> r;
    }
    if (E == 0) v = 0;
    const int64_t r = (int64_t)v;
    return (b >> 63) ? -r : r;
}

// d * 2^58 for 2^-6 <= d < 16, where it is an integer: the 53-bit significand shifted
// left by E - 1017 (0 to 9), with E the biased exponent. Six integer instructions, no FP64
// pipe. Any other input (negative, below 2^-6, 16 or more, zero, not finite) sets `bad`
// and returns an unspecified value; the caller then converts another way. Where this one
// is valid the value is exact, so fix_from_double and fix_from_double_cvt give the same.
LBM_DF_HD int64_t fix_from_double_fast(double d, bool& bad) {
    const uint64_t b = bits_of(d);
    const uint32_t hi = (uint32_t)(b >> 32), lo = (uint32_t)b;
    const uint32_t s = (hi >> 20) - 1017u;   // the sign bit makes s large for negative d
    bad |= s > 9u;
    const uint32_t mh = (hi & 0x000fffffu) | 0x00100000u;
#if defined(__CUDA_ARCH__)
    const uint32_t rh = __funnelshift_l(lo, mh, s);
    const uint32_t rl = lo << (s & 31u);
#else
    const uint32_t rh = (uint32_t)(((((uint64_t)mh << 32) | lo) << (s & 15u)) >> 32);
    const uint32_t rl = lo << (s & 15u);
#endif
    return (int64_t)(((uint64_t)rh << 32) | rl);
}

// d * 2^58 rounded to the nearest integer, ties to even, for normal |d| < 32 (zero and
// subnormals give 0): the scaling adds 58 to the exponent field with one integer add,
// and one conversion on the FP64 pipe rounds. Two instructions and one FP64-pipe
// operation, which GB300 issues at 2 lanes per SM and clock; the step's fallback for
// populations outside the range of fix_from_double_fast. Sums of these stay exact, only
// ties round the other way than in fix_from_double.
LBM_DF_HD int64_t fix_from_double_cvt(double d) {
    const double x = double_of(bits_of(d) + ((uint64_t)FIX_SHIFT << 52));
#if defined(__CUDA_ARCH__)
    return __double2ll_rn(x);
#else
    return (int64_t)std::nearbyint(x);
#endif
}

// Double-float of x * 2^-58 (relative error below 2^-48), from three pieces that each
// convert to FP32 exactly: x = t 2^41 + r1 2^18 + r0 with t = floor(x / 2^41) (|t| <= 2^22),
// 0 <= r1 < 2^23 and 0 <= r0 < 2^18. A piece p becomes a float by the 2^23 magic-number
// trick (the bit pattern of 2^23 + p, or 1.5 * 2^23 + t for the signed piece, minus that
// constant), so no 64-bit integer conversion is executed: GB300 runs those on its 2-lane
// FP64 pipe, where they took a third of the step's FP64 instructions.
static_assert(FIX_SHIFT == 58, "df_from_fix splits x for 2^-58 fixed point");
LBM_DF_HD dfl df_from_fix(int64_t x) {
    const int32_t t = (int32_t)(x >> 41);
    const uint32_t r1 = (uint32_t)(x >> 18) & 0x7fffffu;
    const uint32_t r0 = (uint32_t)x & 0x3ffffu;
    const float tf = LBM_FSUB(float_of(0x4B400000u + (uint32_t)t), 12582912.0f);
    const float r1f = LBM_FSUB(float_of(0x4B000000u | r1), 8388608.0f);
    const float r0f = LBM_FSUB(float_of(0x4B000000u | r0), 8388608.0f);
    // t 2^-17 + r1 2^-40 exactly as a pair, then the last piece (below 2^-40) into its low part
    const dfl s = two_sum(LBM_FMUL(tf, 0x1p-17f), LBM_FMUL(r1f, 0x1p-40f));
    return df_make(s.h, LBM_FADD(s.l, LBM_FMUL(r0f, 0x1p-58f)));
}

}  // namespace lbm
