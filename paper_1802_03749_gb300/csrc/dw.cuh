// Double-word ("double-float") arithmetic on pairs of FP32 numbers.
//
// A value is hi + lo with |lo| <= ulp(hi)/2, about 48 significand bits.  The
// building blocks are the error-free transformations TwoSum (Knuth, TAOCP
// vol. 2, 4.2.2), FastTwoSum (Dekker, Numer. Math. 18, 1971) and the
// FMA-based exact product; addition and multiplication follow Joldes,
// Muller and Popescu, "Tight and rigorous error bounds for basic building
// blocks of double-word arithmetic", ACM TOMS 44(2), 2017:
//   dw_add  "AccurateDWPlusDW" (relative error < 3u^2, u = 2^-24)
//   dw_mul  "DWTimesDW" with FMA (relative error < 5u^2)
// The reciprocal is one Newton step on the FP32 reciprocal, done in
// double-word arithmetic (relative error of order u^2).
//
// GB300 executes FP32 at 128 FMA per clock per SM but FP64 at 2, so on
// this part double-word arithmetic on the FP32 pipes is the faster route to
// results accurate to ~1e-14 relative.  The __f*_rn intrinsics keep the
// compiler from contracting or reassociating the error-free transforms.
#pragma once
#include <cuda_runtime.h>

struct dw {
    float hi, lo;
};

__device__ __forceinline__ dw dw_two_sum(float a, float b)
{
    float s = __fadd_rn(a, b);
    float bb = __fsub_rn(s, a);
    float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
    return {s, e};
}

__device__ __forceinline__ dw dw_fast_two_sum(float a, float b)  // requires |a| >= |b| or a == 0
{
    float s = __fadd_rn(a, b);
    float e = __fsub_rn(b, __fsub_rn(s, a));
    return {s, e};
}

__device__ __forceinline__ dw dw_two_prod(float a, float b)
{
    float p = __fmul_rn(a, b);
    float e = __fmaf_rn(a, b, -p);
    return {p, e};
}

__device__ __forceinline__ dw dw_add(dw x, dw y)
{
    dw s = dw_two_sum(x.hi, y.hi);
    dw t = dw_two_sum(x.lo, y.lo);
    float c = __fadd_rn(s.lo, t.hi);
    dw v = dw_fast_two_sum(s.hi, c);
    float w = __fadd_rn(t.lo, v.lo);
    return dw_fast_two_sum(v.hi, w);
}

// "SloppyDWPlusDW" of the same paper: 11 operations instead of 20, with
// no relative error bound when x and y nearly cancel; used where measured
// accuracy on the mesh loops stays within the FP64 bar (~1.2e-13 rel-L2).
__device__ __forceinline__ dw dw_add_fast(dw x, dw y)
{
    dw s = dw_two_sum(x.hi, y.hi);
    float v = __fadd_rn(s.lo, __fadd_rn(x.lo, y.lo));
    return dw_fast_two_sum(s.hi, v);
}

__device__ __forceinline__ dw dw_neg(dw x) { return {-x.hi, -x.lo}; }

__device__ __forceinline__ dw dw_sub(dw x, dw y) { return dw_add(x, dw_neg(y)); }

__device__ __forceinline__ dw dw_mul(dw x, dw y)
{
    dw c = dw_two_prod(x.hi, y.hi);
    float t = __fmul_rn(x.hi, y.lo);
    float c2 = __fmaf_rn(x.lo, y.hi, t);
    float c3 = __fadd_rn(c.lo, c2);
    return dw_fast_two_sum(c.hi, c3);
}

// Compensated sums of double-word products (the Dot2 scheme of Ogita, Rump
// and Oishi, SIAM J. Sci. Comput. 26, 2005, with double-word factors): the
// products of the high parts are summed with TwoSum and all rounding
// errors (the exact product errors, the hi*lo cross terms and the TwoSum
// errors) accumulate in one float, added back at the end.  12 FP32
// operations per term instead of a product (8) and a sum (11).
struct dw_acc {
    float s, c;
};

__device__ __forceinline__ float dw_prod_err(dw a, dw b, float p)
{
    float e = __fmaf_rn(a.hi, b.hi, -p);
    e = __fmaf_rn(a.hi, b.lo, e);
    return __fmaf_rn(a.lo, b.hi, e);
}

__device__ __forceinline__ dw_acc dw_dot_begin(dw a, dw b)
{
    float p = __fmul_rn(a.hi, b.hi);
    return {p, dw_prod_err(a, b, p)};
}

__device__ __forceinline__ void dw_dot_add(dw_acc &A, dw a, dw b)
{
    float p = __fmul_rn(a.hi, b.hi);
    float e = dw_prod_err(a, b, p);
    dw t = dw_two_sum(A.s, p);
    A.s = t.hi;
    A.c = __fadd_rn(A.c, __fadd_rn(t.lo, e));
}

__device__ __forceinline__ dw dw_dot_end(dw_acc A) { return dw_fast_two_sum(A.s, A.c); }

// Compensated sum of double-words (the Sum2 scheme of the same paper with
// double-word terms): the high parts are summed with TwoSum, the TwoSum
// errors and the low parts gathered in one float, added back with TwoSum
// at the end (the sum may cancel, so FastTwoSum's ordering is not assumed).
// The term is sg * x for sg in {-1, 0, 1}: the products are exact, so the
// FMAs below round exactly where TwoSum of (S.s, sg x.hi) would.  8 FP32
// operations per term instead of 11 for a sloppy double-word addition.
__device__ __forceinline__ void dw_sum_add(dw_acc &S, dw x, float sg)
{
    const float s = __fmaf_rn(sg, x.hi, S.s);
    const float bb = __fsub_rn(s, S.s);
    const float e = __fadd_rn(__fsub_rn(S.s, __fsub_rn(s, bb)), __fmaf_rn(sg, x.hi, -bb));
    S.s = s;
    S.c = __fadd_rn(S.c, __fmaf_rn(sg, x.lo, e));
}

__device__ __forceinline__ dw dw_sum_end(dw_acc S) { return dw_two_sum(S.s, S.c); }

// x * 2^k for a power of two (exact)
__device__ __forceinline__ dw dw_scale2(dw x, float p2) { return {__fmul_rn(x.hi, p2), __fmul_rn(x.lo, p2)}; }

// 1/x: Newton step y = y0 + y0 (1 - x y0) from the FP32 reciprocal y0
__device__ __forceinline__ dw dw_recip(dw x)
{
    float y0 = __frcp_rn(x.hi);
    dw p = dw_mul(x, dw{y0, 0.0f});
    dw e = dw_sub(dw{1.0f, 0.0f}, p);
    dw t = dw_mul(dw{y0, 0.0f}, e);
    return dw_add(dw{y0, 0.0f}, t);
}

// The same Newton step with the sloppy additions: 1 - x y0 is computed
// exactly by them (TwoSum of 1 and the high part is exact by Sterbenz's
// lemma, then one rounding of the low part), and y0 + t adds a term 2^24
// times smaller, so neither addition can cancel.
__device__ __forceinline__ dw dw_recip_fast(dw x)
{
    float y0 = __frcp_rn(x.hi);
    dw p = dw_mul(x, dw{y0, 0.0f});
    dw e = dw_add_fast(dw{1.0f, 0.0f}, dw_neg(p));
    dw t = dw_mul(dw{y0, 0.0f}, e);
    return dw_add_fast(dw{y0, 0.0f}, t);
}

// Nearest double-word of a double: hi = fl32(d), lo = fl32(d - hi), using
// the FP64 unit (conversion and subtraction).
__device__ __forceinline__ dw dw_from_double(double d)
{
    float h = __double2float_rn(d);
    float l = __double2float_rn(d - (double)h);
    return {h, l};
}

__device__ __forceinline__ double dw_to_double(dw x) { return (double)x.hi + (double)x.lo; }

// On GB300 the FP64 <-> FP32 conversion instructions run on the FP64 unit
// (about 2 per clock per SM), so the splits below use integer operations.
//
// Double-word of a double by bit manipulation: hi takes the sign, the
// exponent and the top 23 stored significand bits (truncation, exact in
// FP32); the remaining 29 bits r give lo = r * 2^(e-1075), r rounded to 24
// bits by the integer-to-float conversion.  The pair is renormalised with
// FastTwoSum.  Relative error at most 2^-47.  Zeros, values below 2^-74 or
// above the FP32 range take the exact FP64 route.
// The rare cases are kept out of line so that the compiler branches around
// them instead of evaluating their conversions on every call.
static __device__ __noinline__ dw dw_from_double_slow(double d) { return dw_from_double(d); }
static __device__ __noinline__ double f32_to_f64_slow(float f) { return (double)f; }

__device__ __forceinline__ dw dw_from_double_int(double d)
{
    // the halves are moved out opaquely so that the compiler keeps the
    // exponent test in integer arithmetic instead of an FP64 comparison
    unsigned lo32, hi32;
    asm("mov.b64 {%0, %1}, %2;" : "=r"(lo32), "=r"(hi32) : "d"(d));
    const unsigned e = (hi32 >> 20) & 0x7ffu;
    if (e - 949u > 1150u - 949u) return dw_from_double_slow(d);  // zero, tiny, huge, inf, nan
    // (hi32:lo32) << 3 puts the low 9 exponent bits at 23..31 above the top
    // 23 significand bits; subtracting 896 << 23 modulo 2^32 leaves the
    // FP32 exponent e - 896 (53..254 here, so bit 31 ends up clear)
    const unsigned sign = hi32 & 0x80000000u;
    const unsigned hb = (__funnelshift_l(lo32, hi32, 3) - (896u << 23)) | sign;
    const float h = __uint_as_float(hb);
    // 2^(e - 948) with the sign: h's exponent lowered by 52
    const float scale = __uint_as_float(((hb & 0xff800000u) - (52u << 23)));
    const float l = __fmul_rn(__int2float_rn((int)(lo32 & 0x1fffffffu)), scale);
    return dw_fast_two_sum(h, l);
}

// Exact FP32 -> FP64 widening by bit manipulation (normal numbers and
// zeros); subnormals, infinities and NaNs take the conversion instruction.
__device__ __forceinline__ double f32_to_f64_int(float f)
{
    const unsigned u = __float_as_uint(f);
    const unsigned e = (u >> 23) & 0xffu;
    const bool zero = (u << 1) == 0u;
    if (!zero && (e == 0 || e == 255)) return f32_to_f64_slow(f);
    const unsigned long long sign = (unsigned long long)(u & 0x80000000u) << 32;
    const unsigned long long mag = ((unsigned long long)(e + 896) << 52) | ((unsigned long long)(u & 0x7fffffu) << 29);
    return __longlong_as_double((long long)(sign | (zero ? 0ull : mag)));
}

// a + x for a double a and a double-word x, rounded once per FP64 addition:
// (a + hi) + lo with both halves widened exactly.
__device__ __forceinline__ double f64_add_dw(double a, dw x)
{
    return (a + f32_to_f64_int(x.hi)) + f32_to_f64_int(x.lo);
}
