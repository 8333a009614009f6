// Double-float ("FP32 pair") arithmetic for the density exponentials.
//
// GB300 runs FP32 FMAs at about 64x its FP64 rate, so a value held as an unevaluated
// sum hi + lo of two floats (about 44-48 significant bits) is far cheaper than FP64
// while keeping the density's relative error near 1e-13 -- five orders of magnitude
// below what the 1e-8 sphere-coefficient tolerance needs.
//
// Building blocks (published error-free transformations):
//   two_sum       Knuth (TAOCP vol. 2, 4.2.2): s + e == a + b exactly
//   fast_two_sum  Dekker (1971), requires |a| >= |b|
//   two_prod      with a fused multiply-add: p + e == a * b exactly
// The double-word add / multiply follow the "sloppy" variants analysed by Joldes,
// Muller and Popescu (ACM TOMS 2017); every sum here adds quantities of one sign or
// with bounded cancellation.  exp uses Tang's table-driven reduction
// t = k ln2/64 + f, |f| <= ln2/128, e^-t = 2^(-k/64) e^-f, with a Taylor tail in f.
#pragma once

#include <cuda_runtime.h>

namespace lasto {
namespace dfa {

struct df {
    float h, l;
};

__device__ __forceinline__ df two_sum(float a, float b)
{
    const float s = a + b;
    const float bb = s - a;
    const float e = (a - (s - bb)) + (b - bb);
    return {s, e};
}

__device__ __forceinline__ df fast_two_sum(float a, float b)
{
    const float s = a + b;
    return {s, b - (s - a)};
}

__device__ __forceinline__ df two_prod(float a, float b)
{
    const float p = a * b;
    return {p, fmaf(a, b, -p)};
}

__device__ __forceinline__ df from_double(double x)
{
    const float h = __double2float_rn(x);
    return {h, __double2float_rn(x - (double)h)};
}

__device__ __forceinline__ double to_double(df a) { return (double)a.h + (double)a.l; }

__device__ __forceinline__ df add(df a, df b)
{
    df s = two_sum(a.h, b.h);
    s.l += a.l + b.l;
    return fast_two_sum(s.h, s.l);
}

__device__ __forceinline__ df add_f(df a, float b)
{
    df s = two_sum(a.h, b);
    s.l += a.l;
    return fast_two_sum(s.h, s.l);
}

__device__ __forceinline__ df neg(df a) { return {-a.h, -a.l}; }

__device__ __forceinline__ df mul(df a, df b)
{
    df p = two_prod(a.h, b.h);
    p.l = fmaf(a.h, b.l, p.l);
    p.l = fmaf(a.l, b.h, p.l);
    return fast_two_sum(p.h, p.l);
}

__device__ __forceinline__ df mul_f(df a, float b)
{
    df p = two_prod(a.h, b);
    p.l = fmaf(a.l, b, p.l);
    return fast_two_sum(p.h, p.l);
}

__device__ __forceinline__ df sqr(df a)
{
    df p = two_prod(a.h, a.h);
    p.l = fmaf(2.0f * a.h, a.l, p.l);
    return fast_two_sum(p.h, p.l);
}

// sqrt by one Newton correction of the FP32 root: s + (a - s^2) / (2 s)
__device__ __forceinline__ df sqrt_df(df a)
{
    if (a.h <= 0.0f) return {0.0f, 0.0f};
    const float s = sqrtf(a.h);
    const df p = two_prod(s, s);
    const float r = ((a.h - p.h) - p.l) + a.l;
    return fast_two_sum(s, r * (0.5f / s));
}

// a / b: FP32 quotient plus one correction with the exact remainder
__device__ __forceinline__ df div(df a, df b)
{
    const float q1 = a.h / b.h;
    const df r = add(a, neg(mul_f(b, q1)));
    const float q2 = r.h / b.h;
    return fast_two_sum(q1, q2);
}

// Table of 2^(-j/64), j = 0..63, as double-floats (filled by the host).
struct ExpTable {
    float h[64], l[64];
};

// e^{-t} for |t| <= 80.  ln2/64 is split as c1 + c2 + c3 with c1 carrying 11 bits so
// that k * c1 is exact for |k| < 8192; t - k c1 is then exact by Sterbenz's lemma.
__device__ __forceinline__ df exp_neg(df t, const float* __restrict__ th, const float* __restrict__ tl)
{
    constexpr float INV_C = 92.33248138427734f;           // 64 / ln 2
    constexpr float C1 = 0.010833740234375f;              // ln2/64 rounded to 11 bits (1420 / 2^17)
    constexpr float C2 = -3.3155381515825866e-06f;        // next 24 bits
    constexpr float C3 = 2.5727683872212026e-14f;         // remainder
    const int k = __float2int_rn(t.h * INV_C);
    const float kf = (float)k;
    const float a = fmaf(-kf, C1, t.h);                   // exact
    const df p2 = two_prod(kf, C2);
    df f = two_sum(a, -p2.h);
    f.l += t.l - fmaf(kf, C3, p2.l);
    f = fast_two_sum(f.h, f.l);
    // e^{-f} = 1 - f + f^2/2 - f^3/6 + f^4/24 - f^5/120, |f| <= 0.0055
    const float fh = f.h;
    const float tail = fh * fh * fh * fmaf(fh, fmaf(fh, -1.0f / 120.0f, 1.0f / 24.0f), -1.0f / 6.0f);
    df e = two_sum(1.0f, -f.h);
    e.l -= f.l;
    e = fast_two_sum(e.h, e.l);
    df f2 = sqr(f);
    f2.h *= 0.5f;
    f2.l *= 0.5f;
    e = add(e, f2);
    e = add_f(e, tail);
    const int j = k & 63, q = k >> 6;                     // k = 64 q + j, 0 <= j < 64
    e = mul(e, df{th[j], tl[j]});
    const float sc = __int_as_float((127 - q) << 23);     // 2^{-q}, |q| <= 126
    return {e.h * sc, e.l * sc};
}

}  // namespace dfa
}  // namespace lasto
