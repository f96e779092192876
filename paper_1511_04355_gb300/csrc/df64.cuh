// Float-float ("df64") arithmetic: a value is the unevaluated sum h + l of two floats with
// |l| <= ulp(h)/2, giving ~2^-46 relative precision on the FP32 pipes.  Built from the published
// error-free transformations: Knuth's TwoSum (s + e = a + b exactly) and the FMA form of
// Dekker's TwoProduct (p + e = a * b exactly, e = fma(a, b, -p)).  Additions use the "sloppy"
// variant (one TwoSum on the high parts, low parts added), whose error is bounded by a few ulps
// of 2^-46 relative to max(|a|, |b|) -- ample for a refinement residual that needs ~1e-9.
//
// Transcendentals (written from their series, not from any library):
//   exp(-x), x >= 0: x = k ln2 + t (|t| <= ln2/2), e^{-t} = (e^{-t/16})^16 with the series of
//     e^{u}, |u| <= 0.022, to u^2 in df64 and u^3..u^7 in FP32 (each below 1e-14 absolute error);
//   cos/sin(phi): phi = k pi/2 + r (|r| <= pi/4), r = j pi/64 + u (|u| <= pi/128) with a
//     17-entry table of sin/cos(j pi/64) in df64 and the Taylor series of sin u, cos u (u and
//     u^2/2 in df64, higher terms in FP32).
#pragma once

#include <cuda_runtime.h>

namespace bem {

struct df {
  float h, l;
};
struct cdf {
  df r, i;
};

__host__ __device__ __forceinline__ df dfm(float h, float l) {
  df r;
  r.h = h;
  r.l = l;
  return r;
}
__host__ inline df df_split(double x) {
  const float h = (float)x;
  return dfm(h, (float)(x - (double)h));
}
__device__ __forceinline__ df df_from(double x) {
  const float h = __double2float_rn(x);
  return dfm(h, __double2float_rn(x - (double)h));
}
__device__ __forceinline__ double df_to(df a) { return (double)a.h + (double)a.l; }

// The error-free sums use the round-to-nearest intrinsics, which the compiler never contracts
// into an FMA: a product fused into the sum s = a + b would leave s inconsistent with the a that
// the error term subtracts, and the pair would lose its low part.
__device__ __forceinline__ df quick2(float a, float b) {  // |a| >= |b|
  const float s = __fadd_rn(a, b);
  return dfm(s, __fsub_rn(b, __fsub_rn(s, a)));
}
__device__ __forceinline__ df two_sum2(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  return dfm(s, __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb)));
}
__device__ __forceinline__ df neg(df a) { return dfm(-a.h, -a.l); }
// Inside expressions the pairs are left unnormalised: the sum of the high parts is split exactly
// (TwoSum) and the low parts are added, but no final Quick-Two-Sum renormalises the result
// (|l| may then exceed ulp(h)/2 by a few ulps).  h + l still carries the value; a later product
// loses at most ~u |l| |b| (u = 2^-24), which after a cancellation of ratio c is ~u^2/c relative,
// the order of the error the cancellation itself leaves.  add_n renormalises, for running sums.
__device__ __forceinline__ df add(df a, df b) {
  const df s = two_sum2(a.h, b.h);
  return dfm(s.h, s.l + (a.l + b.l));
}
__device__ __forceinline__ df add_n(df a, df b) {
  const df s = two_sum2(a.h, b.h);
  return two_sum2(s.h, s.l + (a.l + b.l));
}
__device__ __forceinline__ df sub(df a, df b) { return add(a, neg(b)); }
__device__ __forceinline__ df addf(df a, float b) {
  const df s = two_sum2(a.h, b);
  return dfm(s.h, s.l + a.l);
}
__device__ __forceinline__ df mul(df a, df b) {
  const float p = a.h * b.h;
  float e = fmaf(a.h, b.h, -p);
  e = fmaf(a.h, b.l, fmaf(a.l, b.h, e));
  return dfm(p, e);
}
__device__ __forceinline__ df mulf(df a, float b) {
  const float p = a.h * b;
  const float e = fmaf(a.l, b, fmaf(a.h, b, -p));
  return dfm(p, e);
}
__device__ __forceinline__ df scale2(df a, float pow2) { return dfm(a.h * pow2, a.l * pow2); }  // exact

__host__ __device__ __forceinline__ cdf cmk(df r, df i) {
  cdf z;
  z.r = r;
  z.i = i;
  return z;
}

#if defined(__CUDA_ARCH__) && (__CUDA_ARCH__ >= 1000) && !defined(BEM_NO_F32X2)
// Complex float-float on the paired FP32 instructions of sm_100-family GPUs (FADD2 / FMUL2 /
// FFMA2): the real and imaginary parts go through the same error-free steps side by side, one
// paired instruction each, with the same roundings as the scalar forms below.  A difference
// x - y is formed as fma(-1, y, x), which rounds once exactly as the subtraction does; the
// intrinsics are never contracted.  BEM_NO_F32X2 builds the scalar forms instead.
struct df2 {
  float2 h, l;  // (re.h, im.h), (re.l, im.l)
};
__device__ __forceinline__ df2 pk(cdf a) { return {make_float2(a.r.h, a.i.h), make_float2(a.r.l, a.i.l)}; }
__device__ __forceinline__ cdf upk(df2 a) { return cmk(dfm(a.h.x, a.l.x), dfm(a.h.y, a.l.y)); }
__device__ __forceinline__ float2 p_sub(float2 x, float2 y) { return __ffma2_rn(make_float2(-1.f, -1.f), y, x); }
__device__ __forceinline__ df2 p_add(df2 a, df2 b) {  // lazy sum, as add()
  const float2 s = __fadd2_rn(a.h, b.h);
  const float2 bb = p_sub(s, a.h);
  const float2 e = __fadd2_rn(p_sub(a.h, p_sub(s, bb)), p_sub(b.h, bb));
  return {s, __fadd2_rn(e, __fadd2_rn(a.l, b.l))};
}
__device__ __forceinline__ df2 p_neg(df2 a) {
  return {make_float2(-a.h.x, -a.h.y), make_float2(-a.l.x, -a.l.y)};
}
// (k.h, k.l) broadcast times a pair, as mul()
__device__ __forceinline__ df2 p_mul(float2 kh, float2 kl, df2 a) {
  const float2 p = __fmul2_rn(kh, a.h);
  float2 e = __ffma2_rn(kh, a.h, make_float2(-p.x, -p.y));
  e = __ffma2_rn(kh, a.l, __ffma2_rn(kl, a.h, e));
  return {p, e};
}
__device__ __forceinline__ cdf cadd(cdf a, cdf b) { return upk(p_add(pk(a), pk(b))); }
__device__ __forceinline__ cdf csub(cdf a, cdf b) { return upk(p_add(pk(a), p_neg(pk(b)))); }
__device__ __forceinline__ cdf cscale(df k, cdf a) {
  return upk(p_mul(make_float2(k.h, k.h), make_float2(k.l, k.l), pk(a)));
}
__device__ __forceinline__ cdf cscalef(float k, cdf a) {
  const df2 x = pk(a);
  const float2 kk = make_float2(k, k);
  const float2 p = __fmul2_rn(x.h, kk);
  const float2 e = __ffma2_rn(x.l, kk, __ffma2_rn(x.h, kk, make_float2(-p.x, -p.y)));
  return upk({p, e});
}
// (a.r b.r - a.i b.i, a.r b.i + a.i b.r) = a.r (b.r, b.i) + a.i (-b.i, b.r)
__device__ __forceinline__ cdf cmul(cdf a, cdf b) {
  const df2 x = pk(b);
  const df2 y = {make_float2(-b.i.h, b.r.h), make_float2(-b.i.l, b.r.l)};
  const df2 u = p_mul(make_float2(a.r.h, a.r.h), make_float2(a.r.l, a.r.l), x);
  const df2 v = p_mul(make_float2(a.i.h, a.i.h), make_float2(a.i.l, a.i.l), y);
  return upk(p_add(u, v));
}
#else
__device__ __forceinline__ cdf cadd(cdf a, cdf b) { return cmk(add(a.r, b.r), add(a.i, b.i)); }
__device__ __forceinline__ cdf csub(cdf a, cdf b) { return cmk(sub(a.r, b.r), sub(a.i, b.i)); }
__device__ __forceinline__ cdf cmul(cdf a, cdf b) {
  return cmk(sub(mul(a.r, b.r), mul(a.i, b.i)), add(mul(a.r, b.i), mul(a.i, b.r)));
}
__device__ __forceinline__ cdf cscale(df k, cdf a) { return cmk(mul(k, a.r), mul(k, a.i)); }
__device__ __forceinline__ cdf cscalef(float k, cdf a) { return cmk(mulf(a.r, k), mulf(a.i, k)); }
#endif

// ---------------------------------------------------------------------------- exp(-x), x >= 0
struct DfConst {
  df ln2;          // ln 2
  df pio2;         // pi / 2
  df pio64;        // pi / 64
  float inv_ln2, two_over_pi, sixtyfour_over_pi;
  df tab_s[17];    // sin(j pi/64), j = 0..16
  df tab_c[17];    // cos(j pi/64)
};

__device__ __forceinline__ df df_exp_neg(df x, const DfConst& C) {
  const float k = rintf(x.h * C.inv_ln2);
  const df t = sub(x, mulf(C.ln2, k));          // |t| <= ln2/2, x = k ln2 + t
  const df v = scale2(neg(t), 0.0625f);           // v = -t/16, |v| <= 0.0217
  const float vh = v.h;
  // v^3/6 + v^4/24 + v^5/120 + v^6/720 + v^7/5040 in FP32 (< 2e-6, error < 1e-13)
  const float tail = vh * vh * vh * (1.f / 6.f + vh * (1.f / 24.f + vh * (1.f / 120.f + vh * (1.f / 720.f + vh * (1.f / 5040.f)))));
  df e = addf(add(v, scale2(mul(v, v), 0.5f)), tail);  // e^{v} - 1
  e = addf(e, 1.0f);
  e = mul(e, e);
  e = mul(e, e);
  e = mul(e, e);
  e = mul(e, e);                                   // e^{-t}
  const int ki = -(int)k;                          // exact scaling by 2^-k
  return dfm(scalbnf(e.h, ki), scalbnf(e.l, ki));
}

// cos(phi), sin(phi) for a df angle
__device__ __forceinline__ void df_sincos(df phi, const DfConst& C, df& sn, df& cs) {
  const float kq = rintf(phi.h * C.two_over_pi);
  const df r = sub(phi, mulf(C.pio2, kq));        // |r| <= pi/4 (+ rounding)
  const float jf = rintf(r.h * C.sixtyfour_over_pi);
  const df u = sub(r, mulf(C.pio64, jf));         // |u| <= pi/128
  const int j = (int)jf;                           // -16 .. 16
  const int ja = j < 0 ? -j : j;
  const df ts = j < 0 ? neg(C.tab_s[ja]) : C.tab_s[ja];
  const df tc = C.tab_c[ja];
  const float uh = u.h, u2 = uh * uh;
  // sin u = u - u^3/6 + u^5/120 ; cos u = 1 - u^2/2 + u^4/24 - u^6/720
  const df su = addf(u, uh * u2 * (-1.f / 6.f + u2 * (1.f / 120.f)));
  const df cu = addf(addf(scale2(neg(mul(u, u)), 0.5f), u2 * u2 * (1.f / 24.f - u2 * (1.f / 720.f))), 1.0f);
  df s = add(mul(ts, cu), mul(tc, su));             // sin(r)
  df c = sub(mul(tc, cu), mul(ts, su));             // cos(r)
  const int q = ((int)kq) & 3;
  if (q == 0) {
    sn = s;
    cs = c;
  } else if (q == 1) {
    sn = c;
    cs = neg(s);
  } else if (q == 2) {
    sn = neg(s);
    cs = neg(c);
  } else {
    sn = neg(c);
    cs = s;
  }
}

}  // namespace bem
