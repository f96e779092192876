// Device arithmetic of the Laplace-domain elastodynamic fundamental solutions.
//
// The boundary integral equation (Sec. 2.1, Eq. (bie)) uses the displacement and traction
// fundamental solutions U_ij, T_ij of the Laplace-transformed Navier equation (the paper omits
// them as textbook material).  With r = y - x, r = |r|, rh = r / r, n the unit normal at y,
// z = s r / c_s, beta = c_s / c_p, E_s = e^{-z}, E_p = e^{-beta z}, g_s = (1 + z) E_s,
// g_p = (1 + beta z) E_p and
//     J = (g_p - g_s) / z^2            (= beta^2 h(beta z) - h(z), h(z) = ((1+z)e^{-z} - 1)/z^2),
// the kernels reduce to
//     4 pi mu r U_ij = (E_s - J) delta_ij - (P - 3 J) rh_i rh_j,     P = E_s - beta^2 E_p,
//     4 pi r^2 T_ij  = A (delta_ij dr/dn + n_i rh_j) + q1 rh_i n_j + q2 dr/dn rh_i rh_j,
//     Q = 6 J - 2 P,  A = Q - g_s,  q1 = Q - (1 - 2 beta^2) g_p,  q2 = 2 (g_s - beta^2 g_p) - 5 Q.
// (Static limit z -> 0: A -> -beta^2, q1 -> beta^2, q2 -> -3 (1 - beta^2): Kelvin's kernels.)
// J cancels catastrophically for small |z|; there its Taylor series
//     J = sum_m d_m z^m,  d_m = c_{m+2} (beta^{m+2} - 1),  c_n = (-1)^n (1 - n) / n!,
// is used (|z|^2 < 1/4; 9 terms in FP32, 18 in FP64).
#pragma once

#include "bem_internal.cuh"

namespace bem {

constexpr double kPi = 3.14159265358979323846;
constexpr double kInv4Pi = 0.07957747154594767;

// e^{-z} for complex z, FP32: amplitude by the exp unit, phase reduced to [-pi, pi] by a
// two-constant Cody-Waite split of 2 pi before the hardware sine/cosine.
__device__ __forceinline__ cx<float> exp_neg(cx<float> z) {
  const float amp = __expf(-z.r);
  const float k = rintf(z.i * 0.159154943091895336f);
  float red = fmaf(-k, 6.28318548202514648f, z.i);     // 2 pi rounded to float
  red = fmaf(-k, -1.74845560007440834e-07f, red);      // 2 pi - (2 pi rounded to float)
  float sn, cs;
  __sincosf(red, &sn, &cs);
  return mk(amp * cs, -amp * sn);
}

// e^{-z} for complex z, FP64 (library exp and sincos).
__device__ __forceinline__ cx<double> exp_neg(cx<double> z) {
  const double amp = exp(-z.r);
  double sn, cs;
  sincos(z.i, &sn, &cs);
  return mk(amp * cs, -amp * sn);
}

// e^{-(re + i ph)} for FP32 with the phase given as a float-float pair (ph_hi + ph_lo): the
// Cody-Waite reduction acts on ph_hi and ph_lo is added after it, so the reduced argument keeps
// ~1e-7 absolute accuracy even for |ph| ~ 100.
__device__ __forceinline__ cx<float> exp_neg_ff(float re, float ph_hi, float ph_lo) {
  const float amp = __expf(-re);
  const float k = rintf(ph_hi * 0.159154943091895336f);
  float red = fmaf(-k, 6.28318548202514648f, ph_hi);
  red = fmaf(-k, -1.74845560007440834e-07f, red) + ph_lo;
  float sn, cs;
  __sincosf(red, &sn, &cs);
  return mk(amp * cs, -amp * sn);
}

// the same with the amplitude e^{-re} supplied (shared by frequencies with equal Re s)
__device__ __forceinline__ cx<float> cis_neg_ff(float amp, float ph_hi, float ph_lo) {
  const float k = rintf(ph_hi * 0.159154943091895336f);
  float red = fmaf(-k, 6.28318548202514648f, ph_hi);
  red = fmaf(-k, -1.74845560007440834e-07f, red) + ph_lo;
  float sn, cs;
  __sincosf(red, &sn, &cs);
  return mk(amp * cs, -amp * sn);
}

__device__ __forceinline__ float rsqrt_r(float x) { return rsqrtf(x); }
__device__ __forceinline__ double rsqrt_r(double x) { return rsqrt(x); }

template <class R>
struct NSeries;
template <>
struct NSeries<float> {
  static constexpr int n = kSeriesF32;
};
template <>
struct NSeries<double> {
  static constexpr int n = kSeriesF64;
};

// Radial part shared by U and T: E_s, P = E_s - beta^2 E_p, J, g_s, g_p at distance r.
template <class R>
struct Radial {
  cx<R> Es, P, J, gs, gp;
};

// phase factors: FP64 uses z directly; FP32 rebuilds the phase omega r / c from the float-float
// distance (r + r_lo) and float-float slopes
__device__ __forceinline__ void phase_exps(cx<float> zs, cx<float> zp, float r, float r_lo,
                                           const FreqC<float>& fc, cx<float>& Es, cx<float>& Ep) {
  const float ps = fc.ai_hi * r;
  const float ps_lo = fmaf(fc.ai_hi, r, -ps) + fmaf(fc.ai_hi, r_lo, fc.ai_lo * r);
  const float pp = fc.bi_hi * r;
  const float pp_lo = fmaf(fc.bi_hi, r, -pp) + fmaf(fc.bi_hi, r_lo, fc.bi_lo * r);
  Es = exp_neg_ff(zs.r, ps, ps_lo);
  Ep = exp_neg_ff(zp.r, pp, pp_lo);
}
__device__ __forceinline__ void phase_exps(cx<double> zs, cx<double> zp, double, double,
                                           const FreqC<double>&, cx<double>& Es, cx<double>& Ep) {
  Es = exp_neg(zs);
  Ep = exp_neg(zp);
}

// E_s = e^{-z_s}, E_p = e^{-z_p} at distance r.  r_lo: low part of the distance (float-float
// distance in the FP32 kernels, 0 otherwise); amp_s/amp_p >= 0: precomputed amplitudes
// e^{-Re z} (FP32 kernels, common Re s)
template <class R>
__device__ __forceinline__ void radial_exps(R r, const FreqC<R>& fc, const MatC<R>& m, R r_lo, float amp_s,
                                            float amp_p, cx<R>& Es, cx<R>& Ep) {
  const cx<R> zs = r * fc.a;
  const cx<R> zp = m.beta * zs;
  if constexpr (sizeof(R) == 4) {
    if (amp_s >= 0.f) {
      const float ps = fc.ai_hi * r;
      const float ps_lo = fmaf(fc.ai_hi, r, -ps) + fmaf(fc.ai_hi, r_lo, fc.ai_lo * r);
      const float pp = fc.bi_hi * r;
      const float pp_lo = fmaf(fc.bi_hi, r, -pp) + fmaf(fc.bi_hi, r_lo, fc.bi_lo * r);
      Es = cis_neg_ff(amp_s, ps, ps_lo);
      Ep = cis_neg_ff(amp_p, pp, pp_lo);
      return;
    }
  }
  phase_exps(zs, zp, r, r_lo, fc, Es, Ep);
}
// The rest of the radial part from given E_s, E_p.
template <class R>
__device__ __forceinline__ Radial<R> radial_given(R r, R inv_r2, const FreqC<R>& fc, const MatC<R>& m,
                                                  cx<R> Es, cx<R> Ep) {
  Radial<R> o;
  const cx<R> zs = r * fc.a;
  const cx<R> zp = m.beta * zs;
  o.Es = Es;
  o.gs = cfma(zs, Es, Es);
  o.gp = cfma(zp, Ep, Ep);
  o.P = axpy(-m.beta2, Ep, Es);
  const R z2 = r * r * fc.a_abs2;
  if (z2 < R(kZSeries2)) {
    constexpr int NS = NSeries<R>::n;
    cx<R> acc = mk(m.d[NS - 1], R(0));
#pragma unroll
    for (int k = NS - 2; k >= 0; --k) acc = cfma(acc, zs, mk(m.d[k], R(0)));
    o.J = acc;
  } else {
    o.J = inv_r2 * ((o.gp - o.gs) * fc.inv_a2);
  }
  return o;
}
// r_lo: low part of the distance (float-float distance in the FP32 kernels, 0 otherwise);
// amp_s/amp_p > 0: precomputed amplitudes e^{-Re z} (FP32 kernels, common Re s)
template <class R>
__device__ __forceinline__ Radial<R> radial(R r, R inv_r2, const FreqC<R>& fc, const MatC<R>& m,
                                            R r_lo = R(0), float amp_s = -1.f, float amp_p = -1.f) {
  Radial<R> o;
  const cx<R> zs = r * fc.a;
  const cx<R> zp = m.beta * zs;
  cx<R> Ep;
  if constexpr (sizeof(R) == 4) {
    if (amp_s >= 0.f) {
      const float ps = fc.ai_hi * r;
      const float ps_lo = fmaf(fc.ai_hi, r, -ps) + fmaf(fc.ai_hi, r_lo, fc.ai_lo * r);
      const float pp = fc.bi_hi * r;
      const float pp_lo = fmaf(fc.bi_hi, r, -pp) + fmaf(fc.bi_hi, r_lo, fc.bi_lo * r);
      o.Es = cis_neg_ff(amp_s, ps, ps_lo);
      Ep = cis_neg_ff(amp_p, pp, pp_lo);
    } else {
      phase_exps(zs, zp, r, r_lo, fc, o.Es, Ep);
    }
  } else {
    phase_exps(zs, zp, r, r_lo, fc, o.Es, Ep);
  }
  o.gs = cfma(zs, o.Es, o.Es);
  o.gp = cfma(zp, Ep, Ep);
  o.P = axpy(-m.beta2, Ep, o.Es);
  const R z2 = r * r * fc.a_abs2;
  if (z2 < R(kZSeries2)) {
    constexpr int NS = NSeries<R>::n;
    cx<R> acc = mk(m.d[NS - 1], R(0));
#pragma unroll
    for (int k = NS - 2; k >= 0; --k) acc = cfma(acc, zs, mk(m.d[k], R(0)));
    o.J = acc;
  } else {
    o.J = inv_r2 * ((o.gp - o.gs) * fc.inv_a2);
  }
  return o;
}

// Source-target distance.  FP32: float-float difference of the float-float coordinates and a
// float-float |d|^2, so that r carries ~1e-9 relative error (the phase omega r / c reaches ~60 rad
// at the top of the band); rh, dr/dn and the weights only need single precision.  FP64: plain.
template <class R>
struct Dist {
  R dx, dy, dz, r, r_lo, rinv;
};

// Knuth's TwoSum, s + e = a + b exactly; the intrinsics keep the compiler from contracting the
// products of the squared distance into these sums.
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

__device__ __forceinline__ Dist<float> distance(float px, float py, float pz, float4 pl, float x0,
                                                float x1, float x2, float4 xl, bool self) {
  Dist<float> d;
  float ex, ey, ez;
  two_sum(px, -x0, d.dx, ex);
  two_sum(py, -x1, d.dy, ey);
  two_sum(pz, -x2, d.dz, ez);
  const float lx = ex + (pl.x - xl.x), ly = ey + (pl.y - xl.y), lz = ez + (pl.z - xl.z);
  const float sx = d.dx * d.dx, sy = d.dy * d.dy, sz = d.dz * d.dz;
  const float qx = fmaf(d.dx, d.dx, -sx), qy = fmaf(d.dy, d.dy, -sy), qz = fmaf(d.dz, d.dz, -sz);
  float s1, e1, s2, e2;
  two_sum(sx, sy, s1, e1);
  two_sum(s1, sz, s2, e2);
  const float lo = (e1 + e2) + (qx + qy + qz) + 2.f * (d.dx * lx + d.dy * ly + d.dz * lz);
  if (self) s2 = 1.f;
  d.rinv = rsqrtf(s2);
  d.r = s2 * d.rinv;
  d.r_lo = self ? 0.f : (fmaf(-d.r, d.r, s2) + lo) * 0.5f * d.rinv;
  return d;
}

__device__ __forceinline__ Dist<double> distance(double px, double py, double pz, float4, double x0,
                                                 double x1, double x2, float4, bool self) {
  Dist<double> d;
  d.dx = px - x0;
  d.dy = py - x1;
  d.dz = pz - x2;
  const double r2 = self ? 1.0 : d.dx * d.dx + d.dy * d.dy + d.dz * d.dz;
  d.rinv = rsqrt(r2);
  d.r = r2 * d.rinv;
  d.r_lo = 0.0;
  return d;
}

// T coefficients (times 4 pi r^2): A, q1, q2.
template <class R>
struct TCoef {
  cx<R> A, q1, q2;
};
template <class R>
__device__ __forceinline__ TCoef<R> tcoef(const Radial<R>& k, const MatC<R>& m) {
  TCoef<R> t;
  const cx<R> Q = axpy(R(-2), k.P, R(6) * k.J);
  t.A = Q - k.gs;
  t.q1 = axpy(-m.c1m2b2, k.gp, Q);
  t.q2 = axpy(R(-5), Q, R(2) * axpy(-m.beta2, k.gp, k.gs));
  return t;
}

}  // namespace bem
