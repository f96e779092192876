// FP64-class refinement residual on the FP32 pipes: r = K(s) k - A(s) x (Sec. 2.1, Eq. (Aa_b))
// for the far field, in float-float arithmetic (df64.cuh), plus the FP64 near-field/own-element
// kernel.  Same decomposition as the FP32/FP64 far kernels (operator.cu): one thread per
// collocation point, FT frequencies per thread, source tiles in shared memory, split over the
// sources with FP64 atomic adds, every source contributing through T (applied to vT) and U
// (applied to vU):  (vT, vU) = (-x_e, k_e) for traction-given, (-k_e, x_e) for
// displacement-given columns.  Each kernel value is formed with ~1e-13 relative error, so the
// residual's error is far below the 1e-6 tolerance it certifies; GB300's FP32 pipes run this
// several times faster than its FP64 unit runs the same arithmetic.
#include "df64.cuh"
#include "kernel_math.cuh"

namespace bem {

namespace {

#ifndef BEM_RESID_FT
#define BEM_RESID_FT 4  // frequencies per CTA (a build-time choice: registers and shared memory)
#endif
constexpr int kTB = 128, kS = 32, kFT = BEM_RESID_FT;
constexpr int kSeriesDf = 9;            // |z| < 0.1: 9 Taylor terms of J reach 1e-15
constexpr float kZSeriesDf2 = 0.01f;

struct FreqDf {
  df a_re, a_im, b_re, b_im;  // s / c_s and beta s / c_s
  cdf inv_a2;                 // 1 / (s / c_s)^2
  float a_abs2, pad;
};

struct MatDf {
  df beta2, c1m2b2, inv4pimu, inv4pi;
  df d[kSeriesDf];            // Taylor coefficients of J(z)
};

struct ResDfArgs {
  const D4* q4;       // [ne][4] (x, y, z, w * area), FP64
  const D4* cen;      // [ne]
  const D4* nrm;      // [ne]
  const int8_t* bc;
  const double* bcv;  // [ne][3]
  const cx<double>* pfac;
  const cx<double>* x;
  double* yacc;
  const FreqDf* fc;
  const int32_t* flist;
  int64_t nfl, chunk, ne;
  MatDf m;
  DfConst C;
};

__device__ __forceinline__ cdf cdf_from(cx<double> z) { return cmk(df_from(z.r), df_from(z.i)); }

// one complex accumulator update: o += a * v (a, v complex)
__device__ __forceinline__ cdf cfma_df(cdf a, cdf v, cdf o) { return cadd(o, cmul(a, v)); }

// One source point's contribution to r = K k - A x at a target, in float-float, from the
// exponentials E_s, E_p and z_s, z_p: the radial algebra (J, Q, A, q1, q2; the Taylor series of
// J for |z_s| < 0.1) and the T contraction with vT (and n.vT) plus the U contraction with vU
// (v = vT[3], n.vT, vU[3]); cw = w/(4 pi r^2), cwd = cw dr/dn, cu = w/(4 pi mu r) carry the
// signed weight.
__device__ __forceinline__ void point_terms(cdf Es, cdf Ep, cdf zs, cdf zp, df inv_r2, const FreqDf& F,
                                            const MatDf& m, df cw, df cwd, df cu, df drdn, df rx, df ry, df rz,
                                            df n0, df n1, df n2, const cdf* v, cdf* oc) {
  const cdf gs = cadd(Es, cmul(zs, Es));
  const cdf gp = cadd(Ep, cmul(zp, Ep));
  const cdf Pp = csub(Es, cscale(m.beta2, Ep));
  cdf J;
  if (zs.r.h * zs.r.h + zs.i.h * zs.i.h < kZSeriesDf2) {
    J = cmk(m.d[kSeriesDf - 1], dfm(0.f, 0.f));
#pragma unroll 1
    for (int t = kSeriesDf - 2; t >= 0; --t) J = cadd(cmul(J, zs), cmk(m.d[t], dfm(0.f, 0.f)));
  } else {
    J = cscale(inv_r2, cmul(csub(gp, gs), F.inv_a2));
  }
  const cdf Q = csub(cscalef(6.f, J), cmk(scale2(Pp.r, 2.f), scale2(Pp.i, 2.f)));
  const cdf A = csub(Q, gs);
  const cdf q1 = csub(Q, cscale(m.c1m2b2, gp));
  const cdf g2 = csub(gs, cscale(m.beta2, gp));
  const cdf q2 = csub(cmk(scale2(g2.r, 2.f), scale2(g2.i, 2.f)), cscalef(5.f, Q));
  // T applied to vT
  const cdf rv = cadd(cadd(cscale(rx, v[0]), cscale(ry, v[1])), cscale(rz, v[2]));
  const cdf t1 = cscale(cwd, A);
  const cdf t2 = cmul(cscale(cw, A), rv);
  const cdf t3 = cscale(cw, cadd(cmul(q1, v[3]), cscale(drdn, cmul(q2, rv))));
  // U applied to vU
  const cdf psi = cscale(cu, csub(Es, J));
  const cdf ru = cadd(cadd(cscale(rx, v[4]), cscale(ry, v[5])), cscale(rz, v[6]));
  const cdf crv = cmul(cscale(cu, csub(Pp, cscalef(3.f, J))), ru);
  const cdf t3p = csub(t3, crv);
  oc[0] = cadd(cadd(cmul(t1, v[0]), cmul(psi, v[4])), cadd(cscale(n0, t2), cscale(rx, t3p)));
  oc[1] = cadd(cadd(cmul(t1, v[1]), cmul(psi, v[5])), cadd(cscale(n1, t2), cscale(ry, t3p)));
  oc[2] = cadd(cadd(cmul(t1, v[2]), cmul(psi, v[6])), cadd(cscale(n2, t2), cscale(rz, t3p)));
}

// The same point algebra split for a per-element application: oc[c] = rh_c t3' (the part that
// depends on the point's direction), and the scalars that multiply the element's own vectors,
// sc = (t1, psi, t2) with  point contribution_c = t1 vT_c + psi vU_c + n_c t2 + oc[c].  Summing
// sc over the element's points and applying it once per element replaces, per point, six
// complex float-float products and three scalings by three additions.
__device__ __forceinline__ void point_terms_split(cdf Es, cdf Ep, cdf zs, cdf zp, df inv_r2, const FreqDf& F,
                                                  const MatDf& m, df cw, df cwd, df cu, df drdn, df rx, df ry,
                                                  df rz, const cdf* v, cdf* oc, cdf* sc) {
  const cdf gs = cadd(Es, cmul(zs, Es));
  const cdf gp = cadd(Ep, cmul(zp, Ep));
  const cdf Pp = csub(Es, cscale(m.beta2, Ep));
  cdf J;
  if (zs.r.h * zs.r.h + zs.i.h * zs.i.h < kZSeriesDf2) {
    J = cmk(m.d[kSeriesDf - 1], dfm(0.f, 0.f));
#pragma unroll 1
    for (int t = kSeriesDf - 2; t >= 0; --t) J = cadd(cmul(J, zs), cmk(m.d[t], dfm(0.f, 0.f)));
  } else {
    J = cscale(inv_r2, cmul(csub(gp, gs), F.inv_a2));
  }
  const cdf Q = csub(cscalef(6.f, J), cmk(scale2(Pp.r, 2.f), scale2(Pp.i, 2.f)));
  const cdf A = csub(Q, gs);
  const cdf q1 = csub(Q, cscale(m.c1m2b2, gp));
  const cdf g2 = csub(gs, cscale(m.beta2, gp));
  const cdf q2 = csub(cmk(scale2(g2.r, 2.f), scale2(g2.i, 2.f)), cscalef(5.f, Q));
  const cdf rv = cadd(cadd(cscale(rx, v[0]), cscale(ry, v[1])), cscale(rz, v[2]));
  const cdf t3 = cscale(cw, cadd(cmul(q1, v[3]), cscale(drdn, cmul(q2, rv))));
  const cdf ru = cadd(cadd(cscale(rx, v[4]), cscale(ry, v[5])), cscale(rz, v[6]));
  const cdf crv = cmul(cscale(cu, csub(Pp, cscalef(3.f, J))), ru);
  const cdf t3p = csub(t3, crv);
  sc[0] = cscale(cwd, A);                 // t1, multiplies vT_c
  sc[1] = cscale(cu, csub(Es, J));        // psi, multiplies vU_c
  sc[2] = cmul(cscale(cw, A), rv);        // t2, multiplies n_c
  oc[0] = cscale(rx, t3p);
  oc[1] = cscale(ry, t3p);
  oc[2] = cscale(rz, t3p);
}

__global__ void __launch_bounds__(kTB) resid_df_kernel(const ResDfArgs a) {
  constexpr int TB = kTB, S = kS, FT = kFT;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  // float-float accumulators [FT][3 components][4 floats (re.h, re.l, im.h, im.l)][TB]: the
  // frequency loop stays rolled (the float-float body is large; unrolling it overflowed the
  // instruction cache), so its sums live in shared memory rather than in registers
  float* pacc = reinterpret_cast<float*>(smem_raw);                     // [FT * 12][TB]
  float* psum = pacc + FT * 12 * TB;                                     // [FT * 12][TB]: per-element
                                                                         // sums of (t1, psi, t2)
  float* sq = psum + FT * 12 * TB;                                       // [S][4][8]
  float* sn = sq + S * 4 * 8;                                            // [S][8]
  cdf* sv = reinterpret_cast<cdf*>(sn + S * 8);                          // [S][FT][7]
  FreqDf* sfc = reinterpret_cast<FreqDf*>(sv + S * FT * 7);              // [FT]
  DfConst* sC = reinterpret_cast<DfConst*>(sfc + FT);

  const int tid = threadIdx.x;
  const int64_t g0 = (int64_t)blockIdx.y * FT;
  const int nf = (int)min((int64_t)FT, a.nfl - g0);
  const int64_t src0 = (int64_t)blockIdx.z * a.chunk;
  const int64_t src1 = min(a.ne, src0 + a.chunk);
  const int64_t i = (int64_t)blockIdx.x * TB + tid;
  const bool valid = i < a.ne;
  df xi0 = dfm(0.f, 0.f), xi1 = xi0, xi2 = xi0;
  if (valid) {
    const D4 c = a.cen[i];
    xi0 = df_from(c.x);
    xi1 = df_from(c.y);
    xi2 = df_from(c.z);
  }
  if (tid < FT) sfc[tid] = a.fc[a.flist[g0 + min(tid, nf - 1)]];
  if (tid == 0) *sC = a.C;
  for (int k = 0; k < FT * 12; ++k) pacc[k * TB + tid] = 0.f;
  __syncthreads();
  // the amplitude e^{-Re(z)} depends on Re(s) only: shared by the group when Re(s) agrees
  bool same_re = true;
  for (int k = 1; k < nf; ++k)
    same_re = same_re && sfc[k].a_re.h == sfc[0].a_re.h && sfc[k].a_re.l == sfc[0].a_re.l;
  const MatDf& m = a.m;

  for (int64_t e0 = src0; e0 < src1; e0 += S) {
    const int ns = (int)min((int64_t)S, src1 - e0);
    __syncthreads();
    for (int t = tid; t < 4 * ns; t += TB) {
      const D4 p = a.q4[4 * e0 + t];
      float* o = sq + 8 * t;
      const df x = df_from(p.x), y = df_from(p.y), z = df_from(p.z), w = df_from(p.w);
      o[0] = x.h; o[1] = x.l; o[2] = y.h; o[3] = y.l; o[4] = z.h; o[5] = z.l; o[6] = w.h; o[7] = w.l;
    }
    for (int t = tid; t < ns; t += TB) {
      const D4 n = a.nrm[e0 + t];
      float* o = sn + 8 * t;
      const df x = df_from(n.x), y = df_from(n.y), z = df_from(n.z);
      o[0] = x.h; o[1] = x.l; o[2] = y.h; o[3] = y.l; o[4] = z.h; o[5] = z.l; o[6] = 0.f; o[7] = 0.f;
    }
    for (int t = tid; t < ns * FT; t += TB) {
      const int e = t / FT, k = t % FT;
      const int64_t ge = e0 + e;
      cdf* o = sv + 7 * (e * FT + k);
      if (k < nf) {
        const int64_t f = a.flist[g0 + k];
        const cx<double>* xv = a.x + (f * a.ne + ge) * 3;
        const cx<double> pf = a.pfac[f];
        const bool dir = a.bc && a.bc[ge] == BEM_BC_DISPLACEMENT;
        const D4 n = a.nrm[ge];
        cx<double> vT[3], vU[3];
        for (int c = 0; c < 3; ++c) {
          const double kv = a.bcv[3 * ge + c];
          const cx<double> kq = mk(pf.r * kv, pf.i * kv);
          vT[c] = (-1.0) * (dir ? kq : xv[c]);
          vU[c] = dir ? xv[c] : kq;
        }
        const cx<double> nv = mk(n.x * vT[0].r + n.y * vT[1].r + n.z * vT[2].r,
                                 n.x * vT[0].i + n.y * vT[1].i + n.z * vT[2].i);
        o[0] = cdf_from(vT[0]);
        o[1] = cdf_from(vT[1]);
        o[2] = cdf_from(vT[2]);
        o[3] = cdf_from(nv);
        o[4] = cdf_from(vU[0]);
        o[5] = cdf_from(vU[1]);
        o[6] = cdf_from(vU[2]);
      } else {
        const cdf zero = cmk(dfm(0.f, 0.f), dfm(0.f, 0.f));
        for (int c = 0; c < 7; ++c) o[c] = zero;
      }
    }
    __syncthreads();
    const DfConst& C = *sC;

    for (int e = 0; e < ns; ++e) {
      const bool self = (e0 + e == i);
      const float* nn = sn + 8 * e;
      const df n0 = dfm(nn[0], nn[1]), n1 = dfm(nn[2], nn[3]), n2 = dfm(nn[4], nn[5]);
#pragma unroll 1
      for (int q = 0; q < 4; ++q) {
        const float* P = sq + 8 * (4 * e + q);
        const df dx = sub(dfm(P[0], P[1]), xi0), dy = sub(dfm(P[2], P[3]), xi1),
                 dz = sub(dfm(P[4], P[5]), xi2);
        df r2 = add(add(mul(dx, dx), mul(dy, dy)), mul(dz, dz));
        if (self) r2 = dfm(1.f, 0.f);
        const float q0 = rsqrtf(r2.h);
        const float rh_ = r2.h * q0;
        const df r = quick2(rh_, (fmaf(-rh_, rh_, r2.h) + r2.l) * (0.5f * q0));
        const df corr = addf(neg(mulf(r, q0)), 1.0f);                 // 1 - r q0
        const df rinv = add(dfm(q0, 0.f), mulf(corr, q0));
        const df inv_r2 = mul(rinv, rinv);
        const df rx = mul(dx, rinv), ry = mul(dy, rinv), rz = mul(dz, rinv);
        const df drdn = add(add(mul(rx, n0), mul(ry, n1)), mul(rz, n2));
        const df w = self ? dfm(0.f, 0.f) : dfm(P[6], P[7]);
        const df cw = mul(mul(w, inv_r2), m.inv4pi);
        const df cu = mul(mul(w, rinv), m.inv4pimu);
        const df cwd = mul(cw, drdn);
        df amp_s = dfm(0.f, 0.f), amp_p = amp_s;
        if (same_re) {
          amp_s = df_exp_neg(mul(sfc[0].a_re, r), C);
          amp_p = df_exp_neg(mul(sfc[0].b_re, r), C);
        }
#pragma unroll 1
        for (int k = 0; k < nf; ++k) {
          const FreqDf& F = sfc[k];
          const cdf* v = sv + 7 * (e * FT + k);
          const df zr_s = mul(F.a_re, r), zr_p = mul(F.b_re, r);
          const df ph_s = mul(F.a_im, r), ph_p = mul(F.b_im, r);
          const df As = same_re ? amp_s : df_exp_neg(zr_s, C);
          const df Ap = same_re ? amp_p : df_exp_neg(zr_p, C);
          df sn_, cs_;
          df_sincos(ph_s, C, sn_, cs_);
          const cdf Es = cmk(mul(As, cs_), neg(mul(As, sn_)));
          df_sincos(ph_p, C, sn_, cs_);
          const cdf Ep = cmk(mul(Ap, cs_), neg(mul(Ap, sn_)));
          const cdf zs = cmk(zr_s, ph_s), zp = cmk(zr_p, ph_p);
          cdf oc[3], sc[3];
          point_terms_split(Es, Ep, zs, zp, inv_r2, F, m, cw, cwd, cu, drdn, rx, ry, rz, v, oc, sc);
          float* pa = pacc + (k * 12) * TB + tid;
          float* ps = psum + (k * 12) * TB + tid;
#pragma unroll
          for (int c = 0; c < 3; ++c) {
            float* pc = pa + (4 * c) * TB;
            const df re = add_n(dfm(pc[0], pc[TB]), oc[c].r);
            const df im = add_n(dfm(pc[2 * TB], pc[3 * TB]), oc[c].i);
            pc[0] = re.h;
            pc[TB] = re.l;
            pc[2 * TB] = im.h;
            pc[3 * TB] = im.l;
            float* pt = ps + (4 * c) * TB;
            const df sr = q == 0 ? sc[c].r : add_n(dfm(pt[0], pt[TB]), sc[c].r);
            const df si = q == 0 ? sc[c].i : add_n(dfm(pt[2 * TB], pt[3 * TB]), sc[c].i);
            pt[0] = sr.h;
            pt[TB] = sr.l;
            pt[2 * TB] = si.h;
            pt[3 * TB] = si.l;
          }
        }
      }
      // the element's sums applied once: t1 vT_c + psi vU_c + n_c t2
#pragma unroll 1
      for (int k = 0; k < nf; ++k) {
        const cdf* v = sv + 7 * (e * FT + k);
        const float* ps = psum + (k * 12) * TB + tid;
        const cdf S1 = cmk(dfm(ps[0], ps[TB]), dfm(ps[2 * TB], ps[3 * TB]));
        const cdf S2 = cmk(dfm(ps[4 * TB], ps[5 * TB]), dfm(ps[6 * TB], ps[7 * TB]));
        const cdf S3 = cmk(dfm(ps[8 * TB], ps[9 * TB]), dfm(ps[10 * TB], ps[11 * TB]));
        const df nn3[3] = {n0, n1, n2};
        float* pa = pacc + (k * 12) * TB + tid;
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          const cdf o = cadd(cadd(cmul(S1, v[c]), cmul(S2, v[4 + c])), cscale(nn3[c], S3));
          float* pc = pa + (4 * c) * TB;
          const df re = add_n(dfm(pc[0], pc[TB]), o.r);
          const df im = add_n(dfm(pc[2 * TB], pc[3 * TB]), o.i);
          pc[0] = re.h;
          pc[TB] = re.l;
          pc[2 * TB] = im.h;
          pc[3 * TB] = im.l;
        }
      }
    }
  }
  if (!valid) return;
  for (int k = 0; k < nf; ++k) {
    double* yo = a.yacc + ((int64_t)a.flist[g0 + k] * a.ne + i) * 6;
#pragma unroll
    for (int c = 0; c < 6; ++c) {
      const float* pc = pacc + (k * 12 + 2 * c) * TB + tid;
      atomicAdd(yo + c, (double)pc[0] + (double)pc[TB]);
    }
  }
}

// Near field and own element of r = K k - A x in float-float: one thread per (listed frequency,
// collocation point).  For every near source, the 7-point rule minus the 4-point rule the far
// sweep already applied (the same point algebra as the far sweep); the own element through its
// FP64 blocks, r_i += -(1/2 I + H_ii) vT_i + G_ii vU_i, in FP64.  Adds the far-field sums.
struct NearDfArgs {
  const D4 *q4, *q7, *cen, *nrm;  // FP64 geometry
  const int32_t *ptr, *col;       // near lists (CSR)
  const int8_t* bc;
  const double* bcv;              // [ne][3]
  const cx<double>* pfac;         // [F]
  const cx<double>* Tself;        // [F][ne][9]
  const cx<double>* Gself;
  const cx<double>* x;            // [F][ne][3]
  cx<double>* r;                  // [F][ne][3] out
  const double* yacc;             // far-field sums [F][ne][3] complex
  const FreqDf* fc;
  const int32_t* flist;
  int64_t nfl, ne;
  MatDf m;
  DfConst C;
};

__global__ void __launch_bounds__(128) near_df_kernel(const NearDfArgs a) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= a.nfl * a.ne) return;
  const int64_t f = a.flist[t / a.ne], i = t % a.ne;
  const FreqDf F = a.fc[f];
  const MatDf& m = a.m;
  const DfConst& C = a.C;
  const cx<double> pf = a.pfac[f];
  const D4 c = a.cen[i];
  const df xi0 = df_from(c.x), xi1 = df_from(c.y), xi2 = df_from(c.z);
  const df z0 = dfm(0.f, 0.f);
  cdf o[3] = {cmk(z0, z0), cmk(z0, z0), cmk(z0, z0)};
  // vT = -x or -k, vU = k or x of a source element (FP64), as in the far sweep
  auto sources = [&](int64_t e, cx<double>* vT, cx<double>* vU) {
    const cx<double>* xv = a.x + (f * a.ne + e) * 3;
    const bool dir = a.bc && a.bc[e] == BEM_BC_DISPLACEMENT;
    for (int q = 0; q < 3; ++q) {
      const double kv = a.bcv[3 * e + q];
      const cx<double> kq = mk(pf.r * kv, pf.i * kv);
      vT[q] = (-1.0) * (dir ? kq : xv[q]);
      vU[q] = dir ? xv[q] : kq;
    }
  };
  for (int32_t p = a.ptr[i]; p < a.ptr[i + 1]; ++p) {
    const int64_t e = a.col[p];
    cx<double> vT[3], vU[3];
    sources(e, vT, vU);
    const D4 nn = a.nrm[e];
    cdf v[7];
    for (int q = 0; q < 3; ++q) {
      v[q] = cmk(df_from(vT[q].r), df_from(vT[q].i));
      v[4 + q] = cmk(df_from(vU[q].r), df_from(vU[q].i));
    }
    v[3] = cmk(df_from(nn.x * vT[0].r + nn.y * vT[1].r + nn.z * vT[2].r),
               df_from(nn.x * vT[0].i + nn.y * vT[1].i + nn.z * vT[2].i));
    const df n0 = df_from(nn.x), n1 = df_from(nn.y), n2 = df_from(nn.z);
#pragma unroll 1
    for (int q = 0; q < 11; ++q) {
      const bool seven = q < 7;
      const D4 P = seven ? a.q7[7 * e + q] : a.q4[4 * e + (q - 7)];
      const df dx = sub(df_from(P.x), xi0), dy = sub(df_from(P.y), xi1), dz = sub(df_from(P.z), xi2);
      const df r2 = add(add(mul(dx, dx), mul(dy, dy)), mul(dz, dz));
      const float q0 = rsqrtf(r2.h);
      const float rh_ = r2.h * q0;
      const df r = quick2(rh_, (fmaf(-rh_, rh_, r2.h) + r2.l) * (0.5f * q0));
      const df rinv = add(dfm(q0, 0.f), mulf(addf(neg(mulf(r, q0)), 1.0f), q0));
      const df inv_r2 = mul(rinv, rinv);
      const df rx = mul(dx, rinv), ry = mul(dy, rinv), rz = mul(dz, rinv);
      const df drdn = add(add(mul(rx, n0), mul(ry, n1)), mul(rz, n2));
      const df w = seven ? df_from(P.w) : neg(df_from(P.w));   // 7-point rule minus 4-point rule
      const df cw = mul(mul(w, inv_r2), m.inv4pi);
      const df cu = mul(mul(w, rinv), m.inv4pimu);
      const df cwd = mul(cw, drdn);
      const df zr_s = mul(F.a_re, r), zr_p = mul(F.b_re, r);
      const df ph_s = mul(F.a_im, r), ph_p = mul(F.b_im, r);
      const df As = df_exp_neg(zr_s, C), Ap = df_exp_neg(zr_p, C);
      df sn_, cs_;
      df_sincos(ph_s, C, sn_, cs_);
      const cdf Es = cmk(mul(As, cs_), neg(mul(As, sn_)));
      df_sincos(ph_p, C, sn_, cs_);
      const cdf Ep = cmk(mul(Ap, cs_), neg(mul(Ap, sn_)));
      cdf oc[3];
      point_terms(Es, Ep, cmk(zr_s, ph_s), cmk(zr_p, ph_p), inv_r2, F, m, cw, cwd, cu, drdn, rx, ry, rz, n0,
                  n1, n2, v, oc);
      for (int k = 0; k < 3; ++k) o[k] = cmk(add_n(o[k].r, oc[k].r), add_n(o[k].i, oc[k].i));
    }
  }
  // own element (FP64 blocks): -(1/2 I + H_ii) x-part through vT, G_ii through vU
  cx<double> vT[3], vU[3];
  sources(i, vT, vU);
  const cx<double>* Hb = a.Tself + (f * a.ne + i) * 9;
  const cx<double>* Gb = a.Gself + (f * a.ne + i) * 9;
  const double* ya = a.yacc + (f * a.ne + i) * 6;
  cx<double>* ro = a.r + (f * a.ne + i) * 3;
  for (int rr = 0; rr < 3; ++rr) {
    cx<double> sacc = mk(ya[2 * rr], ya[2 * rr + 1]);
    for (int cc = 0; cc < 3; ++cc) {
      cx<double> d = Hb[3 * rr + cc];
      if (rr == cc) d.r += 0.5;
      sacc = cfma(d, vT[cc], sacc);
      sacc = cfma(Gb[3 * rr + cc], vU[cc], sacc);
    }
    ro[rr] = mk(sacc.r + df_to(o[rr].r), sacc.i + df_to(o[rr].i));
  }
}

// Own-element Duffy sums (the frequency-dependent part of the singular blocks, Sec. 2.1) in
// float-float: one warp per (frequency, element), lanes over the element's 3 x 13 x 13 Duffy
// points (SelfPt table), 13 complex sums per warp:
//   psi = sum w/r (E_s - J),  chi_ab = sum w/r (P - 3J) rh_a rh_b (6),
//   a_c = sum w/(4 pi r^2) (A + beta^2) rh_c,  b_c = sum w/(4 pi r^2) (q1 - beta^2) rh_c,
// the same sums the FP64 path forms point by point; the static CPV, the assembly of the 3 x 3
// blocks and the preconditioner inverse stay in FP64 (self_blocks_kernel).
struct SelfDfArgs {
  const SelfPt* pts;     // [ne][3 kDuffyN^2]
  const FreqDf* fc;      // [F]
  int64_t ne, F;
  MatDf m;
  DfConst C;
  cx<double>* out;       // [F][ne][13]
};

__device__ __forceinline__ df warp_sum_df(df v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const float h = __shfl_xor_sync(0xffffffffu, v.h, o), l = __shfl_xor_sync(0xffffffffu, v.l, o);
    v = add_n(v, dfm(h, l));
  }
  return v;
}

__global__ void __launch_bounds__(128) self_sums_df_kernel(const SelfDfArgs a) {
  constexpr int NP = 3 * kDuffyN * kDuffyN;
  const int64_t w = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (w >= a.F * a.ne) return;   // whole warps leave together: blockDim is a multiple of 32
  const int64_t f = w / a.ne, i = w % a.ne;
  const FreqDf F = a.fc[f];
  const MatDf& m = a.m;
  const DfConst& C = a.C;
  const df z0 = dfm(0.f, 0.f);
  cdf acc[13];
#pragma unroll
  for (int k = 0; k < 13; ++k) acc[k] = cmk(z0, z0);
  const SelfPt* P = a.pts + i * NP;
  for (int t = lane; t < NP; t += 32) {
    const SelfPt q = P[t];
    const df r = dfm(q.a.x, q.a.y), rh0 = dfm(q.a.z, q.a.w), rh1 = dfm(q.b.x, q.b.y), rh2 = dfm(q.b.z, q.b.w);
    const df wq = dfm(q.c.x, q.c.y);
    const float q0 = 1.0f / r.h;
    const df rinv = add(dfm(q0, 0.f), mulf(addf(neg(mulf(r, q0)), 1.0f), q0));   // 1/r, one Newton step
    const df inv_r2 = mul(rinv, rinv);
    const df zr_s = mul(F.a_re, r), zr_p = mul(F.b_re, r);
    const df ph_s = mul(F.a_im, r), ph_p = mul(F.b_im, r);
    const df As = df_exp_neg(zr_s, C), Ap = df_exp_neg(zr_p, C);
    df sn_, cs_;
    df_sincos(ph_s, C, sn_, cs_);
    const cdf Es = cmk(mul(As, cs_), neg(mul(As, sn_)));
    df_sincos(ph_p, C, sn_, cs_);
    const cdf Ep = cmk(mul(Ap, cs_), neg(mul(Ap, sn_)));
    const cdf zs = cmk(zr_s, ph_s), zp = cmk(zr_p, ph_p);
    const cdf gs = cadd(Es, cmul(zs, Es));
    const cdf gp = cadd(Ep, cmul(zp, Ep));
    const cdf Pp = csub(Es, cscale(m.beta2, Ep));
    cdf J;
    if (zr_s.h * zr_s.h + ph_s.h * ph_s.h < kZSeriesDf2) {
      J = cmk(m.d[kSeriesDf - 1], z0);
#pragma unroll 1
      for (int k = kSeriesDf - 2; k >= 0; --k) J = cadd(cmul(J, zs), cmk(m.d[k], z0));
    } else {
      J = cscale(inv_r2, cmul(csub(gp, gs), F.inv_a2));
    }
    const cdf Q = csub(cscalef(6.f, J), cmk(scale2(Pp.r, 2.f), scale2(Pp.i, 2.f)));
    const cdf A = csub(Q, gs);
    const cdf q1 = csub(Q, cscale(m.c1m2b2, gp));
    const df cu = mul(wq, rinv);
    const cdf psi = cscale(cu, csub(Es, J));
    const cdf chi = cscale(cu, csub(Pp, cscalef(3.f, J)));
    const df sc = mul(mul(wq, inv_r2), m.inv4pi);
    const cdf ra = cscale(sc, cmk(add(A.r, m.beta2), A.i));
    const cdf rb = cscale(sc, cmk(sub(q1.r, m.beta2), q1.i));
    // running sums stay normalised (add_n); the terms may be lazily normalised
    auto accum = [](cdf& s, cdf t) { s = cmk(add_n(s.r, t.r), add_n(s.i, t.i)); };
    accum(acc[0], psi);
    const df rr[6] = {mul(rh0, rh0), mul(rh0, rh1), mul(rh0, rh2), mul(rh1, rh1), mul(rh1, rh2), mul(rh2, rh2)};
#pragma unroll
    for (int k = 0; k < 6; ++k) accum(acc[1 + k], cscale(rr[k], chi));
    const df rh[3] = {rh0, rh1, rh2};
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      accum(acc[7 + c], cscale(rh[c], ra));
      accum(acc[10 + c], cscale(rh[c], rb));
    }
  }
#pragma unroll
  for (int k = 0; k < 13; ++k) acc[k] = cmk(warp_sum_df(acc[k].r), warp_sum_df(acc[k].i));
  if (lane == 0) {
    cx<double>* o = a.out + w * 13;
#pragma unroll
    for (int k = 0; k < 13; ++k) o[k] = mk(df_to(acc[k].r), df_to(acc[k].i));
  }
}

size_t resid_df_smem() {
  return sizeof(float) * 2 * 12 * kFT * kTB + sizeof(float) * kS * 4 * 8 + sizeof(float) * kS * 8 +
         sizeof(cdf) * kS * kFT * 7 + sizeof(FreqDf) * kFT + sizeof(DfConst);
}

DfConst make_df_const() {
  DfConst C;
  C.ln2 = df_split(0.69314718055994530942);
  C.pio2 = df_split(kPi / 2);
  C.pio64 = df_split(kPi / 64);
  C.inv_ln2 = (float)(1.0 / 0.69314718055994530942);
  C.two_over_pi = (float)(2.0 / kPi);
  C.sixtyfour_over_pi = (float)(64.0 / kPi);
  for (int j = 0; j <= 16; ++j) {
    C.tab_s[j] = df_split(std::sin(j * kPi / 64));
    C.tab_c[j] = df_split(std::cos(j * kPi / 64));
  }
  return C;
}

}  // namespace

// r[f] = K(s_f) k_f - A(s_f) x[f] for the listed frequencies: far and near field in float-float,
// the own element's blocks applied in FP64.
void residual_df(bem_ctx* ctx, const cx<double>* x, cx<double>* r, const std::vector<int32_t>* flist,
                 const cx<double>* pfac_override) {
  BEM_REQUIRE(ctx->bc.set, "residual needs boundary conditions");
  const int64_t nfl = stage_flist(ctx, flist, 0);
  if (!nfl) return;
  const MatC<double> md = mat_constants64(ctx->mat);
  ResDfArgs a;
  a.q4 = ctx->mesh.q4_64.as<D4>();
  a.cen = ctx->mesh.c64.as<D4>();
  a.nrm = ctx->mesh.n64.as<D4>();
  a.bc = ctx->bc.d_type.as<int8_t>();
  a.bcv = ctx->bc.d_value.as<double>();
  a.pfac = pfac_override ? pfac_override : ctx->fs.pfac.as<cx<double>>();
  a.x = x;
  a.yacc = ctx->yacc.as<double>();
  a.fc = ctx->fs.fcdf.as<FreqDf>();
  a.flist = ctx->flist_d.as<int32_t>();
  a.nfl = nfl;
  a.ne = ctx->mesh.ne;
  a.m.beta2 = df_split(md.beta2);
  a.m.c1m2b2 = df_split(md.c1m2b2);
  a.m.inv4pimu = df_split(md.inv4pimu);
  a.m.inv4pi = df_split(kInv4Pi);
  for (int t = 0; t < kSeriesDf; ++t) a.m.d[t] = df_split(md.d[t]);
  a.C = make_df_const();
  const int64_t tb = grid_for(a.ne, kTB), groups = grid_for(nfl, kFT);
  const size_t smem = resid_df_smem();
  BEM_CUDA(cudaFuncSetAttribute(resid_df_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  // Split the sources so that the last wave of CTAs is nearly full: every CTA does the same
  // work (its share of the sources for its targets and frequencies), so the launch takes
  // ceil(CTAs / resident slots) CTA-durations, each 1/nsplit of an unsplit CTA, plus a fixed
  // cost per CTA (set-up and the FP64 atomic adds, counted as one source tile).  The split
  // minimising that, with chunks of at least 8 source tiles, wins (ties: the smaller split).
  // Unsplit, 128 frequencies on 5120 triangles made 2.1 waves of which the third ran on a tenth
  // of the SMs.
  int per_sm = 0;
  BEM_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, resid_df_kernel, kTB, smem));
  const int64_t slots = (int64_t)std::max(per_sm, 1) * (ctx->n_sm > 0 ? ctx->n_sm : 152);
  const int64_t max_split = std::max<int64_t>(1, std::min<int64_t>(65535, a.ne / (8 * kS)));
  int64_t nsplit = 1;
  double best = 1e300;
  for (int64_t ns = 1; ns <= max_split; ++ns) {
    int64_t chunk = (a.ne + ns - 1) / ns;
    chunk = ((chunk + kS - 1) / kS) * kS;
    const int64_t real_ns = (a.ne + chunk - 1) / chunk;
    const int64_t waves = (tb * groups * real_ns + slots - 1) / slots;
    const double cost = (double)waves * (double)(chunk + kS);  // CTA-durations x (sources + overhead)
    if (cost < best * (1.0 - 1e-9)) {
      best = cost;
      nsplit = real_ns;
    }
  }
  int64_t chunk = (a.ne + nsplit - 1) / nsplit;
  chunk = ((chunk + kS - 1) / kS) * kS;
  nsplit = (a.ne + chunk - 1) / chunk;
  a.chunk = chunk;
  {
    ProfScope ps(ctx, PK_RES64, nfl);
    resid_df_kernel<<<dim3((unsigned)tb, (unsigned)groups, (unsigned)nsplit), kTB, smem, ctx->stream>>>(a);
    BEM_LAUNCHED();
    ctx->launches++;
  }
  {
    NearDfArgs b;
    b.q4 = ctx->mesh.q4_64.as<D4>();
    b.q7 = ctx->mesh.q7_64.as<D4>();
    b.cen = ctx->mesh.c64.as<D4>();
    b.nrm = ctx->mesh.n64.as<D4>();
    b.ptr = ctx->mesh.near_ptr.as<int32_t>();
    b.col = ctx->mesh.near_col.as<int32_t>();
    b.bc = ctx->bc.d_type.as<int8_t>();
    b.bcv = ctx->bc.d_value.as<double>();
    b.pfac = a.pfac;
    b.Tself = ctx->fs.Tself.as<cx<double>>();
    b.Gself = ctx->fs.Gself.as<cx<double>>();
    b.x = x;
    b.r = r;
    b.yacc = ctx->yacc.as<double>();
    b.fc = ctx->fs.fcdf.as<FreqDf>();
    b.flist = ctx->flist_d.as<int32_t>();
    b.nfl = nfl;
    b.ne = ctx->mesh.ne;
    b.m = a.m;
    b.C = a.C;
    ProfScope ps(ctx, PK_NEAR64, nfl);
    near_df_kernel<<<grid_for(nfl * b.ne, 128), 128, 0, ctx->stream>>>(b);
    BEM_LAUNCHED();
    ctx->launches++;
  }
  ctx->f64_applies++;
}

void self_sums_df(bem_ctx* ctx, cx<double>* out) {
  const MatC<double> md = mat_constants64(ctx->mat);
  SelfDfArgs a;
  a.pts = ctx->mesh.self_pts.as<SelfPt>();
  a.fc = ctx->fs.fcdf.as<FreqDf>();
  a.ne = ctx->mesh.ne;
  a.F = ctx->fs.F;
  a.m.beta2 = df_split(md.beta2);
  a.m.c1m2b2 = df_split(md.c1m2b2);
  a.m.inv4pimu = df_split(md.inv4pimu);
  a.m.inv4pi = df_split(kInv4Pi);
  for (int t = 0; t < kSeriesDf; ++t) a.m.d[t] = df_split(md.d[t]);
  a.C = make_df_const();
  a.out = out;
  const int64_t threads = 32 * a.F * a.ne;
  self_sums_df_kernel<<<grid_for(threads, 128), 128, 0, ctx->stream>>>(a);
  BEM_LAUNCHED();
  ctx->launches++;
}

// y = A(s) x in float-float for the listed frequencies: the residual sweep with the known data
// switched off gives r = -A x, negated in place.
__global__ void negate_rows_kernel(cx<double>* y, const int32_t* flist, int64_t nfl, int64_t n) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= nfl * n) return;
  cx<double>& v = y[(int64_t)flist[t / n] * n + t % n];
  v = mk(-v.r, -v.i);
}

void apply_operator_df(bem_ctx* ctx, const cx<double>* x, cx<double>* y, const std::vector<int32_t>* flist) {
  const int64_t F = ctx->fs.F;
  ctx->zero_pfac.reserve(sizeof(cx<double>) * F);
  BEM_CUDA(cudaMemsetAsync(ctx->zero_pfac.p, 0, sizeof(cx<double>) * F, ctx->stream));
  residual_df(ctx, x, y, flist, ctx->zero_pfac.as<cx<double>>());
  const int64_t nfl = (int64_t)ctx->flist_h.size(), n = 3 * ctx->mesh.ne;
  if (nfl) {
    negate_rows_kernel<<<grid_for(nfl * n, 256), 256, 0, ctx->stream>>>(y, ctx->flist_d.as<int32_t>(), nfl, n);
    BEM_LAUNCHED();
    ctx->launches++;
  }
}

// FreqDf table for the current frequency set (called by prepare_frequencies)
void build_freq_df(bem_ctx* ctx, const double* s, int64_t F) {
  const MatC<double> m = mat_constants64(ctx->mat);
  const double cs = 1.0 / m.inv_cs;
  std::vector<FreqDf> h(F);
  for (int64_t k = 0; k < F; ++k) {
    const double ar = s[2 * k] / cs, ai = s[2 * k + 1] / cs;
    const double a2r = ar * ar - ai * ai, a2i = 2 * ar * ai, n2 = a2r * a2r + a2i * a2i;
    h[k].a_re = df_split(ar);
    h[k].a_im = df_split(ai);
    h[k].b_re = df_split(m.beta * ar);
    h[k].b_im = df_split(m.beta * ai);
    h[k].inv_a2 = cmk(df_split(a2r / n2), df_split(-a2i / n2));
    h[k].a_abs2 = (float)(ar * ar + ai * ai);
    h[k].pad = 0;
  }
  ctx->fs.fcdf.reserve(sizeof(FreqDf) * F);
  BEM_CUDA(cudaMemcpyAsync(ctx->fs.fcdf.p, h.data(), sizeof(FreqDf) * F, cudaMemcpyHostToDevice, ctx->stream));
  BEM_CUDA(cudaStreamSynchronize(ctx->stream));
}

}  // namespace bem
