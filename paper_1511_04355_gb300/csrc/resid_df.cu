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

constexpr int kTB = 128, kS = 32, kFT = 4;
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

__global__ void __launch_bounds__(kTB) resid_df_kernel(const ResDfArgs a) {
  constexpr int TB = kTB, S = kS, FT = kFT;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  // float-float accumulators [FT][3 components][4 floats (re.h, re.l, im.h, im.l)][TB]: the
  // frequency loop stays rolled (the float-float body is large; unrolling it overflowed the
  // instruction cache), so its sums live in shared memory rather than in registers
  float* pacc = reinterpret_cast<float*>(smem_raw);                     // [FT * 12][TB]
  float* sq = pacc + FT * 12 * TB;                                       // [S][4][8]
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
          const cdf gs = cadd(Es, cmul(zs, Es));
          const cdf gp = cadd(Ep, cmul(zp, Ep));
          const cdf Pp = csub(Es, cscale(m.beta2, Ep));
          cdf J;
          if (zr_s.h * zr_s.h + ph_s.h * ph_s.h < kZSeriesDf2) {
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
          const cdf o0 = cadd(cadd(cmul(t1, v[0]), cmul(psi, v[4])), cadd(cscale(n0, t2), cscale(rx, t3p)));
          const cdf o1 = cadd(cadd(cmul(t1, v[1]), cmul(psi, v[5])), cadd(cscale(n1, t2), cscale(ry, t3p)));
          const cdf o2 = cadd(cadd(cmul(t1, v[2]), cmul(psi, v[6])), cadd(cscale(n2, t2), cscale(rz, t3p)));
          float* pa = pacc + (k * 12) * TB + tid;
          const cdf oc[3] = {o0, o1, o2};
#pragma unroll
          for (int c = 0; c < 3; ++c) {
            float* pc = pa + (4 * c) * TB;
            const df re = add_n(dfm(pc[0], pc[TB]), oc[c].r);
            const df im = add_n(dfm(pc[2 * TB], pc[3 * TB]), oc[c].i);
            pc[0] = re.h;
            pc[TB] = re.l;
            pc[2 * TB] = im.h;
            pc[3 * TB] = im.l;
          }
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

size_t resid_df_smem() {
  return sizeof(float) * 12 * kFT * kTB + sizeof(float) * kS * 4 * 8 + sizeof(float) * kS * 8 +
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

// r[f] = K(s_f) k_f - A(s_f) x[f] for the listed frequencies: far field in float-float, near
// field and own element in FP64.
void residual_df(bem_ctx* ctx, const cx<double>* x, cx<double>* r, const std::vector<int32_t>* flist) {
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
  a.pfac = ctx->fs.pfac.as<cx<double>>();
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
  const int64_t want = 4 * 152 * 2;
  int64_t nsplit = std::max<int64_t>(1, (want + tb * groups - 1) / (tb * groups));
  nsplit = std::min<int64_t>(nsplit, 65535);
  int64_t chunk = (a.ne + nsplit - 1) / nsplit;
  chunk = ((chunk + kS - 1) / kS) * kS;
  nsplit = (a.ne + chunk - 1) / chunk;
  a.chunk = chunk;
  const size_t smem = resid_df_smem();
  BEM_CUDA(cudaFuncSetAttribute(resid_df_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  {
    ProfScope ps(ctx, PK_RES64, nfl);
    resid_df_kernel<<<dim3((unsigned)tb, (unsigned)groups, (unsigned)nsplit), kTB, smem, ctx->stream>>>(a);
    BEM_LAUNCHED();
    ctx->launches++;
  }
  near_residual64(ctx, x, r, nfl);
  ctx->f64_applies++;
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
