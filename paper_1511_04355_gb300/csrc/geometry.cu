// Element geometry, near-source lists, own-element (singular) blocks and the block-Jacobi
// preconditioner: the per-mesh and per-frequency set-up of the frequency solve.
//
// Discretisation (Sec. 2.1, Eq. (bie) -> Eq. (Aa_b)): flat triangles, collocation at the
// centroid, constant displacement/traction per element.  Source integrals use
//   far  : the degree-3 four-point rule (centroid weight -27/48, (3/5,1/5,1/5) weights 25/48),
//   near : Radon's degree-5 seven-point rule, when |x_i - c_e| < 2 h_e (h_e = longest edge),
//   self : 13 x 13 Gauss-Legendre on the three Duffy squares around x_i for U and for the
//          bounded dynamic remainder of T, plus the closed-form Cauchy principal value of the
//          static part of T (on a flat element only rh_i n_j - n_i rh_j survives:
//          int T0 = beta^2/(4 pi) (C_i n_j - n_i C_j),  C_k = -sum_edges nu_k int ds / r).
#include <algorithm>
#include <cstring>

#include "kernel_math.cuh"

namespace bem {

// ------------------------------------------------------------------------------- rules
struct Rules {
  double b4[4][3], w4[4];
  double b7[7][3], w7[7];
  double gl[kDuffyN], glw[kDuffyN];  // Gauss-Legendre on [0, 1]
};

// Gauss-Legendre nodes/weights on [-1, 1] by Newton iteration on P_n (three-term recurrence),
// mapped to [0, 1].
static void gauss_legendre01(int n, double* x, double* w) {
  for (int k = 0; k < n; ++k) {
    double t = std::cos(kPi * (k + 0.75) / (n + 0.5));
    for (int it = 0; it < 100; ++it) {
      double p0 = 1.0, p1 = t;
      for (int j = 2; j <= n; ++j) {
        double p2 = ((2.0 * j - 1.0) * t * p1 - (j - 1.0) * p0) / j;
        p0 = p1;
        p1 = p2;
      }
      double dp = n * (t * p1 - p0) / (t * t - 1.0);
      double dt = p1 / dp;
      t -= dt;
      if (std::fabs(dt) < 1e-16) {
        // recompute derivative at the converged node for the weight
        p0 = 1.0;
        p1 = t;
        for (int j = 2; j <= n; ++j) {
          double p2 = ((2.0 * j - 1.0) * t * p1 - (j - 1.0) * p0) / j;
          p0 = p1;
          p1 = p2;
        }
        dp = n * (t * p1 - p0) / (t * t - 1.0);
        x[k] = 0.5 * (1.0 - t);
        w[k] = 1.0 / ((1.0 - t * t) * dp * dp);  // 2/((1-t^2) P'^2) scaled by 1/2
        break;
      }
    }
  }
}

static Rules make_rules() {
  Rules r;
  const double third = 1.0 / 3.0;
  double b4[4][3] = {{third, third, third}, {0.6, 0.2, 0.2}, {0.2, 0.6, 0.2}, {0.2, 0.2, 0.6}};
  double w4[4] = {-27.0 / 48.0, 25.0 / 48.0, 25.0 / 48.0, 25.0 / 48.0};
  std::memcpy(r.b4, b4, sizeof b4);
  std::memcpy(r.w4, w4, sizeof w4);
  const double s15 = std::sqrt(15.0);
  const double a[2] = {(6.0 - s15) / 21.0, (6.0 + s15) / 21.0};
  const double wa[2] = {(155.0 - s15) / 1200.0, (155.0 + s15) / 1200.0};
  r.b7[0][0] = r.b7[0][1] = r.b7[0][2] = third;
  r.w7[0] = 9.0 / 40.0;
  int q = 1;
  for (int o = 0; o < 2; ++o) {
    const double b = 1.0 - 2.0 * a[o];
    for (int p = 0; p < 3; ++p, ++q) {
      for (int c = 0; c < 3; ++c) r.b7[q][c] = (c == p) ? b : a[o];
      r.w7[q] = wa[o];
    }
  }
  gauss_legendre01(kDuffyN, r.gl, r.glw);
  return r;
}

static const Rules& rules() {
  static const Rules r = make_rules();
  return r;
}

__constant__ double c_gl[kDuffyN];
__constant__ double c_glw[kDuffyN];

// ------------------------------------------------------------------------------- geometry
struct GeoArgs {
  const double* verts;
  const int32_t* tris;
  int64_t ne, nv;
  double b4[4][3], w4[4], b7[7][3], w7[7];
  Elem64* elem;
  double* tri64;
  float4 *c32, *n32;
  D4 *c64, *n64;
  double *q4_64, *q7_64;
  float4 *q4_32, *q7_32;
  float4 *q4_32lo, *c32lo;
  int* bad;  // set to 1 + element index of a degenerate triangle
};

__global__ void geometry_kernel(GeoArgs a) {
  const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= a.ne) return;
  double p[3][3];
  for (int k = 0; k < 3; ++k) {
    const int32_t v = a.tris[3 * e + k];
    for (int c = 0; c < 3; ++c) p[k][c] = a.verts[3 * (int64_t)v + c];
  }
  double e1[3], e2[3], cr[3];
  for (int c = 0; c < 3; ++c) {
    e1[c] = p[1][c] - p[0][c];
    e2[c] = p[2][c] - p[0][c];
  }
  cr[0] = e1[1] * e2[2] - e1[2] * e2[1];
  cr[1] = e1[2] * e2[0] - e1[0] * e2[2];
  cr[2] = e1[0] * e2[1] - e1[1] * e2[0];
  const double a2 = sqrt(cr[0] * cr[0] + cr[1] * cr[1] + cr[2] * cr[2]);
  if (!(a2 > 0.0)) {
    atomicMax(a.bad, (int)(e + 1));
    return;
  }
  Elem64 el;
  double hmax = 0.0;
  for (int k = 0; k < 3; ++k) {
    double l2 = 0.0;
    for (int c = 0; c < 3; ++c) {
      const double d = p[(k + 1) % 3][c] - p[k][c];
      l2 += d * d;
    }
    hmax = fmax(hmax, sqrt(l2));
  }
  for (int c = 0; c < 3; ++c) {
    el.c[c] = (p[0][c] + p[1][c] + p[2][c]) / 3.0;
    el.n[c] = cr[c] / a2;
  }
  el.area = 0.5 * a2;
  el.h = hmax;
  a.elem[e] = el;
  for (int k = 0; k < 3; ++k)
    for (int c = 0; c < 3; ++c) a.tri64[9 * e + 3 * k + c] = p[k][c];
  a.c32[e] = make_float4((float)el.c[0], (float)el.c[1], (float)el.c[2], (float)el.h);
  a.c64[e] = D4{el.c[0], el.c[1], el.c[2], el.h};
  a.c32lo[e] = make_float4((float)(el.c[0] - (double)(float)el.c[0]), (float)(el.c[1] - (double)(float)el.c[1]),
                           (float)(el.c[2] - (double)(float)el.c[2]), 0.f);
  a.n64[e] = D4{el.n[0], el.n[1], el.n[2], el.area};
  a.n32[e] = make_float4((float)el.n[0], (float)el.n[1], (float)el.n[2], (float)el.area);
  for (int q = 0; q < 4; ++q) {
    double y[3];
    for (int c = 0; c < 3; ++c)
      y[c] = a.b4[q][0] * p[0][c] + a.b4[q][1] * p[1][c] + a.b4[q][2] * p[2][c];
    const double w = a.w4[q] * el.area;
    double* o = a.q4_64 + 4 * (4 * e + q);
    o[0] = y[0];
    o[1] = y[1];
    o[2] = y[2];
    o[3] = w;
    a.q4_32[4 * e + q] = make_float4((float)y[0], (float)y[1], (float)y[2], (float)w);
    a.q4_32lo[4 * e + q] = make_float4((float)(y[0] - (double)(float)y[0]), (float)(y[1] - (double)(float)y[1]),
                                       (float)(y[2] - (double)(float)y[2]), 0.f);
  }
  for (int q = 0; q < 7; ++q) {
    double y[3];
    for (int c = 0; c < 3; ++c)
      y[c] = a.b7[q][0] * p[0][c] + a.b7[q][1] * p[1][c] + a.b7[q][2] * p[2][c];
    const double w = a.w7[q] * el.area;
    double* o = a.q7_64 + 4 * (7 * e + q);
    o[0] = y[0];
    o[1] = y[1];
    o[2] = y[2];
    o[3] = w;
    a.q7_32[7 * e + q] = make_float4((float)y[0], (float)y[1], (float)y[2], (float)w);
  }
}

__global__ void self_pts_kernel(const Elem64* elem, const double* tri64, int64_t ne, SelfPt* out);

void build_geometry(bem_ctx* ctx) {
  Mesh& m = ctx->mesh;
  const int64_t ne = m.ne, nv = (int64_t)m.verts.size() / 3;
  DevBuf dv, dt, dbad;
  dv.reserve(sizeof(double) * 3 * nv);
  dt.reserve(sizeof(int32_t) * 3 * ne);
  dbad.reserve(sizeof(int));
  BEM_CUDA(cudaMemcpyAsync(dv.p, m.verts.data(), dv.bytes, cudaMemcpyHostToDevice, ctx->stream));
  BEM_CUDA(cudaMemcpyAsync(dt.p, m.tris.data(), dt.bytes, cudaMemcpyHostToDevice, ctx->stream));
  BEM_CUDA(cudaMemsetAsync(dbad.p, 0, sizeof(int), ctx->stream));
  m.elem64.reserve(sizeof(Elem64) * ne);
  m.tri64.reserve(sizeof(double) * 9 * ne);
  m.c32.reserve(sizeof(float4) * ne);
  m.n32.reserve(sizeof(float4) * ne);
  m.c64.reserve(sizeof(D4) * ne);
  m.n64.reserve(sizeof(D4) * ne);
  m.q4_64.reserve(sizeof(double) * 16 * ne);
  m.q7_64.reserve(sizeof(double) * 28 * ne);
  m.q4_32.reserve(sizeof(float4) * 4 * ne);
  m.q7_32.reserve(sizeof(float4) * 7 * ne);
  m.q4_32lo.reserve(sizeof(float4) * 4 * ne);
  m.c32lo.reserve(sizeof(float4) * ne);
  GeoArgs a;
  a.verts = dv.as<double>();
  a.tris = dt.as<int32_t>();
  a.ne = ne;
  a.nv = nv;
  const Rules& R = rules();
  std::memcpy(a.b4, R.b4, sizeof a.b4);
  std::memcpy(a.w4, R.w4, sizeof a.w4);
  std::memcpy(a.b7, R.b7, sizeof a.b7);
  std::memcpy(a.w7, R.w7, sizeof a.w7);
  a.elem = m.elem64.as<Elem64>();
  a.tri64 = m.tri64.as<double>();
  a.c32 = m.c32.as<float4>();
  a.n32 = m.n32.as<float4>();
  a.c64 = m.c64.as<D4>();
  a.n64 = m.n64.as<D4>();
  a.q4_64 = m.q4_64.as<double>();
  a.q7_64 = m.q7_64.as<double>();
  a.q4_32 = m.q4_32.as<float4>();
  a.q7_32 = m.q7_32.as<float4>();
  a.q4_32lo = m.q4_32lo.as<float4>();
  a.c32lo = m.c32lo.as<float4>();
  a.bad = dbad.as<int>();
  geometry_kernel<<<grid_for(ne, 128), 128, 0, ctx->stream>>>(a);
  BEM_LAUNCHED();
  ctx->launches++;
  int bad = 0;
  BEM_CUDA(cudaMemcpyAsync(&bad, dbad.p, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
  BEM_CUDA(cudaStreamSynchronize(ctx->stream));
  if (bad) throw Error(BEM_ERR_INVALID_ARG, "degenerate (zero-area) triangle " + std::to_string(bad - 1));
  BEM_CUDA(cudaMemcpyToSymbolAsync(c_gl, R.gl, sizeof R.gl, 0, cudaMemcpyHostToDevice, ctx->stream));
  BEM_CUDA(cudaMemcpyToSymbolAsync(c_glw, R.glw, sizeof R.glw, 0, cudaMemcpyHostToDevice, ctx->stream));
  const int64_t npts = ne * 3 * kDuffyN * kDuffyN;
  m.self_pts.reserve(sizeof(SelfPt) * npts);
  self_pts_kernel<<<grid_for(npts, 128), 128, 0, ctx->stream>>>(m.elem64.as<Elem64>(), m.tri64.as<double>(), ne,
                                                                 m.self_pts.as<SelfPt>());
  BEM_LAUNCHED();
  ctx->launches++;
}

// ------------------------------------------------------------------------------- near lists
// Row i lists the sources e != i with |x_i - c_e| < 2 h_e, ascending.  The distance is formed
// with explicitly rounded operations so the counting and the filling pass agree bit for bit.
__device__ __forceinline__ bool is_near(const Elem64& s, double x0, double x1, double x2) {
  const double d0 = __dsub_rn(s.c[0], x0), d1 = __dsub_rn(s.c[1], x1), d2 = __dsub_rn(s.c[2], x2);
  const double d = __dsqrt_rn(__dadd_rn(__dadd_rn(__dmul_rn(d0, d0), __dmul_rn(d1, d1)), __dmul_rn(d2, d2)));
  return d < __dmul_rn(kNearFactor, s.h);
}

// One thread per row; all lanes of a warp stream the same source element (broadcast loads).
__global__ void near_count_kernel(const Elem64* el, int64_t ne, int32_t* cnt) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const bool ok = i < ne;
  double x0 = 0, x1 = 0, x2 = 0;
  if (ok) {
    x0 = el[i].c[0];
    x1 = el[i].c[1];
    x2 = el[i].c[2];
  }
  int32_t c = 0;
  for (int64_t e = 0; e < ne; ++e)
    if (e != i && is_near(el[e], x0, x1, x2)) ++c;
  if (ok) cnt[i] = c;
}

__global__ void near_fill_kernel(const Elem64* el, int64_t ne, const int32_t* ptr, int32_t* col) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const bool ok = i < ne;
  double x0 = 0, x1 = 0, x2 = 0;
  if (ok) {
    x0 = el[i].c[0];
    x1 = el[i].c[1];
    x2 = el[i].c[2];
  }
  int32_t o = ok ? ptr[i] : 0;
  const int32_t end = ok ? ptr[i + 1] : 0;
  for (int64_t e = 0; e < ne; ++e)
    if (e != i && o < end && is_near(el[e], x0, x1, x2)) col[o++] = (int32_t)e;
}

void build_near_lists(bem_ctx* ctx) {
  Mesh& m = ctx->mesh;
  const int64_t ne = m.ne;
  m.near_ptr.reserve(sizeof(int32_t) * (ne + 1));
  DevBuf cnt;
  cnt.reserve(sizeof(int32_t) * ne);
  near_count_kernel<<<grid_for(ne, 128), 128, 0, ctx->stream>>>(m.elem64.as<Elem64>(), ne,
                                                                 cnt.as<int32_t>());
  BEM_LAUNCHED();
  ctx->launches++;
  std::vector<int32_t> h(ne);
  BEM_CUDA(cudaMemcpyAsync(h.data(), cnt.p, sizeof(int32_t) * ne, cudaMemcpyDeviceToHost, ctx->stream));
  BEM_CUDA(cudaStreamSynchronize(ctx->stream));
  m.h_near_ptr.assign(ne + 1, 0);
  for (int64_t i = 0; i < ne; ++i) {
    const int64_t next = (int64_t)m.h_near_ptr[i] + h[i];
    if (next > INT32_MAX) throw Error(BEM_ERR_INVALID_ARG, "near lists exceed 2^31 entries");
    m.h_near_ptr[i + 1] = (int32_t)next;
  }
  m.nnz = m.h_near_ptr[ne];
  m.near_col.reserve(sizeof(int32_t) * std::max<int64_t>(m.nnz, 1));
  BEM_CUDA(cudaMemcpyAsync(m.near_ptr.p, m.h_near_ptr.data(), sizeof(int32_t) * (ne + 1),
                           cudaMemcpyHostToDevice, ctx->stream));
  near_fill_kernel<<<grid_for(ne, 128), 128, 0, ctx->stream>>>(
      m.elem64.as<Elem64>(), ne, m.near_ptr.as<int32_t>(), m.near_col.as<int32_t>());
  BEM_LAUNCHED();
  ctx->launches++;
  m.h_near_col.resize(m.nnz);
  if (m.nnz)
    BEM_CUDA(cudaMemcpyAsync(m.h_near_col.data(), m.near_col.p, sizeof(int32_t) * m.nnz,
                             cudaMemcpyDeviceToHost, ctx->stream));
  BEM_CUDA(cudaStreamSynchronize(ctx->stream));
}

// ------------------------------------------------------------------------------- constants
static double series_coeff(int n) {  // c_n = (-1)^n (1 - n) / n!
  double f = 1.0;
  for (int k = 2; k <= n; ++k) f *= k;
  return ((n % 2) ? -1.0 : 1.0) * (1.0 - n) / f;
}

MatC<double> mat_constants64(const Material& mt) {
  const double lam = 2.0 * mt.mu * mt.nu / (1.0 - 2.0 * mt.nu);
  const double cs = std::sqrt(mt.mu / mt.rho), cp = std::sqrt((lam + 2.0 * mt.mu) / mt.rho);
  MatC<double> m;
  m.mu = mt.mu;
  m.inv_cs = 1.0 / cs;
  m.beta = cs / cp;
  m.beta2 = m.beta * m.beta;
  m.c1m2b2 = 1.0 - 2.0 * m.beta2;
  m.inv4pimu = 1.0 / (4.0 * kPi * mt.mu);
  for (int k = 0; k < kSeriesMax; ++k) m.d[k] = series_coeff(k + 2) * (std::pow(m.beta, k + 2) - 1.0);
  return m;
}

MatC<float> mat_constants32(const Material& mt) {
  const MatC<double> d = mat_constants64(mt);
  MatC<float> m;
  m.mu = (float)d.mu;
  m.inv_cs = (float)d.inv_cs;
  m.beta = (float)d.beta;
  m.beta2 = (float)d.beta2;
  m.c1m2b2 = (float)d.c1m2b2;
  m.inv4pimu = (float)d.inv4pimu;
  for (int k = 0; k < kSeriesMax; ++k) m.d[k] = (float)d.d[k];
  return m;
}

// ------------------------------------------------------------------------------- self blocks
struct SelfArgs {
  const Elem64* elem;
  const double* tri64;
  const int8_t* bc;
  const FreqC<double>* fc;
  int64_t ne, F;
  MatC<double> m;
  cx<double>* Tself;   // [F][ne][9]
  cx<double>* Gself;   // [F][ne][9]
  cx<double>* Minv64;  // [F][ne][9] (nullable)
  cx<float>* Minv32;   // [F][ne][9] (nullable)
  const int32_t* idx;  // optional element list (element_blocks); null = all
  int* singular;       // set when a diagonal block is singular
  const cx<double>* sums;  // [F][ne][13] Duffy sums formed in float-float (nullable: FP64 here)
};

// Own-element Duffy points of every element (frequency independent), FP64, stored as
// float-float pairs for the float-float sums: thread (i, t), t over the 3 kDuffyN^2 points of
// the three sub-triangles around the centroid.
__global__ void self_pts_kernel(const Elem64* elem, const double* tri64, int64_t ne, SelfPt* out) {
  constexpr int NPT = kDuffyN * kDuffyN;
  const int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (g >= ne * 3 * NPT) return;
  const int64_t i = g / (3 * NPT);
  const int t = (int)(g % (3 * NPT));
  const int sub = t / NPT, k = t % NPT, iu = k / kDuffyN, iv = k % kDuffyN;
  const double u = c_gl[iu], v = c_gl[iv];
  const Elem64 el = elem[i];
  double ea[3], eb[3], d[3];
  for (int c = 0; c < 3; ++c) {
    const double va = tri64[9 * i + 3 * sub + c], vb = tri64[9 * i + 3 * ((sub + 1) % 3) + c];
    ea[c] = va - el.c[c];
    eb[c] = vb - va;
    d[c] = u * ea[c] + u * v * eb[c];
  }
  const double cr0 = ea[1] * eb[2] - ea[2] * eb[1], cr1 = ea[2] * eb[0] - ea[0] * eb[2],
               cr2 = ea[0] * eb[1] - ea[1] * eb[0];
  const double wq = c_glw[iu] * c_glw[iv] * u * sqrt(cr0 * cr0 + cr1 * cr1 + cr2 * cr2);
  const double r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
  const double rinv = rsqrt(r2), r = r2 * rinv;
  auto hi = [](double x) { return __double2float_rn(x); };
  auto lo = [](double x) { return __double2float_rn(x - (double)__double2float_rn(x)); };
  const double rh0 = d[0] * rinv, rh1 = d[1] * rinv, rh2 = d[2] * rinv;
  SelfPt o;
  o.a = make_float4(hi(r), lo(r), hi(rh0), lo(rh0));
  o.b = make_float4(hi(rh1), lo(rh1), hi(rh2), lo(rh2));
  o.c = make_float2(hi(wq), lo(wq));
  out[g] = o;
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// 3x3 complex inverse by the adjugate (FP64); returns false if the determinant vanishes.
__device__ bool inv3(const cx<double>* A, cx<double>* B) {
  auto at = [&](int i, int j) { return A[3 * i + j]; };
  cx<double> C[9];
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      const int i1 = (i + 1) % 3, i2 = (i + 2) % 3, j1 = (j + 1) % 3, j2 = (j + 2) % 3;
      C[3 * j + i] = at(i1, j1) * at(i2, j2) - at(i1, j2) * at(i2, j1);  // adj = cof^T
    }
  const cx<double> det = at(0, 0) * C[0] + at(0, 1) * C[3] + at(0, 2) * C[6];
  const double d2 = det.r * det.r + det.i * det.i;
  if (!(d2 > 0.0)) return false;
  const cx<double> inv = mk(det.r / d2, -det.i / d2);
  for (int k = 0; k < 9; ++k) B[k] = C[k] * inv;
  return true;
}

// One warp per (frequency, element): 3 x 169 Duffy points spread over the lanes.  When the Duffy
// sums come precomputed (a.sums, float-float), what is left (closed-form CPV, assembly, inverse)
// is one thread's work: one thread per (frequency, element).
__global__ void self_blocks_kernel(SelfArgs a) {
  const int64_t gt = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int64_t w = a.sums ? gt : gt >> 5;
  const int lane = a.sums ? 0 : (int)(threadIdx.x & 31);
  const int64_t nitem = a.idx ? a.F : a.F * a.ne;  // with idx: F = number of listed elements
  if (w >= nitem) return;
  int64_t f, i;
  if (a.idx) {
    f = 0;
    i = a.idx[w];
  } else {
    f = w / a.ne;
    i = w % a.ne;
  }
  const Elem64 el = a.elem[i];
  double p[3][3];
  for (int k = 0; k < 3; ++k)
    for (int c = 0; c < 3; ++c) p[k][c] = a.tri64[9 * i + 3 * k + c];
  const FreqC<double> fc = a.fc[f];
  const MatC<double>& m = a.m;
  // accumulators: U: psi (1), chi rh rh (6 sym); T remainder: avec (3), bvec (3)
  cx<double> gpsi = mk(0.0, 0.0), gchi[6], av[3], bv[3];
  for (int k = 0; k < 6; ++k) gchi[k] = mk(0.0, 0.0);
  for (int k = 0; k < 3; ++k) av[k] = bv[k] = mk(0.0, 0.0);
  if (a.sums) {  // the Duffy sums were formed in float-float (self_sums_df)
    if (lane != 0) return;
    const cx<double>* sm = a.sums + w * 13;
    gpsi = sm[0];
    for (int k = 0; k < 6; ++k) gchi[k] = sm[1 + k];
    for (int k = 0; k < 3; ++k) {
      av[k] = sm[7 + k];
      bv[k] = sm[10 + k];
    }
  } else {
  constexpr int NPT = kDuffyN * kDuffyN;
  for (int t = lane; t < 3 * NPT; t += 32) {
    const int sub = t / NPT, k = t % NPT, iu = k / kDuffyN, iv = k % kDuffyN;
    const double u = c_gl[iu], v = c_gl[iv];
    const double* va = p[sub];
    const double* vb = p[(sub + 1) % 3];
    double ea[3], eb[3], d[3];
    for (int c = 0; c < 3; ++c) {
      ea[c] = va[c] - el.c[c];
      eb[c] = vb[c] - va[c];
      d[c] = u * ea[c] + u * v * eb[c];
    }
    const double cr0 = ea[1] * eb[2] - ea[2] * eb[1], cr1 = ea[2] * eb[0] - ea[0] * eb[2],
                 cr2 = ea[0] * eb[1] - ea[1] * eb[0];
    const double wq = c_glw[iu] * c_glw[iv] * u * sqrt(cr0 * cr0 + cr1 * cr1 + cr2 * cr2);
    const double r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
    const double rinv = rsqrt(r2), r = r2 * rinv, inv_r2 = rinv * rinv;
    const double rh[3] = {d[0] * rinv, d[1] * rinv, d[2] * rinv};
    const Radial<double> K = radial(r, inv_r2, fc, m);
    const cx<double> psi = (wq * rinv) * (K.Es - K.J);
    const cx<double> chi = (wq * rinv) * axpy(-3.0, K.J, K.P);
    gpsi = gpsi + psi;
    gchi[0] = axpy(rh[0] * rh[0], chi, gchi[0]);
    gchi[1] = axpy(rh[0] * rh[1], chi, gchi[1]);
    gchi[2] = axpy(rh[0] * rh[2], chi, gchi[2]);
    gchi[3] = axpy(rh[1] * rh[1], chi, gchi[3]);
    gchi[4] = axpy(rh[1] * rh[2], chi, gchi[4]);
    gchi[5] = axpy(rh[2] * rh[2], chi, gchi[5]);
    const TCoef<double> T = tcoef(K, m);
    const double sc = wq * inv_r2 * kInv4Pi;
    const cx<double> ra = sc * mk(T.A.r + m.beta2, T.A.i);     // A + beta^2 (A -> -beta^2)
    const cx<double> rb = sc * mk(T.q1.r - m.beta2, T.q1.i);   // q1 - beta^2 (q1 -> beta^2)
    for (int c = 0; c < 3; ++c) {
      av[c] = axpy(rh[c], ra, av[c]);
      bv[c] = axpy(rh[c], rb, bv[c]);
    }
  }
  gpsi = mk(warp_sum(gpsi.r), warp_sum(gpsi.i));
  for (int k = 0; k < 6; ++k) gchi[k] = mk(warp_sum(gchi[k].r), warp_sum(gchi[k].i));
  for (int k = 0; k < 3; ++k) {
    av[k] = mk(warp_sum(av[k].r), warp_sum(av[k].i));
    bv[k] = mk(warp_sum(bv[k].r), warp_sum(bv[k].i));
  }
  if (lane != 0) return;
  }
  // static CPV: C_k = -sum_edges nu_k int ds / r, nu = (b - a) x n / |b - a|
  double C[3] = {0, 0, 0};
  for (int k = 0; k < 3; ++k) {
    const double* pa = p[k];
    const double* pb = p[(k + 1) % 3];
    double t[3], ap[3];
    double L = 0;
    for (int c = 0; c < 3; ++c) {
      t[c] = pb[c] - pa[c];
      L += t[c] * t[c];
    }
    L = sqrt(L);
    for (int c = 0; c < 3; ++c) t[c] /= L;
    double t1 = 0;
    for (int c = 0; c < 3; ++c) t1 += (pa[c] - el.c[c]) * t[c];
    double pp = 0;
    for (int c = 0; c < 3; ++c) {
      ap[c] = (pa[c] - el.c[c]) - t1 * t[c];
      pp += ap[c] * ap[c];
    }
    pp = sqrt(pp);
    const double I = asinh((t1 + L) / pp) - asinh(t1 / pp);
    const double nu0 = t[1] * el.n[2] - t[2] * el.n[1];
    const double nu1 = t[2] * el.n[0] - t[0] * el.n[2];
    const double nu2 = t[0] * el.n[1] - t[1] * el.n[0];
    C[0] -= nu0 * I;
    C[1] -= nu1 * I;
    C[2] -= nu2 * I;
  }
  const double cs = m.beta2 * kInv4Pi;
  cx<double> Tb[9], Gb[9];
  const int sym[3][3] = {{0, 1, 2}, {1, 3, 4}, {2, 4, 5}};
  for (int r = 0; r < 3; ++r)
    for (int c = 0; c < 3; ++c) {
      const double stat = cs * (C[r] * el.n[c] - el.n[r] * C[c]);
      Tb[3 * r + c] = mk(stat, 0.0) + el.n[r] * av[c] + el.n[c] * bv[r];
      cx<double> g = (-1.0) * gchi[sym[r][c]];
      if (r == c) g = g + gpsi;
      Gb[3 * r + c] = m.inv4pimu * g;
    }
  const int64_t o = 9 * (f * a.ne + (a.idx ? w : i));
  for (int k = 0; k < 9; ++k) {
    a.Tself[o + k] = Tb[k];
    a.Gself[o + k] = Gb[k];
  }
  if (a.Minv64) {
    // diagonal block of A: traction given -> 1/2 I + H_ii ; displacement given -> -G_ii
    cx<double> D[9], B[9];
    const bool neu = a.bc ? (a.bc[i] == BEM_BC_TRACTION) : true;
    for (int k = 0; k < 9; ++k) D[k] = neu ? Tb[k] : (-1.0) * Gb[k];
    if (neu) {
      D[0].r += 0.5;
      D[4].r += 0.5;
      D[8].r += 0.5;
    }
    if (!inv3(D, B)) {
      atomicMax(a.singular, 1);
      for (int k = 0; k < 9; ++k) B[k] = mk((k % 4 == 0) ? 1.0 : 0.0, 0.0);
    }
    for (int k = 0; k < 9; ++k) {
      a.Minv64[o + k] = B[k];
      a.Minv32[o + k] = mk((float)B[k].r, (float)B[k].i);
    }
  }
}

// ------------------------------------------------------------------------------- frequencies
void prepare_frequencies(bem_ctx* ctx, const double* s, int64_t F, bool df_self) {
  hm_invalidate(ctx, false);  // H-matrix factors belong to the previous frequency set
  Mesh& me = ctx->mesh;
  FreqSet& fs = ctx->fs;
  const MatC<double> m = mat_constants64(ctx->mat);
  const double cs = 1.0 / m.inv_cs;
  std::vector<FreqC<double>> h64(F);
  std::vector<FreqC<float>> h32(F);
  std::vector<cx<double>> pf(F);
  for (int64_t k = 0; k < F; ++k) {
    const double sr = s[2 * k], si = s[2 * k + 1];
    BEM_REQUIRE(sr > 0.0 && std::isfinite(sr) && std::isfinite(si),
                "every frequency needs 0 < Re s < inf");
    const cx<double> a = mk(sr / cs, si / cs);
    const cx<double> a2 = a * a;
    const double n2 = a2.r * a2.r + a2.i * a2.i;
    h64[k].a = a;
    h64[k].inv_a2 = mk(a2.r / n2, -a2.i / n2);
    h64[k].a_abs2 = a.r * a.r + a.i * a.i;
    h64[k].pad = 0;
    h32[k].a = mk((float)a.r, (float)a.i);
    h32[k].inv_a2 = mk((float)h64[k].inv_a2.r, (float)h64[k].inv_a2.i);
    h32[k].a_abs2 = (float)h64[k].a_abs2;
    h32[k].pad = 0;
    const double bi = m.beta * a.i;
    h32[k].ai_hi = (float)a.i;
    h32[k].ai_lo = (float)(a.i - (double)h32[k].ai_hi);
    h32[k].bi_hi = (float)bi;
    h32[k].bi_lo = (float)(bi - (double)h32[k].bi_hi);
    h64[k].ai_hi = a.i;
    h64[k].ai_lo = 0;
    h64[k].bi_hi = bi;
    h64[k].bi_lo = 0;
    const double ss = sr * sr + si * si;
    pf[k] = (ctx->bc.profile == BEM_PROFILE_STEP) ? mk(sr / ss, -si / ss) : mk(1.0, 0.0);
  }
  fs.F = F;
  fs.s.assign(s, s + 2 * F);
  fs.fc64.reserve(sizeof(FreqC<double>) * F);
  fs.fc32.reserve(sizeof(FreqC<float>) * F);
  fs.pfac.reserve(sizeof(cx<double>) * F);
  BEM_CUDA(cudaMemcpyAsync(fs.fc64.p, h64.data(), sizeof(FreqC<double>) * F, cudaMemcpyHostToDevice, ctx->stream));
  BEM_CUDA(cudaMemcpyAsync(fs.fc32.p, h32.data(), sizeof(FreqC<float>) * F, cudaMemcpyHostToDevice, ctx->stream));
  BEM_CUDA(cudaMemcpyAsync(fs.pfac.p, pf.data(), sizeof(cx<double>) * F, cudaMemcpyHostToDevice, ctx->stream));
  build_freq_df(ctx, s, F);
  const size_t nb = sizeof(cx<double>) * 9 * F * me.ne;
  fs.Tself.reserve(nb);
  fs.Gself.reserve(nb);
  fs.Minv64.reserve(nb);
  fs.Minv32.reserve(nb / 2);
  DevBuf sing;
  sing.reserve(sizeof(int));
  BEM_CUDA(cudaMemsetAsync(sing.p, 0, sizeof(int), ctx->stream));
  SelfArgs a;
  a.elem = me.elem64.as<Elem64>();
  a.tri64 = me.tri64.as<double>();
  a.bc = ctx->bc.set ? ctx->bc.d_type.as<int8_t>() : nullptr;
  a.fc = fs.fc64.as<FreqC<double>>();
  a.ne = me.ne;
  a.F = F;
  a.m = m;
  a.Tself = fs.Tself.as<cx<double>>();
  a.Gself = fs.Gself.as<cx<double>>();
  a.Minv64 = fs.Minv64.as<cx<double>>();
  a.Minv32 = fs.Minv32.as<cx<float>>();
  a.idx = nullptr;
  a.singular = sing.as<int>();
  ProfScope ps(ctx, PK_SELF);
  DevBuf sums;
  a.sums = nullptr;
  if (df_self) {
    sums.reserve(sizeof(cx<double>) * 13 * F * me.ne);
    self_sums_df(ctx, sums.as<cx<double>>());
    a.sums = sums.as<cx<double>>();
  }
  const int64_t threads = (df_self ? 1 : 32) * F * me.ne;
  self_blocks_kernel<<<grid_for(threads, 128), 128, 0, ctx->stream>>>(a);
  BEM_LAUNCHED();
  ctx->launches++;
  int singular = 0;
  BEM_CUDA(cudaMemcpyAsync(&singular, sing.p, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
  BEM_CUDA(cudaStreamSynchronize(ctx->stream));
  if (singular) throw Error(BEM_ERR_BREAKDOWN, "singular 3x3 diagonal block (preconditioner)");
  fs.valid = true;
}

// ------------------------------------------------------------------------------- pair blocks
// Full 3 x 3 H and G blocks of non-self pairs, FP64, with the operator's rule selection.
struct PairArgs {
  const Elem64* elem;
  const double *q4, *q7;
  const int32_t *rows, *cols;
  int64_t n;
  FreqC<double> fc;
  MatC<double> m;
  cx<double>*H, *G;
};

__global__ void pair_blocks_kernel(PairArgs a) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= a.n) return;
  const int i = a.rows[t], e = a.cols[t];
  if (i == e) return;  // own element: filled by the self kernel
  const Elem64 xi = a.elem[i], se = a.elem[e];
  double dc2 = 0;
  for (int c = 0; c < 3; ++c) dc2 += (xi.c[c] - se.c[c]) * (xi.c[c] - se.c[c]);
  const bool near = dc2 < (kNearFactor * se.h) * (kNearFactor * se.h);
  const int nq = near ? 7 : 4;
  const double* q = near ? a.q7 + 28 * (int64_t)e : a.q4 + 16 * (int64_t)e;
  cx<double> H[9], G[9];
  for (int k = 0; k < 9; ++k) H[k] = G[k] = mk(0.0, 0.0);
  for (int p = 0; p < nq; ++p) {
    double d[3] = {q[4 * p] - xi.c[0], q[4 * p + 1] - xi.c[1], q[4 * p + 2] - xi.c[2]};
    const double w = q[4 * p + 3];
    const double r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
    const double rinv = rsqrt(r2), r = r2 * rinv, inv_r2 = rinv * rinv;
    const double rh[3] = {d[0] * rinv, d[1] * rinv, d[2] * rinv};
    const double drdn = rh[0] * se.n[0] + rh[1] * se.n[1] + rh[2] * se.n[2];
    const Radial<double> K = radial(r, inv_r2, a.fc, a.m);
    const TCoef<double> T = tcoef(K, a.m);
    const double st = w * inv_r2 * kInv4Pi, su = w * rinv * a.m.inv4pimu;
    const cx<double> psi = K.Es - K.J, chi = axpy(-3.0, K.J, K.P);
    for (int r_ = 0; r_ < 3; ++r_)
      for (int c = 0; c < 3; ++c) {
        cx<double> t = (rh[r_] * rh[c] * drdn) * T.q2 + (rh[r_] * se.n[c]) * T.q1 +
                       (((r_ == c) ? drdn : 0.0) + se.n[r_] * rh[c]) * T.A;
        H[3 * r_ + c] = axpy(st, t, H[3 * r_ + c]);
        cx<double> g = (-rh[r_] * rh[c]) * chi;
        if (r_ == c) g = g + psi;
        G[3 * r_ + c] = axpy(su, g, G[3 * r_ + c]);
      }
  }
  for (int k = 0; k < 9; ++k) {
    a.H[9 * t + k] = H[k];
    a.G[9 * t + k] = G[k];
  }
}

void element_blocks(bem_ctx* ctx, double sr, double si, const int32_t* rows, const int32_t* cols,
                    int64_t npairs, cx<double>* H, cx<double>* G) {
  Mesh& me = ctx->mesh;
  const MatC<double> m = mat_constants64(ctx->mat);
  const double cs = 1.0 / m.inv_cs;
  FreqC<double> fc;
  fc.a = mk(sr / cs, si / cs);
  const cx<double> a2 = fc.a * fc.a;
  const double n2 = a2.r * a2.r + a2.i * a2.i;
  fc.inv_a2 = mk(a2.r / n2, -a2.i / n2);
  fc.a_abs2 = fc.a.r * fc.a.r + fc.a.i * fc.a.i;
  fc.pad = 0;
  fc.ai_hi = fc.a.i;
  fc.ai_lo = 0;
  fc.bi_hi = m.beta * fc.a.i;
  fc.bi_lo = 0;
  for (int64_t k = 0; k < npairs; ++k)
    BEM_REQUIRE(rows[k] >= 0 && rows[k] < me.ne && cols[k] >= 0 && cols[k] < me.ne,
                "element index out of range");
  DevBuf dr, dc, dH, dG, dfc, dself, dTs, dGs;
  dr.reserve(sizeof(int32_t) * npairs);
  dc.reserve(sizeof(int32_t) * npairs);
  dH.reserve(sizeof(cx<double>) * 9 * npairs);
  dG.reserve(sizeof(cx<double>) * 9 * npairs);
  BEM_CUDA(cudaMemcpyAsync(dr.p, rows, sizeof(int32_t) * npairs, cudaMemcpyHostToDevice, ctx->stream));
  BEM_CUDA(cudaMemcpyAsync(dc.p, cols, sizeof(int32_t) * npairs, cudaMemcpyHostToDevice, ctx->stream));
  PairArgs pa;
  pa.elem = me.elem64.as<Elem64>();
  pa.q4 = me.q4_64.as<double>();
  pa.q7 = me.q7_64.as<double>();
  pa.rows = dr.as<int32_t>();
  pa.cols = dc.as<int32_t>();
  pa.n = npairs;
  pa.fc = fc;
  pa.m = m;
  pa.H = dH.as<cx<double>>();
  pa.G = dG.as<cx<double>>();
  pair_blocks_kernel<<<grid_for(npairs, 128), 128, 0, ctx->stream>>>(pa);
  BEM_LAUNCHED();
  ctx->launches++;
  // self pairs
  std::vector<int32_t> self_idx, self_pos;
  for (int64_t k = 0; k < npairs; ++k)
    if (rows[k] == cols[k]) {
      self_idx.push_back(rows[k]);
      self_pos.push_back((int32_t)k);
    }
  std::vector<cx<double>> hH(9 * npairs), hG(9 * npairs);
  BEM_CUDA(cudaMemcpyAsync(hH.data(), dH.p, dH.bytes, cudaMemcpyDeviceToHost, ctx->stream));
  BEM_CUDA(cudaMemcpyAsync(hG.data(), dG.p, dG.bytes, cudaMemcpyDeviceToHost, ctx->stream));
  if (!self_idx.empty()) {
    const int64_t ns = (int64_t)self_idx.size();
    dself.reserve(sizeof(int32_t) * ns);
    dfc.reserve(sizeof(FreqC<double>));
    dTs.reserve(sizeof(cx<double>) * 9 * ns);
    dGs.reserve(sizeof(cx<double>) * 9 * ns);
    BEM_CUDA(cudaMemcpyAsync(dself.p, self_idx.data(), sizeof(int32_t) * ns, cudaMemcpyHostToDevice, ctx->stream));
    BEM_CUDA(cudaMemcpyAsync(dfc.p, &fc, sizeof fc, cudaMemcpyHostToDevice, ctx->stream));
    SelfArgs a;
    a.elem = me.elem64.as<Elem64>();
    a.tri64 = me.tri64.as<double>();
    a.bc = nullptr;
    a.fc = dfc.as<FreqC<double>>();
    a.ne = 0;  // output index = position in the list (f = 0)
    a.F = ns;
    a.m = m;
    a.Tself = dTs.as<cx<double>>();
    a.Gself = dGs.as<cx<double>>();
    a.Minv64 = nullptr;
    a.Minv32 = nullptr;
    a.idx = dself.as<int32_t>();
    a.singular = nullptr;
    a.sums = nullptr;  // this verification entry point integrates in FP64
    self_blocks_kernel<<<grid_for(32 * ns, 128), 128, 0, ctx->stream>>>(a);
    BEM_LAUNCHED();
    ctx->launches++;
    std::vector<cx<double>> ts(9 * ns), gs(9 * ns);
    BEM_CUDA(cudaMemcpyAsync(ts.data(), dTs.p, dTs.bytes, cudaMemcpyDeviceToHost, ctx->stream));
    BEM_CUDA(cudaMemcpyAsync(gs.data(), dGs.p, dGs.bytes, cudaMemcpyDeviceToHost, ctx->stream));
    BEM_CUDA(cudaStreamSynchronize(ctx->stream));
    for (int64_t k = 0; k < ns; ++k)
      for (int j = 0; j < 9; ++j) {
        hH[9 * self_pos[k] + j] = ts[9 * k + j];
        hG[9 * self_pos[k] + j] = gs[9 * k + j];
      }
  }
  BEM_CUDA(cudaStreamSynchronize(ctx->stream));
  copy_out(ctx, H, hH.data(), sizeof(cx<double>) * 9 * npairs);
  copy_out(ctx, G, hG.data(), sizeof(cx<double>) * 9 * npairs);
}

}  // namespace bem
