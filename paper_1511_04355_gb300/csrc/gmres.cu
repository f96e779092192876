// Batched GMRES(m) with right block-Jacobi preconditioning and FP64 iterative refinement:
// the linear solver of Sec. 2.1 ("the linear system is solved iteratively by GMRES", with the
// block-diagonal preconditioner of Sec. 4), run for every frequency of the batch at once.
//
// Outer loop (FP64-class): r = b - A x, formed in one sweep with b recomputed from the boundary
//                      data (float-float operator on the FP32 pipes by default, native FP64 with
//                      residual_mode BEM_RESID_FP64); later steps of a frequency update it,
//                      r <- r - A d, with the inner solve's correction d
//                      stop instance f when ||r_f|| <= tol ||b_f||
// Inner loop (precision T = float in MIXED mode, double in FP64 mode):
//                      GMRES(m) on A M^{-1} y = r, x += M^{-1} V y
//   Arnoldi: classical Gram-Schmidt applied twice (CGS2); every inner product and norm is
//   accumulated in FP64 and the Hessenberg matrix, Givens rotations and least-squares vector
//   are FP64; basis vectors are stored in T (they are the operator's input).
// Instances retire individually: a converged frequency clears its active flag and every
// kernel (including the operator tiles of its frequency group) skips it.
#include <algorithm>
#include <chrono>

#include "kernel_math.cuh"

namespace bem {

// ------------------------------------------------------------------------------- kernels
template <class T>
__device__ __forceinline__ cx<double> widen(cx<T> a) {
  return mk((double)a.r, (double)a.i);
}
template <class T>
__device__ __forceinline__ cx<T> narrow(cx<double> a) {
  return mk((T)a.r, (T)a.i);
}

__device__ __forceinline__ double block_sum(double v, double* sh) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();
  if (l == 0) sh[w] = v;
  __syncthreads();
  double s = 0;
  if (threadIdx.x < 32) {
    s = (l < (int)(blockDim.x >> 5)) ? sh[l] : 0.0;
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  }
  return s;  // valid in thread 0
}

// out[f] = sum_n |x[f][n]|^2 over instances with act[f] (one block per instance)
template <class T>
__global__ void norm2_kernel(const cx<T>* x, int64_t N, const int32_t* act, double* out) {
  __shared__ double sh[32];
  const int64_t f = blockIdx.x;
  if (act && !act[f]) return;
  const cx<T>* v = x + f * N;
  double s = 0;
  for (int64_t n = threadIdx.x; n < N; n += blockDim.x) {
    const cx<double> z = widen(v[n]);
    s = fma(z.r, z.r, fma(z.i, z.i, s));
  }
  s = block_sum(s, sh);
  if (threadIdx.x == 0) out[f] = s;
}

// dots[f][k] = sum_n conj(V[f][k][n]) w[f][n], k = 0..j  (grid: (j+1, F))
template <class T>
__global__ void gs_dots_kernel(const cx<T>* V, const cx<T>* w, int64_t N, int m1, int j,
                               const int32_t* act, cx<double>* dots) {
  __shared__ double sh[32];
  const int k = blockIdx.x;
  const int64_t f = blockIdx.y;
  if (!act[f] || k > j) return;
  const cx<T>* vk = V + (f * m1 + k) * N;
  const cx<T>* wv = w + f * N;
  double sr = 0, si = 0;
  for (int64_t n = threadIdx.x; n < N; n += blockDim.x) {
    const cx<double> a = widen(vk[n]), b = widen(wv[n]);
    sr = fma(a.r, b.r, fma(a.i, b.i, sr));
    si = fma(a.r, b.i, fma(-a.i, b.r, si));
  }
  sr = block_sum(sr, sh);
  si = block_sum(si, sh);
  if (threadIdx.x == 0) dots[f * m1 + k] = mk(sr, si);
}

// w[f][n] -= sum_{k<=j} dots[f][k] V[f][k][n]; hacc[f][k] += dots[f][k] (grid: (nb, F))
template <class T>
__global__ void gs_update_kernel(const cx<T>* V, cx<T>* w, int64_t N, int m1, int j,
                                 const int32_t* act, const cx<double>* dots, cx<double>* hacc) {
  extern __shared__ cx<double> sd[];
  const int64_t f = blockIdx.y;
  if (!act[f]) return;
  for (int k = threadIdx.x; k <= j; k += blockDim.x) sd[k] = dots[f * m1 + k];
  __syncthreads();
  if (blockIdx.x == 0)
    for (int k = threadIdx.x; k <= j; k += blockDim.x) hacc[f * m1 + k] = hacc[f * m1 + k] + sd[k];
  const int64_t n = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (n >= N) return;
  cx<double> s = widen(w[f * N + n]);
  for (int k = 0; k <= j; ++k) {
    const cx<double> v = widen(V[(f * m1 + k) * N + n]);
    s = s - sd[k] * v;
  }
  w[f * N + n] = narrow<T>(s);
}

struct GState {
  cx<double>* H;      // [F][m1][m] column-major by j: H[f][j*m1 + k]
  double* cs;         // [F][m]
  cx<double>* sn;     // [F][m]
  cx<double>* g;      // [F][m1]
  cx<double>* hacc;   // [F][m1] current column accumulator
  double* hnorm2;     // [F]
  double* target;     // [F] absolute residual target of this inner solve
  double* inv_h;      // [F] 1 / H[j+1][j]
  int32_t* act;       // [F] active in the current cycle
  int32_t* kcols;     // [F] Krylov columns used
  int32_t* status;    // [F] 0 ok, BEM_ERR_BREAKDOWN
  double* est;        // [F] residual estimate |g_{k}|
  int32_t* nact;      // [1] number of active instances after the step
};

// Finish Arnoldi column j for every active instance: Givens rotations, residual estimate,
// retirement (one thread per instance).
__global__ void arnoldi_finish_kernel(GState s, int64_t F, int m, int j) {
  const int64_t f = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (f >= F || !s.act[f]) return;
  const int m1 = m + 1;
  cx<double>* h = s.H + f * (int64_t)m1 * m + (int64_t)j * m1;
  for (int k = 0; k <= j; ++k) h[k] = s.hacc[f * m1 + k];
  const double hn = sqrt(s.hnorm2[f]);
  h[j + 1] = mk(hn, 0.0);
  // previous rotations
  for (int k = 0; k < j; ++k) {
    const double c = s.cs[f * m + k];
    const cx<double> sk = s.sn[f * m + k];
    const cx<double> a = h[k], b = h[k + 1];
    h[k] = c * a + sk * b;
    h[k + 1] = c * b - conj(sk) * a;
  }
  const cx<double> a = h[j];
  const double aa = sqrt(a.r * a.r + a.i * a.i);
  const double rho = sqrt(aa * aa + hn * hn);
  double c;
  cx<double> sj;
  if (aa == 0.0) {
    c = 0.0;
    sj = mk(1.0, 0.0);
    h[j] = mk(hn, 0.0);
  } else {
    c = aa / rho;
    sj = mk(a.r / aa * hn / rho, a.i / aa * hn / rho);  // (a/|a|) conj(b) / rho, b = hn real
    h[j] = mk(a.r / aa * rho, a.i / aa * rho);
  }
  h[j + 1] = mk(0.0, 0.0);
  s.cs[f * m + j] = c;
  s.sn[f * m + j] = sj;
  const cx<double> gj = s.g[f * m1 + j];
  s.g[f * m1 + j] = c * gj;
  s.g[f * m1 + j + 1] = (-1.0) * (conj(sj) * gj);
  const cx<double> gn = s.g[f * m1 + j + 1];
  const double res = sqrt(gn.r * gn.r + gn.i * gn.i);
  s.est[f] = res;
  s.kcols[f] = j + 1;
  const bool bad = !isfinite(res) || !isfinite(hn) || !isfinite(rho);
  if (bad) s.status[f] = BEM_ERR_BREAKDOWN;
  const bool done = bad || res <= s.target[f] || hn <= 1e-300 || j + 1 >= m;
  s.inv_h[f] = hn > 1e-300 ? 1.0 / hn : 0.0;
  if (done) s.act[f] = 0;
  else atomicAdd(s.nact, 1);
}

template <class T>
__global__ void normalize_kernel(const cx<T>* w, cx<T>* V, int64_t N, int m1, int j,
                                 const int32_t* act, const double* inv_h) {
  const int64_t f = blockIdx.y;
  if (!act[f]) return;
  const int64_t n = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (n >= N) return;
  const double s = inv_h[f];
  const cx<double> v = widen(w[f * N + n]);
  V[(f * m1 + j + 1) * N + n] = narrow<T>(s * v);
}

// v0 = r / ||r|| (to T), g = (beta, 0, ...), H accumulators cleared.
template <class T>
__global__ void start_kernel(const cx<double>* r, const double* rn2, cx<T>* V, int64_t N, int m1,
                             const int32_t* act, cx<double>* g) {
  const int64_t f = blockIdx.y;
  if (!act[f]) return;
  const int64_t n = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const double beta = sqrt(rn2[f]);
  if (n < m1) g[f * m1 + n] = mk(n == 0 ? beta : 0.0, 0.0);
  if (n >= N) return;
  const double s = beta > 0 ? 1.0 / beta : 0.0;
  V[f * m1 * N + n] = narrow<T>(s * r[f * N + n]);
}

__global__ void clear_hacc_kernel(cx<double>* hacc, int64_t F, int m1, const int32_t* act) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= F * m1) return;
  if (act[t / m1]) hacc[t] = mk(0.0, 0.0);
}

// y = R^{-1} g on the first k columns (back substitution), per instance.
__global__ void lsq_kernel(GState s, int64_t F, int m, const int32_t* part, cx<double>* y) {
  const int64_t f = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (f >= F || !part[f]) return;
  const int m1 = m + 1;
  const int k = s.kcols[f];
  const cx<double>* H = s.H + f * (int64_t)m1 * m;
  cx<double>* yf = y + f * m1;
  for (int r = k - 1; r >= 0; --r) {
    cx<double> acc = s.g[f * m1 + r];
    for (int c = r + 1; c < k; ++c) acc = acc - H[(int64_t)c * m1 + r] * yf[c];
    const cx<double> d = H[(int64_t)r * m1 + r];
    const double dd = d.r * d.r + d.i * d.i;
    yf[r] = dd > 0 ? acc * mk(d.r / dd, -d.i / dd) : mk(0.0, 0.0);
  }
}

// u[f] = sum_{k < kcols[f]} y[f][k] V[f][k]  (into T buffer)
template <class T>
__global__ void combine_kernel(const cx<T>* V, const cx<double>* y, const int32_t* kcols,
                               int64_t N, int m1, const int32_t* part, cx<T>* u) {
  const int64_t f = blockIdx.y;
  if (!part[f]) return;
  const int64_t n = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (n >= N) return;
  cx<double> s = mk(0.0, 0.0);
  const int k = kcols[f];
  for (int c = 0; c < k; ++c) s = s + y[f * m1 + c] * widen(V[(f * m1 + c) * N + n]);
  u[f * N + n] = narrow<T>(s);
}

// x64 += d (widened), for participating instances
template <class T>
__global__ void add_correction_kernel(cx<double>* x, const cx<T>* d, int64_t N, int64_t F,
                                      const int32_t* part) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= F * N || !part[t / N]) return;
  x[t] = x[t] + widen(d[t]);
}

// r -= widen(y) for the instances flagged in mask
__global__ void sub_widen_masked_kernel(cx<double>* r, const cx<float>* y, const int32_t* mask, int64_t N,
                                        int64_t n) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t < n && mask[t / N]) r[t] = r[t] - widen(y[t]);
}

// Warm-start scaling, one block per frequency f: alpha = (y^H b) / (y^H y) with y = A x^ (the
// complex scalar minimising |b - alpha y|; 0 when y = 0), then x0 = alpha x^ and r = b - alpha y.
// r may alias b (each element is read before it is written, by the same thread).
template <class Ry>
__global__ void warm_scale_kernel(const cx<double>* b, const cx<Ry>* y, cx<double>* x0, cx<double>* r, int64_t N) {
  __shared__ double s_yb_r[256], s_yb_i[256], s_yy[256];
  const int64_t f = blockIdx.x;
  const cx<double>* bf = b + f * N;
  const cx<Ry>* yf = y + f * N;
  double ybr = 0, ybi = 0, yy = 0;
  for (int64_t n = threadIdx.x; n < N; n += blockDim.x) {
    const cx<double> bv = bf[n];
    const double yr = (double)yf[n].r, yi = (double)yf[n].i;
    ybr += yr * bv.r + yi * bv.i;
    ybi += yr * bv.i - yi * bv.r;
    yy += yr * yr + yi * yi;
  }
  s_yb_r[threadIdx.x] = ybr;
  s_yb_i[threadIdx.x] = ybi;
  s_yy[threadIdx.x] = yy;
  __syncthreads();
  for (int k = blockDim.x / 2; k > 0; k >>= 1) {
    if ((int)threadIdx.x < k) {
      s_yb_r[threadIdx.x] += s_yb_r[threadIdx.x + k];
      s_yb_i[threadIdx.x] += s_yb_i[threadIdx.x + k];
      s_yy[threadIdx.x] += s_yy[threadIdx.x + k];
    }
    __syncthreads();
  }
  const double d = s_yy[0];
  const cx<double> alpha = d > 0 ? mk(s_yb_r[0] / d, s_yb_i[0] / d) : mk(0.0, 0.0);
  cx<double>* xf = x0 + f * N;
  cx<double>* rf = r + f * N;
  for (int64_t n = threadIdx.x; n < N; n += blockDim.x) {
    const cx<double> yv = mk((double)yf[n].r, (double)yf[n].i);
    const cx<double> bv = bf[n];
    xf[n] = alpha * xf[n];
    rf[n] = bv - alpha * yv;
  }
}

// Two-direction warm start, one block per frequency f: x0 = a1 x1 + a2 x2 with the complex
// (a1, a2) minimising |b - a1 y1 - a2 y2| (y_j = A x_j), by the 2 x 2 normal equations; when the
// directions are nearly parallel (Gram determinant below 1e-10 of its scale) the better single
// direction is used.  x1 is overwritten by x0, r = b - a1 y1 - a2 y2 (r may alias b).  Also
// writes the squared residuals of the combination and of x2 alone (rn2[2 f], rn2[2 f + 1]).
template <class Ry>
__global__ void warm_combine_kernel(const cx<double>* b, const cx<Ry>* y1, const cx<Ry>* y2, cx<double>* x1,
                                    const cx<double>* x2, cx<double>* r, int64_t N, double* rn2) {
  constexpr int NT = 256;
  __shared__ double sm[9][NT];
  const int64_t f = blockIdx.x;
  const cx<double>* bf = b + f * N;
  const cx<Ry>* p = y1 + f * N;
  const cx<Ry>* q = y2 + f * N;
  double acc[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};  // g11 g22 g12(r,i) c1(r,i) c2(r,i) bb
  for (int64_t n = threadIdx.x; n < N; n += NT) {
    const cx<double> bv = bf[n];
    const double pr = (double)p[n].r, pi = (double)p[n].i, qr = (double)q[n].r, qi = (double)q[n].i;
    acc[0] += pr * pr + pi * pi;
    acc[1] += qr * qr + qi * qi;
    acc[2] += pr * qr + pi * qi;          // conj(y1) y2
    acc[3] += pr * qi - pi * qr;
    acc[4] += pr * bv.r + pi * bv.i;      // conj(y1) b
    acc[5] += pr * bv.i - pi * bv.r;
    acc[6] += qr * bv.r + qi * bv.i;      // conj(y2) b
    acc[7] += qr * bv.i - qi * bv.r;
    acc[8] += bv.r * bv.r + bv.i * bv.i;
  }
  for (int k = 0; k < 9; ++k) sm[k][threadIdx.x] = acc[k];
  __syncthreads();
  for (int h = NT / 2; h > 0; h >>= 1) {
    if ((int)threadIdx.x < h)
      for (int k = 0; k < 9; ++k) sm[k][threadIdx.x] += sm[k][threadIdx.x + h];
    __syncthreads();
  }
  const double g11 = sm[0][0], g22 = sm[1][0], bb = sm[8][0];
  const cx<double> g12 = mk(sm[2][0], sm[3][0]), c1 = mk(sm[4][0], sm[5][0]), c2 = mk(sm[6][0], sm[7][0]);
  const double det = g11 * g22 - (g12.r * g12.r + g12.i * g12.i);
  cx<double> a1 = mk(0.0, 0.0), a2 = mk(0.0, 0.0);
  double res2;
  // x2 alone (the nearest stored solution)
  const double near2 = g22 > 0 ? bb - (c2.r * c2.r + c2.i * c2.i) / g22 : bb;
  if (g11 > 0 && g22 > 0 && det > 1e-10 * g11 * g22) {
    // [g11 g12; conj(g12) g22] [a1; a2] = [c1; c2]
    const cx<double> n1 = g22 * c1 - g12 * c2;
    const cx<double> n2 = g11 * c2 - conj(g12) * c1;
    a1 = mk(n1.r / det, n1.i / det);
    a2 = mk(n2.r / det, n2.i / det);
    res2 = bb - ((conj(c1) * a1).r + (conj(c2) * a2).r);
  } else {
    const double one2 = g11 > 0 ? bb - (c1.r * c1.r + c1.i * c1.i) / g11 : bb;
    if (g11 > 0 && one2 <= near2) {
      a1 = mk(c1.r / g11, c1.i / g11);
      res2 = one2;
    } else {
      if (g22 > 0) a2 = mk(c2.r / g22, c2.i / g22);
      res2 = near2;
    }
  }
  if (threadIdx.x == 0) {
    rn2[2 * f] = res2;
    rn2[2 * f + 1] = near2;
  }
  cx<double>* xf = x1 + f * N;
  const cx<double>* xn = x2 + f * N;
  cx<double>* rf = r + f * N;
  for (int64_t n = threadIdx.x; n < N; n += NT) {
    const cx<double> yv1 = mk((double)p[n].r, (double)p[n].i), yv2 = mk((double)q[n].r, (double)q[n].i);
    const cx<double> bv = bf[n];
    xf[n] = a1 * xf[n] + a2 * xn[n];
    rf[n] = bv - a1 * yv1 - a2 * yv2;
  }
}

// r = b - Ax  (for active instances)
__global__ void residual_kernel(const cx<double>* b, const cx<double>* Ax, cx<double>* r,
                                int64_t N, int64_t F, const int32_t* act) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= F * N || (act && !act[t / N])) return;
  r[t] = b[t] - Ax[t];
}

// ------------------------------------------------------------------------------- host driver
namespace {

struct Work {
  cx<double>* x = nullptr;    // FP64 [F][N] solution (caller-owned)
  DevBuf b, r, Ax;            // FP64 [F][N]
  DevBuf V, z, w, u;          // T
  DevBuf V64, z64, w64;       // FP64 inner-solve buffers of the mixed path's fallback
  DevBuf H, cs, sn, g, hacc, dots, y;
  DevBuf hnorm2, target, inv_h, est, bn2, rn2;
  DevBuf act, part, kcols, status, nact, upd;
};

template <class T>
struct Ops;
template <>
struct Ops<float> {
  static void op(bem_ctx* c, const cx<float>* x, cx<float>* y, const std::vector<int32_t>* l) {
    apply_operator32(c, x, y, BEM_APPLY_A, l);
  }
  static void pre(bem_ctx* c, const cx<float>* x, cx<float>* y, const int32_t* a) {
    apply_precond32(c, x, y, a);
  }
};
template <>
struct Ops<double> {
  static void op(bem_ctx* c, const cx<double>* x, cx<double>* y, const std::vector<int32_t>* l) {
    if (c->fp64_op_df) apply_operator_df(c, x, y, l);
    else apply_operator64(c, x, y, BEM_APPLY_A, l);
  }
  static void pre(bem_ctx* c, const cx<double>* x, cx<double>* y, const int32_t* a) {
    apply_precond64(c, x, y, a);
  }
};

// One GMRES(m) cycle on A M^{-1} y = r for the instances flagged in `part` (device), starting
// from x = 0 of the correction; adds the correction to x64.  Returns iterations performed.
template <class T>
int gmres_cycle(bem_ctx* ctx, Work& W, DevBuf& Vb, DevBuf& zb, DevBuf& wb, int64_t F, int64_t N, int m,
                std::vector<int32_t>& iters_host, const std::vector<int32_t>& part_h) {
  cudaStream_t st = ctx->stream;
  const int m1 = m + 1;
  GState s;
  s.H = W.H.as<cx<double>>();
  s.cs = W.cs.as<double>();
  s.sn = W.sn.as<cx<double>>();
  s.g = W.g.as<cx<double>>();
  s.hacc = W.hacc.as<cx<double>>();
  s.hnorm2 = W.hnorm2.as<double>();
  s.target = W.target.as<double>();
  s.inv_h = W.inv_h.as<double>();
  s.act = W.act.as<int32_t>();
  s.kcols = W.kcols.as<int32_t>();
  s.status = W.status.as<int32_t>();
  s.est = W.est.as<double>();
  s.nact = W.nact.as<int32_t>();
  cx<T>* V = Vb.as<cx<T>>();
  cx<T>* z = zb.as<cx<T>>();
  cx<T>* w = wb.as<cx<T>>();
  const int32_t* part = W.part.as<int32_t>();
  int32_t* act = W.act.as<int32_t>();
  BEM_CUDA(cudaMemcpyAsync(act, part, sizeof(int32_t) * F, cudaMemcpyDeviceToDevice, st));
  BEM_CUDA(cudaMemsetAsync(s.kcols, 0, sizeof(int32_t) * F, st));
  const dim3 gv(grid_for(N, 256), (unsigned)F);
  start_kernel<T><<<dim3(grid_for(std::max<int64_t>(N, m1), 256), (unsigned)F), 256, 0, st>>>(
      W.r.as<cx<double>>(), W.rn2.as<double>(), V, N, m1, act, s.g);
  BEM_LAUNCHED();
  ctx->launches++;
  std::vector<int32_t> act_h(F), list;
  for (int64_t f = 0; f < F; ++f)
    if (part_h[f]) list.push_back((int32_t)f);
  int it = 0;
  for (int j = 0; j < m; ++j) {
    // z = M^{-1} v_j: column j of V is strided by m1 N, gather it into w first
    BEM_CUDA(cudaMemcpy2DAsync(w, sizeof(cx<T>) * N, V + (size_t)j * N, sizeof(cx<T>) * N * m1,
                               sizeof(cx<T>) * N, F, cudaMemcpyDeviceToDevice, st));
    Ops<T>::pre(ctx, w, z, act);
    Ops<T>::op(ctx, z, w, &list);
    {
    ProfScope ps(ctx, PK_VEC);
    clear_hacc_kernel<<<grid_for(F * m1, 256), 256, 0, st>>>(s.hacc, F, m1, act);
    ctx->launches++;
    for (int pass = 0; pass < 2; ++pass) {
      gs_dots_kernel<T><<<dim3(j + 1, (unsigned)F), 256, 0, st>>>(V, w, N, m1, j, act,
                                                                 W.dots.as<cx<double>>());
      ctx->launches++;
      gs_update_kernel<T><<<gv, 256, sizeof(cx<double>) * m1, st>>>(
          V, w, N, m1, j, act, W.dots.as<cx<double>>(), s.hacc);
      ctx->launches++;
    }
    norm2_kernel<T><<<(unsigned)F, 256, 0, st>>>(w, N, act, s.hnorm2);
    ctx->launches++;
    BEM_CUDA(cudaMemsetAsync(s.nact, 0, sizeof(int32_t), st));
    arnoldi_finish_kernel<<<grid_for(F, 128), 128, 0, st>>>(s, F, m, j);
    ctx->launches++;
    normalize_kernel<T><<<gv, 256, 0, st>>>(w, V, N, m1, j, act, s.inv_h);
    ctx->launches++;
    }
    BEM_LAUNCHED();
    int32_t nact = 0;
    BEM_CUDA(cudaMemcpyAsync(&nact, s.nact, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
    BEM_CUDA(cudaMemcpyAsync(act_h.data(), act, sizeof(int32_t) * F, cudaMemcpyDeviceToHost, st));
    BEM_CUDA(cudaStreamSynchronize(st));
    ++it;
    if (nact == 0) break;
    list.clear();
    for (int64_t f = 0; f < F; ++f)
      if (act_h[f]) list.push_back((int32_t)f);
  }
  // update: x += M^{-1} V y
  lsq_kernel<<<grid_for(F, 128), 128, 0, st>>>(s, F, m, part, W.y.as<cx<double>>());
  combine_kernel<T><<<gv, 256, 0, st>>>(V, W.y.as<cx<double>>(), s.kcols, N, m1, part, w);
  Ops<T>::pre(ctx, w, z, part);
  add_correction_kernel<T><<<grid_for(F * N, 256), 256, 0, st>>>(W.x, z, N, F, part);
  ctx->launches += 3;
  BEM_LAUNCHED();
  std::vector<int32_t> kc(F), ph(F);
  BEM_CUDA(cudaMemcpyAsync(kc.data(), s.kcols, sizeof(int32_t) * F, cudaMemcpyDeviceToHost, st));
  BEM_CUDA(cudaMemcpyAsync(ph.data(), part, sizeof(int32_t) * F, cudaMemcpyDeviceToHost, st));
  BEM_CUDA(cudaStreamSynchronize(st));
  for (int64_t f = 0; f < F; ++f)
    if (ph[f]) iters_host[f] += kc[f];
  return it;
}

template <class T>
void reserve_inner(DevBuf& V, DevBuf& z, DevBuf& w, int64_t F, int64_t N, int m) {
  const int m1 = m + 1;
  V.reserve(sizeof(cx<T>) * F * m1 * N);
  z.reserve(sizeof(cx<T>) * F * N);
  w.reserve(sizeof(cx<T>) * F * N);
}

}  // namespace

void solve_batch(bem_ctx* ctx, cx<double>* x_dev, bem_solve_stats* /*st*/,
                 std::vector<int32_t>& iters, std::vector<int32_t>& refines,
                 std::vector<double>& resid, std::vector<int32_t>& status) {
  const int64_t F = ctx->fs.F, N = 3 * ctx->mesh.ne;
  const bem_options& o = ctx->opt;
  const int m = std::max(1, o.restart);
  const int m1 = m + 1;
  const bool mixed = o.precision == BEM_PREC_MIXED;
  cudaStream_t st = ctx->stream;
  Work W;
  W.b.reserve(sizeof(cx<double>) * F * N);
  W.r.reserve(sizeof(cx<double>) * F * N);
  W.Ax.reserve(sizeof(cx<double>) * F * N);
  W.x = x_dev;
  if (mixed) reserve_inner<float>(W.V, W.z, W.w, F, N, m);
  else reserve_inner<double>(W.V, W.z, W.w, F, N, m);
  W.H.reserve(sizeof(cx<double>) * F * m1 * m);
  W.cs.reserve(sizeof(double) * F * m);
  W.sn.reserve(sizeof(cx<double>) * F * m);
  W.g.reserve(sizeof(cx<double>) * F * m1);
  W.hacc.reserve(sizeof(cx<double>) * F * m1);
  W.dots.reserve(sizeof(cx<double>) * F * m1);
  W.y.reserve(sizeof(cx<double>) * F * m1);
  for (DevBuf* b : {&W.hnorm2, &W.target, &W.inv_h, &W.est, &W.bn2, &W.rn2}) b->reserve(sizeof(double) * F);
  for (DevBuf* b : {&W.act, &W.part, &W.kcols, &W.status, &W.upd}) b->reserve(sizeof(int32_t) * F);
  W.nact.reserve(sizeof(int32_t));
  BEM_CUDA(cudaMemsetAsync(W.status.p, 0, sizeof(int32_t) * F, st));

  if (mixed) {
    // b in FP32 (K applied by the FP32 operator) seeds the first inner solve; the FP64 residual
    // r = K k - A x of every refinement step recomputes the data term in FP64
    known_data(ctx, W.Ax.as<cx<double>>());
    DevBuf kf, bf;
    kf.reserve(sizeof(cx<float>) * F * N);
    bf.reserve(sizeof(cx<float>) * F * N);
    narrow_array(ctx, W.Ax.as<cx<double>>(), kf.as<cx<float>>(), F * N);
    apply_operator32(ctx, kf.as<cx<float>>(), bf.as<cx<float>>(), BEM_APPLY_K, nullptr);
    widen_array(ctx, bf.as<cx<float>>(), W.r.as<cx<double>>(), F * N);
    norm2_kernel<double><<<(unsigned)F, 256, 0, st>>>(W.r.as<cx<double>>(), N, nullptr, W.bn2.as<double>());
    ctx->launches++;
  } else {
    // b = K (profile * data) in FP64
    known_data(ctx, W.Ax.as<cx<double>>());
    apply_operator64(ctx, W.Ax.as<cx<double>>(), W.b.as<cx<double>>(), BEM_APPLY_K, nullptr);
    norm2_kernel<double><<<(unsigned)F, 256, 0, st>>>(W.b.as<cx<double>>(), N, nullptr, W.bn2.as<double>());
    ctx->launches++;
    BEM_CUDA(cudaMemcpyAsync(W.r.p, W.b.p, sizeof(cx<double>) * F * N, cudaMemcpyDeviceToDevice, st));
  }
  // a sweep's passes arrive here as ZERO or VF; a sweep option on a direct call acts as VF
  const int wstart = o.warm_start == BEM_WARM_SWEEP ? BEM_WARM_VF : o.warm_start;
  const bool warm = wstart != BEM_WARM_ZERO && ctx->warm.N == N && !ctx->warm.s.empty() &&
                    (wstart != BEM_WARM_MLP || ctx->warm.trained);
  ctx->warm_learned_gains = 0;
  if (warm) {
    // direction x^ from the warm start, y = A x^ with the operator of the inner solve's
    // precision, then x0 = alpha x^ and r = b - alpha y with the alpha minimising |r|.  The
    // learned start combines its direction with the nearest stored solution (see below).
    const cx<double>* bsrc = mixed ? W.r.as<cx<double>>() : W.b.as<cx<double>>();
    auto candidate = [&](int mode, cx<double>* x, cx<double>* r, double* rn2) {
      warm_initial(ctx, mode, ctx->fs.s.data(), F, x);
      if (mixed) {
        DevBuf xf, yf;
        xf.reserve(sizeof(cx<float>) * F * N);
        yf.reserve(sizeof(cx<float>) * F * N);
        narrow_array(ctx, x, xf.as<cx<float>>(), F * N);
        apply_operator32(ctx, xf.as<cx<float>>(), yf.as<cx<float>>(), BEM_APPLY_A, nullptr);
        warm_scale_kernel<float><<<(unsigned)F, 256, 0, st>>>(bsrc, yf.as<cx<float>>(), x, r, N);
      } else {
        apply_operator64(ctx, x, W.Ax.as<cx<double>>(), BEM_APPLY_A, nullptr);
        warm_scale_kernel<double><<<(unsigned)F, 256, 0, st>>>(bsrc, W.Ax.as<cx<double>>(), x, r, N);
      }
      ctx->launches++;
      BEM_LAUNCHED();
      norm2_kernel<double><<<(unsigned)F, 256, 0, st>>>(r, N, nullptr, rn2);
      ctx->launches++;
    };
    DevBuf r1;
    r1.reserve(sizeof(cx<double>) * F * N);
    if (wstart == BEM_WARM_MLP || wstart == BEM_WARM_VF) {
      // predicted direction x1 (the network's Phi c(s), or the rational prediction of the AFS
      // fit) and nearest stored solution x2, combined as x0 = a1 x1 + a2 x2 with the (a1, a2)
      // minimising |b - A x0|: never worse than either alone
      DevBuf x2, rr;
      x2.reserve(sizeof(cx<double>) * F * N);
      rr.reserve(sizeof(double) * 2 * F);
      warm_initial(ctx, wstart, ctx->fs.s.data(), F, x_dev);
      warm_initial(ctx, BEM_WARM_NEAREST, ctx->fs.s.data(), F, x2.as<cx<double>>());
      if (mixed) {
        DevBuf xf, y1, y2;
        xf.reserve(sizeof(cx<float>) * F * N);
        y1.reserve(sizeof(cx<float>) * F * N);
        y2.reserve(sizeof(cx<float>) * F * N);
        narrow_array(ctx, x_dev, xf.as<cx<float>>(), F * N);
        apply_operator32(ctx, xf.as<cx<float>>(), y1.as<cx<float>>(), BEM_APPLY_A, nullptr);
        narrow_array(ctx, x2.as<cx<double>>(), xf.as<cx<float>>(), F * N);
        apply_operator32(ctx, xf.as<cx<float>>(), y2.as<cx<float>>(), BEM_APPLY_A, nullptr);
        warm_combine_kernel<float><<<(unsigned)F, 256, 0, st>>>(bsrc, y1.as<cx<float>>(), y2.as<cx<float>>(), x_dev,
                                                                x2.as<cx<double>>(), r1.as<cx<double>>(), N,
                                                                rr.as<double>());
        BEM_LAUNCHED();
        BEM_CUDA(cudaStreamSynchronize(st));
      } else {
        DevBuf y2;
        y2.reserve(sizeof(cx<double>) * F * N);
        apply_operator64(ctx, x_dev, W.Ax.as<cx<double>>(), BEM_APPLY_A, nullptr);
        apply_operator64(ctx, x2.as<cx<double>>(), y2.as<cx<double>>(), BEM_APPLY_A, nullptr);
        warm_combine_kernel<double><<<(unsigned)F, 256, 0, st>>>(bsrc, W.Ax.as<cx<double>>(), y2.as<cx<double>>(),
                                                                 x_dev, x2.as<cx<double>>(), r1.as<cx<double>>(), N,
                                                                 rr.as<double>());
        BEM_LAUNCHED();
        BEM_CUDA(cudaStreamSynchronize(st));
      }
      ctx->launches++;
      std::vector<double> rh(2 * F);
      BEM_CUDA(cudaMemcpy(rh.data(), rr.p, sizeof(double) * 2 * F, cudaMemcpyDeviceToHost));
      for (int64_t f = 0; f < F; ++f)
        if (rh[2 * f] < 0.81 * rh[2 * f + 1]) ctx->warm_learned_gains++;  // residual >= 10 % lower
      norm2_kernel<double><<<(unsigned)F, 256, 0, st>>>(r1.as<cx<double>>(), N, nullptr, W.rn2.as<double>());
      ctx->launches++;
    } else {
      candidate(wstart, x_dev, r1.as<cx<double>>(), W.rn2.as<double>());
    }
    BEM_CUDA(cudaMemcpyAsync(W.r.p, r1.p, sizeof(cx<double>) * F * N, cudaMemcpyDeviceToDevice, st));
    BEM_CUDA(cudaStreamSynchronize(st));
  } else {
    // x = 0, r = b
    BEM_CUDA(cudaMemsetAsync(x_dev, 0, sizeof(cx<double>) * F * N, st));
    BEM_CUDA(cudaMemcpyAsync(W.rn2.p, W.bn2.p, sizeof(double) * F, cudaMemcpyDeviceToDevice, st));
  }
  std::vector<double> bn2(F), rn2(F), est(F), tgt(F);
  std::vector<int32_t> part(F, 1), stat(F);
  BEM_CUDA(cudaMemcpyAsync(bn2.data(), W.bn2.p, sizeof(double) * F, cudaMemcpyDeviceToHost, st));
  BEM_CUDA(cudaMemcpyAsync(rn2.data(), W.rn2.p, sizeof(double) * F, cudaMemcpyDeviceToHost, st));
  BEM_CUDA(cudaStreamSynchronize(st));
  iters.assign(F, 0);
  refines.assign(F, 0);
  resid.assign(F, 1.0);
  status.assign(F, BEM_ERR_NOT_CONVERGED);
  std::vector<char> done(F, 0);
  std::vector<char> full_done(F, 0);  // the full residual has been formed once
  std::vector<double> prev_rel(F, 1.0);
  for (int64_t f = 0; f < F; ++f)
    if (bn2[f] == 0.0) {  // zero right-hand side: x = 0 is exact
      done[f] = 1;
      resid[f] = 0.0;
      status[f] = 0;
    }

  // Plain FP64 GMRES(m) on the frequencies not done: restarted cycles, each accepted when the FP64
  // GMRES residual estimate meets the tolerance, else restarted from the true FP64 residual.
  auto fp64_loop = [&](DevBuf& Vb, DevBuf& zb, DevBuf& wb) {
    const int max_cycles = std::max(1, o.max_iters / m + 1);
    int total = 0;
    for (int cycle = 0; cycle < max_cycles; ++cycle) {
      int64_t nwork = 0;
      for (int64_t f = 0; f < F; ++f) {
        part[f] = done[f] ? 0 : 1;
        nwork += part[f];
        tgt[f] = 0.999 * o.tol * std::sqrt(bn2[f]);
      }
      if (nwork == 0 || total >= o.max_iters) break;
      BEM_CUDA(cudaMemcpyAsync(W.target.p, tgt.data(), sizeof(double) * F, cudaMemcpyHostToDevice, st));
      BEM_CUDA(cudaMemcpyAsync(W.part.p, part.data(), sizeof(int32_t) * F, cudaMemcpyHostToDevice, st));
      total += gmres_cycle<double>(ctx, W, Vb, zb, wb, F, N, m, iters, part);
      BEM_CUDA(cudaMemcpyAsync(est.data(), W.est.p, sizeof(double) * F, cudaMemcpyDeviceToHost, st));
      BEM_CUDA(cudaMemcpyAsync(stat.data(), W.status.p, sizeof(int32_t) * F, cudaMemcpyDeviceToHost, st));
      BEM_CUDA(cudaStreamSynchronize(st));
      std::vector<int32_t> rlist;
      for (int64_t f = 0; f < F; ++f) {
        if (!part[f]) continue;
        const double rel = est[f] / std::sqrt(bn2[f]);
        resid[f] = rel;
        if (stat[f] == BEM_ERR_BREAKDOWN) {
          done[f] = 1;
          status[f] = BEM_ERR_BREAKDOWN;
        } else if (est[f] <= o.tol * std::sqrt(bn2[f])) {
          done[f] = 1;
          status[f] = 0;
        } else {
          rlist.push_back((int32_t)f);
        }
        part[f] = done[f] ? 0 : 1;
      }
      if (rlist.empty()) break;
      // restart from the true residual
      BEM_CUDA(cudaMemcpyAsync(W.part.p, part.data(), sizeof(int32_t) * F, cudaMemcpyHostToDevice, st));
      if (ctx->fp64_op_df) residual_df(ctx, x_dev, W.r.as<cx<double>>(), &rlist);
      else residual64(ctx, x_dev, W.r.as<cx<double>>(), &rlist);
      norm2_kernel<double><<<(unsigned)F, 256, 0, st>>>(W.r.as<cx<double>>(), N, W.part.as<int32_t>(),
                                                        W.rn2.as<double>());
      ctx->launches++;
      BEM_LAUNCHED();
      for (int32_t f : rlist) refines[f]++;
    }
  };

  if (!mixed) {
    fp64_loop(W.V, W.z, W.w);
    return;
  }

  // Mixed: FP32 inner GMRES(m) solves to a relative inner tolerance, each followed by an
  // FP64-class residual, until that residual meets the tolerance.
  std::vector<char> fallback(F, 0);
  const int max_outer = std::max(1, o.max_refine);
  int total_inner = 0;
  for (int outer = 0; outer < max_outer; ++outer) {
    int64_t nwork = 0;
    for (int64_t f = 0; f < F; ++f) {
      part[f] = done[f] ? 0 : 1;
      nwork += part[f];
      const double rn = std::sqrt(rn2[f]), bnrm = std::sqrt(bn2[f]);
      // The first inner solve stops at 0.8 tol: below that its own residual drops under the FP32
      // operator's error floor (~1e-6 at the top of the band), so further iterations are lost to
      // the refinement that follows anyway.  Later solves correct a small d, whose FP32 product
      // is accurate, and stop at 0.5 tol.  The relative reduction inner_tol is measured against
      // |b| in the first solve: its right-hand side and, after a warm start, its initial residual
      // b - alpha A x^ carry the FP32 operator's error (~1e-7 |b|), so a reduction relative to a
      // small warm-start residual would chase that error.  Later solves start from an FP64-class
      // residual and reduce it by inner_tol.
      tgt[f] = std::max(o.inner_tol * (full_done[f] ? rn : bnrm), (full_done[f] ? 0.5 : 0.8) * o.tol * bnrm);
    }
    if (nwork == 0) break;
    if (total_inner >= o.max_iters) break;
    BEM_CUDA(cudaMemcpyAsync(W.target.p, tgt.data(), sizeof(double) * F, cudaMemcpyHostToDevice, st));
    BEM_CUDA(cudaMemcpyAsync(W.part.p, part.data(), sizeof(int32_t) * F, cudaMemcpyHostToDevice, st));
    total_inner += gmres_cycle<float>(ctx, W, W.V, W.z, W.w, F, N, m, iters, part);
    BEM_CUDA(cudaMemcpyAsync(stat.data(), W.status.p, sizeof(int32_t) * F, cudaMemcpyDeviceToHost, st));
    BEM_CUDA(cudaStreamSynchronize(st));
    for (int64_t f = 0; f < F; ++f)
      if (part[f] && stat[f] == BEM_ERR_BREAKDOWN) {
        done[f] = 1;
        part[f] = 0;
        status[f] = BEM_ERR_BREAKDOWN;
      }
    // FP64-class residual r = b - A x for the instances still working
    BEM_CUDA(cudaMemcpyAsync(W.part.p, part.data(), sizeof(int32_t) * F, cudaMemcpyHostToDevice, st));
    {
      std::vector<int32_t> upd(F);
      for (int64_t f = 0; f < F; ++f) upd[f] = (part[f] && full_done[f]) ? 1 : 0;
      BEM_CUDA(cudaMemcpyAsync(W.upd.p, upd.data(), sizeof(int32_t) * F, cudaMemcpyHostToDevice, st));
    }
    std::vector<int32_t> rlist, ulist, flist;
    for (int64_t f = 0; f < F; ++f)
      if (part[f]) {
        rlist.push_back((int32_t)f);
        (full_done[f] ? ulist : flist).push_back((int32_t)f);
      }
    if (rlist.empty()) break;
    // First refinement step of a frequency: the full FP64-class residual r = b - A x.  Later
    // steps update it, r <- r - A d, with the correction d of the inner solve applied in the
    // inner solve's precision: d is small (|d| ~ kappa |r| / |A|), so the product's rounding,
    // ~eps_32 |A| |d|, stays ~1e-10 |b| below the tolerance being certified.
    if (!flist.empty()) {
      if (o.residual_mode == BEM_RESID_DF64) residual_df(ctx, x_dev, W.r.as<cx<double>>(), &flist);
      else residual64(ctx, x_dev, W.r.as<cx<double>>(), &flist);
    }
    if (!ulist.empty()) {
      apply_operator32(ctx, W.z.as<cx<float>>(), W.w.as<cx<float>>(), BEM_APPLY_A, &ulist);
      sub_widen_masked_kernel<<<grid_for(F * N, 256), 256, 0, st>>>(W.r.as<cx<double>>(), W.w.as<cx<float>>(),
                                                                     W.upd.as<int32_t>(), N, F * N);
      ctx->launches++;
    }
    for (int32_t f : flist) full_done[f] = 1;
    norm2_kernel<double><<<(unsigned)F, 256, 0, st>>>(W.r.as<cx<double>>(), N, W.part.as<int32_t>(),
                                                      W.rn2.as<double>());
    ctx->launches += 1;
    BEM_LAUNCHED();
    BEM_CUDA(cudaMemcpyAsync(rn2.data(), W.rn2.p, sizeof(double) * F, cudaMemcpyDeviceToHost, st));
    BEM_CUDA(cudaStreamSynchronize(st));
    for (int64_t f = 0; f < F; ++f) {
      if (!part[f]) continue;
      refines[f]++;
      const double rel = std::sqrt(rn2[f] / bn2[f]);
      resid[f] = rel;
      if (!std::isfinite(rel)) {
        done[f] = 1;
        status[f] = BEM_ERR_BREAKDOWN;
      } else if (rel <= o.tol) {
        done[f] = 1;
        status[f] = 0;
      } else if (refines[f] >= 2 && rel > 0.25 * prev_rel[f]) {
        // refinement stalled (a healthy step gains >= 10x): the FP32 operator is too inaccurate
        // for this frequency, |A - A_32| |A^{-1}| near 1
        done[f] = 1;
        fallback[f] = 1;
      }
      prev_rel[f] = rel;
    }
  }
  // Stalled or unconverged frequencies: a fresh FP64 solve from x = 0 (a restarted GMRES from
  // the mixed iterate can stagnate where one from zero converges), with the FP64 right-hand side
  // and its result certified by the native FP64 residual.
  std::vector<int32_t> fl;
  for (int64_t f = 0; f < F; ++f)
    if (fallback[f] || (status[f] == BEM_ERR_NOT_CONVERGED && !done[f])) fl.push_back((int32_t)f);
  if (fl.empty()) return;
  for (int64_t f = 0; f < F; ++f) done[f] = 1;
  for (int32_t f : fl) {
    done[f] = 0;
    part[f] = 1;
    status[f] = BEM_ERR_NOT_CONVERGED;
  }
  BEM_CUDA(cudaMemcpyAsync(W.part.p, part.data(), sizeof(int32_t) * F, cudaMemcpyHostToDevice, st));
  known_data(ctx, W.Ax.as<cx<double>>());
  apply_operator64(ctx, W.Ax.as<cx<double>>(), W.b.as<cx<double>>(), BEM_APPLY_K, &fl);
  for (int32_t f : fl) {
    BEM_CUDA(cudaMemsetAsync(x_dev + (int64_t)f * N, 0, sizeof(cx<double>) * N, st));
    BEM_CUDA(cudaMemcpyAsync(W.r.as<cx<double>>() + (int64_t)f * N, W.b.as<cx<double>>() + (int64_t)f * N,
                             sizeof(cx<double>) * N, cudaMemcpyDeviceToDevice, st));
  }
  {
    std::vector<int32_t> sel(F, 0);
    for (int32_t f : fl) sel[f] = 1;
    BEM_CUDA(cudaMemcpyAsync(W.part.p, sel.data(), sizeof(int32_t) * F, cudaMemcpyHostToDevice, st));
    norm2_kernel<double><<<(unsigned)F, 256, 0, st>>>(W.b.as<cx<double>>(), N, W.part.as<int32_t>(),
                                                      W.bn2.as<double>());
    ctx->launches++;
    BEM_CUDA(cudaMemcpyAsync(W.rn2.p, W.bn2.p, sizeof(double) * F, cudaMemcpyDeviceToDevice, st));
    BEM_CUDA(cudaMemcpyAsync(bn2.data(), W.bn2.p, sizeof(double) * F, cudaMemcpyDeviceToHost, st));
    BEM_CUDA(cudaStreamSynchronize(st));
  }
  reserve_inner<double>(W.V64, W.z64, W.w64, F, N, m);
  // the fallback's operator: float-float (FP64-class to ~1e-10, several times faster than the
  // FP64 unit) when the tolerance leaves room for that, native FP64 below 1e-8
  struct DfOpScope {
    bem_ctx* c;
    DfOpScope(bem_ctx* c_, bool on) : c(c_) { c->fp64_op_df = on; }
    ~DfOpScope() { c->fp64_op_df = false; }
  } df_scope(ctx, o.tol >= 1e-8);
  fp64_loop(W.V64, W.z64, W.w64);
  // certify with the true FP64 residual
  {
    std::vector<int32_t> sel(F, 0);
    for (int32_t f : fl) sel[f] = 1;
    BEM_CUDA(cudaMemcpyAsync(W.part.p, sel.data(), sizeof(int32_t) * F, cudaMemcpyHostToDevice, st));
    residual64(ctx, x_dev, W.r.as<cx<double>>(), &fl);
    norm2_kernel<double><<<(unsigned)F, 256, 0, st>>>(W.r.as<cx<double>>(), N, W.part.as<int32_t>(),
                                                      W.rn2.as<double>());
    ctx->launches++;
    BEM_CUDA(cudaMemcpyAsync(rn2.data(), W.rn2.p, sizeof(double) * F, cudaMemcpyDeviceToHost, st));
    BEM_CUDA(cudaStreamSynchronize(st));
    for (int32_t f : fl) {
      refines[f]++;
      const double rel = std::sqrt(rn2[f] / bn2[f]);
      resid[f] = rel;
      if (status[f] != BEM_ERR_BREAKDOWN) status[f] = rel <= o.tol ? 0 : BEM_ERR_NOT_CONVERGED;
    }
  }
}

}  // namespace bem
