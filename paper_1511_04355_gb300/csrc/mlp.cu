// Learned warm start for the frequency solves (not part of the paper; the paper's adaptive
// sampling of Sec. 3 solves one new frequency at a time, next to frequencies already solved).
//
// Memory: solutions x(s_j) of solved frequencies (FP64 on the device).
// POD:    Phi = the r leading left singular vectors of X = [x(s_1) .. x(s_J)]: Gram matrix
//         G = X^H X on the device (FP64), eigenpairs of G on the host (cyclic complex Jacobi with
//         a relative stopping test), Phi_k = X v_k / sigma_k; r is the
//         smallest rank whose discarded energy is <= energy_tol * trace(G).  The Gram route
//         resolves sigma_k only down to ~1e-8 sigma_1, so energy_tol must stay well above 1e-16.
// MLP:    u = (Re s, Im s) / Omega -> 128 -> 128 -> 2r (tanh-GELU), trained on the device to
//         predict the direction of c_j = Phi^H x(s_j): c_j / |c_j| turned so that its first entry
//         is real and non-negative.  Each target then has unit size whatever |x(s_j)|, which the
//         FP16 products need: solution norms span decades over a frequency band, and a common
//         scale would leave the small ones below FP16 resolution.  MSE loss and Adam: FP32 master weights; the
//         three dense layers' products run on the tensor cores (mma.sync m16n8k16, FP16
//         operands, FP32 accumulation), elementwise parts in FP32.  The products are tiny
//         (at most 256 x 128 x 256), so one warp computes one 16 x 8 output tile.
// Warm start: the direction x^(s) = Phi c(s) (BEM_WARM_MLP) or the stored solution at the
//         nearest solved frequency (BEM_WARM_NEAREST); the solver scales it by the complex alpha
//         minimising |b - alpha A x^| (warm_scale).
#include <algorithm>
#include <chrono>
#include <cuda_fp16.h>
#include <random>

#include "kernel_math.cuh"

namespace bem {

constexpr int kHidden = 128;
constexpr float kGeluC = 0.7978845608028654f;  // sqrt(2/pi)

// ------------------------------------------------------------------------------- tensor-core GEMM
// C[m, n] = beta C[m, n] + sum_k A(m, k) B(k, n), with A(m, k) = A[m lam + k lak] and
// B(k, n) = B[k lbk + n lbn] (FP32 in memory, rounded to FP16 for the MMA), C row-major (ldc).
__global__ void mma_gemm_kernel(const float* A, int lam, int lak, const float* B, int lbk, int lbn,
                                float* C, int ldc, int M, int N, int K, float beta) {
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  const int tiles_n = (N + 7) / 8;
  const int tm = warp / tiles_n, tn = warp % tiles_n;
  if (tm * 16 >= M) return;
  const int gid = lane >> 2, tig = lane & 3;
  const int r0 = tm * 16 + gid, r1 = r0 + 8, col = tn * 8 + gid;
  auto a_at = [&](int m, int k) -> float { return (m < M && k < K) ? A[(int64_t)m * lam + (int64_t)k * lak] : 0.f; };
  auto b_at = [&](int k, int n) -> float { return (k < K && n < N) ? B[(int64_t)k * lbk + (int64_t)n * lbn] : 0.f; };
  float d0 = 0.f, d1 = 0.f, d2 = 0.f, d3 = 0.f;
  for (int k0 = 0; k0 < K; k0 += 16) {
    const int c0 = k0 + tig * 2, c2 = k0 + 8 + tig * 2;
    const __half2 a01 = __floats2half2_rn(a_at(r0, c0), a_at(r0, c0 + 1));
    const __half2 a23 = __floats2half2_rn(a_at(r1, c0), a_at(r1, c0 + 1));
    const __half2 a45 = __floats2half2_rn(a_at(r0, c2), a_at(r0, c2 + 1));
    const __half2 a67 = __floats2half2_rn(a_at(r1, c2), a_at(r1, c2 + 1));
    const __half2 b01 = __floats2half2_rn(b_at(c0, col), b_at(c0 + 1, col));
    const __half2 b23 = __floats2half2_rn(b_at(c2, col), b_at(c2 + 1, col));
    const unsigned ra0 = *reinterpret_cast<const unsigned*>(&a01);
    const unsigned ra1 = *reinterpret_cast<const unsigned*>(&a23);
    const unsigned ra2 = *reinterpret_cast<const unsigned*>(&a45);
    const unsigned ra3 = *reinterpret_cast<const unsigned*>(&a67);
    const unsigned rb0 = *reinterpret_cast<const unsigned*>(&b01);
    const unsigned rb1 = *reinterpret_cast<const unsigned*>(&b23);
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.f16.f16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};\n"
        : "+f"(d0), "+f"(d1), "+f"(d2), "+f"(d3)
        : "r"(ra0), "r"(ra1), "r"(ra2), "r"(ra3), "r"(rb0), "r"(rb1));
  }
  const int cc = tn * 8 + tig * 2;
  auto store = [&](int m, int n, float v) {
    if (m < M && n < N) {
      float* p = C + (int64_t)m * ldc + n;
      *p = (beta == 0.f ? 0.f : beta * *p) + v;
    }
  };
  store(r0, cc, d0);
  store(r0, cc + 1, d1);
  store(r1, cc, d2);
  store(r1, cc + 1, d3);
}

static void gemm(cudaStream_t st, const float* A, int lam, int lak, const float* B, int lbk, int lbn,
                 float* C, int ldc, int M, int N, int K, float beta, int64_t& launches) {
  const int warps = ((M + 15) / 16) * ((N + 7) / 8);
  mma_gemm_kernel<<<grid_for((int64_t)warps * 32, 128), 128, 0, st>>>(A, lam, lak, B, lbk, lbn, C, ldc,
                                                                     M, N, K, beta);
  BEM_LAUNCHED();
  ++launches;
}

// ------------------------------------------------------------------------------- elementwise
__device__ __forceinline__ float gelu_f(float x) {
  return 0.5f * x * (1.f + tanhf(kGeluC * (x + 0.044715f * x * x * x)));
}
__device__ __forceinline__ float gelu_d(float x) {
  const float t = tanhf(kGeluC * (x + 0.044715f * x * x * x));
  return 0.5f * (1.f + t) + 0.5f * x * (1.f - t * t) * kGeluC * (1.f + 3.f * 0.044715f * x * x);
}

// layer 1 (fan-in 2) on the CUDA cores: Z1 = U W1^T + b1, H1 = g(Z1)
__global__ void layer1_kernel(const float* U, const float* W1, const float* b1, float* Z1, float* H1, int B) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= B * kHidden) return;
  const int b = t / kHidden, j = t % kHidden;
  const float z = fmaf(U[2 * b], W1[2 * j], fmaf(U[2 * b + 1], W1[2 * j + 1], b1[j]));
  Z1[t] = z;
  H1[t] = gelu_f(z);
}

// X[b][j] += bias[j]; optionally H = g(X)
__global__ void bias_act_kernel(float* X, const float* bias, float* H, int B, int n) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= B * n) return;
  const float z = X[t] + bias[t % n];
  X[t] = z;
  if (H) H[t] = gelu_f(z);
}

// dY = (Y - T) / B, loss += 0.5 |Y - T|^2 / B
__global__ void loss_kernel(const float* Y, const float* T, float* dY, int n, int B, double* loss) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n) return;
  const float d = Y[t] - T[t];
  dY[t] = d / B;
  atomicAdd(loss, 0.5 * (double)d * (double)d / B);
}

// dZ = dH * g'(Z)
__global__ void act_back_kernel(const float* dH, const float* Z, float* dZ, int n) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t < n) dZ[t] = dH[t] * gelu_d(Z[t]);
}

// column sums: out[j] = sum_b X[b][j]
__global__ void colsum_kernel(const float* X, float* out, int B, int n) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n) return;
  float s = 0.f;
  for (int b = 0; b < B; ++b) s += X[b * n + j];
  out[j] = s;
}

// dW1[j][c] = sum_b dZ1[b][j] U[b][c]
__global__ void dw1_kernel(const float* dZ1, const float* U, float* dW1, int B) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= 2 * kHidden) return;
  const int j = t / 2, c = t % 2;
  float s = 0.f;
  for (int b = 0; b < B; ++b) s += dZ1[b * kHidden + j] * U[2 * b + c];
  dW1[t] = s;
}

__global__ void adam_kernel(float* w, const float* g, float* m, float* v, int n, float lr, float b1,
                            float b2, float c1, float c2, float eps) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n) return;
  const float gg = g[t];
  const float mm = b1 * m[t] + (1.f - b1) * gg;
  const float vv = b2 * v[t] + (1.f - b2) * gg * gg;
  m[t] = mm;
  v[t] = vv;
  w[t] -= lr * (mm / c1) / (sqrtf(vv / c2) + eps);
}

// ------------------------------------------------------------------------------- POD kernels
// G[a][b] = sum_n conj(X_a[n]) X_b[n] (one block per (a, b), a <= b)
__global__ void gram_kernel(const cx<double>* X, int64_t N, int J, cx<double>* G) {
  __shared__ double sr[256], si[256];
  const int a = blockIdx.x, b = blockIdx.y;
  if (a > b) return;
  double r = 0, im = 0;
  for (int64_t n = threadIdx.x; n < N; n += blockDim.x) {
    const cx<double> u = X[(int64_t)a * N + n], v = X[(int64_t)b * N + n];
    r += u.r * v.r + u.i * v.i;
    im += u.r * v.i - u.i * v.r;
  }
  sr[threadIdx.x] = r;
  si[threadIdx.x] = im;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if ((int)threadIdx.x < s) {
      sr[threadIdx.x] += sr[threadIdx.x + s];
      si[threadIdx.x] += si[threadIdx.x + s];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    G[a * J + b] = mk(sr[0], si[0]);
    G[b * J + a] = mk(sr[0], -si[0]);
  }
}

// Phi[k][n] = sum_j X[j][n] V[j][k]  (V already divided by sigma_k)
__global__ void combine_basis_kernel(const cx<double>* X, const cx<double>* V, int64_t N, int J, int r,
                                     cx<double>* Phi) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= N * r) return;
  const int k = (int)(t / N);
  const int64_t n = t % N;
  cx<double> s = mk(0.0, 0.0);
  for (int j = 0; j < J; ++j) s = cfma(X[(int64_t)j * N + n], V[j * r + k], s);
  Phi[t] = s;
}

// x0[f][n] = sum_k (y[f][k] + i y[f][r + k]) Phi[k][n]
__global__ void expand_kernel(const float* y, const cx<double>* Phi, int64_t N, int r, int F, cx<double>* x0) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= N * F) return;
  const int f = (int)(t / N);
  const int64_t n = t % N;
  cx<double> s = mk(0.0, 0.0);
  for (int k = 0; k < r; ++k)
    s = cfma(mk((double)y[f * 2 * r + k], (double)y[f * 2 * r + r + k]), Phi[(int64_t)k * N + n], s);
  x0[t] = s;
}

// x0[f][n] = sum_j w[f][j] X[j][n]: the rational prediction from the stored solutions
__global__ void weighted_sum_kernel(const cx<double>* w, const cx<double>* X, int64_t N, int64_t J, int64_t F,
                                    cx<double>* x0) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= N * F) return;
  const int64_t f = t / N, n = t % N;
  cx<double> s = mk(0.0, 0.0);
  for (int64_t j = 0; j < J; ++j) s = cfma(w[f * J + j], X[j * N + n], s);
  x0[t] = s;
}

// C[j][k] = (Phi^H x_j)_k (one block per (j, k))
__global__ void project_kernel(const cx<double>* Phi, const cx<double>* X, int64_t N, int r, cx<double>* C) {
  __shared__ double sr[256], si[256];
  const int j = blockIdx.x, k = blockIdx.y;
  double a = 0, b = 0;
  for (int64_t n = threadIdx.x; n < N; n += blockDim.x) {
    const cx<double> p = Phi[(int64_t)k * N + n], x = X[(int64_t)j * N + n];
    a += p.r * x.r + p.i * x.i;
    b += p.r * x.i - p.i * x.r;
  }
  sr[threadIdx.x] = a;
  si[threadIdx.x] = b;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if ((int)threadIdx.x < s) {
      sr[threadIdx.x] += sr[threadIdx.x + s];
      si[threadIdx.x] += si[threadIdx.x + s];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) C[j * r + k] = mk(sr[0], si[0]);
}

// ------------------------------------------------------------------------------- host helpers
namespace {

// Eigen-decomposition of a Hermitian n x n matrix (row-major) by cyclic complex Jacobi
// rotations: eigenvalues in w, eigenvectors in the columns of V.  A pair (p, q) is rotated while
// |a_pq| > 1e-15 sqrt(a_pp a_qq) (a relative criterion, so that small eigenvalues of a Gram
// matrix keep high relative accuracy, Demmel and Veselic), until a sweep rotates nothing.
// Rotation: with a_pq = m e^{i phi}, R = diag(1, e^{-i phi}) P(theta), P the real Jacobi rotation
// that annihilates the now real off-diagonal entry m; A <- R^H A R, V <- V R.
void hermitian_jacobi(int n, std::vector<cx<double>>& A, std::vector<double>& w, std::vector<cx<double>>& V) {
  V.assign((size_t)n * n, mk(0.0, 0.0));
  for (int i = 0; i < n; ++i) V[(size_t)i * n + i] = mk(1.0, 0.0);
  auto a = [&](int i, int j) -> cx<double>& { return A[(size_t)i * n + j]; };
  for (int sweep = 0; sweep < 100; ++sweep) {
    bool rotated = false;
    for (int p = 0; p < n - 1; ++p)
      for (int q = p + 1; q < n; ++q) {
        const cx<double> apq = a(p, q);
        const double m = std::hypot(apq.r, apq.i);
        const double app = a(p, p).r, aqq = a(q, q).r;
        if (m <= 1e-300 || m <= 1e-15 * std::sqrt(std::fabs(app * aqq))) continue;
        rotated = true;
        const cx<double> ph = mk(apq.r / m, apq.i / m);  // e^{i phi}
        const cx<double> phc = conj(ph);
        const double theta = (aqq - app) / (2.0 * m);
        const double t = (theta >= 0 ? 1.0 : -1.0) / (std::fabs(theta) + std::sqrt(theta * theta + 1.0));
        const double c = 1.0 / std::sqrt(t * t + 1.0), sn = t * c;
        for (int k = 0; k < n; ++k) {  // columns: A R
          const cx<double> akp = a(k, p), akq = phc * a(k, q);
          a(k, p) = c * akp - sn * akq;
          a(k, q) = sn * akp + c * akq;
        }
        for (int k = 0; k < n; ++k) {  // rows: R^H (A R)
          const cx<double> apk = a(p, k), aqk = ph * a(q, k);
          a(p, k) = c * apk - sn * aqk;
          a(q, k) = sn * apk + c * aqk;
        }
        a(p, q) = mk(0.0, 0.0);
        a(q, p) = mk(0.0, 0.0);
        a(p, p).i = 0.0;
        a(q, q).i = 0.0;
        for (int k = 0; k < n; ++k) {  // V R
          const cx<double> vkp = V[(size_t)k * n + p], vkq = phc * V[(size_t)k * n + q];
          V[(size_t)k * n + p] = c * vkp - sn * vkq;
          V[(size_t)k * n + q] = sn * vkp + c * vkq;
        }
      }
    if (!rotated) break;
  }
  w.resize(n);
  for (int i = 0; i < n; ++i) w[i] = a(i, i).r;
}

int64_t n_params(int r) { return 2 * kHidden + kHidden + kHidden * kHidden + kHidden + 2 * r * kHidden + 2 * r; }

struct ParamView {
  float *W1, *b1, *W2, *b2, *W3, *b3;
};
ParamView view(float* p, int r) {
  ParamView v;
  v.W1 = p;
  v.b1 = v.W1 + 2 * kHidden;
  v.W2 = v.b1 + kHidden;
  v.b2 = v.W2 + kHidden * kHidden;
  v.W3 = v.b2 + kHidden;
  v.b3 = v.W3 + 2 * r * kHidden;
  return v;
}

// Forward (and optionally backward) of the MLP for a batch: U (B x 2), T (B x 2r) targets.
void mlp_pass(bem_ctx* ctx, float* params, int r, const float* U, int B, const float* T, float* Y,
              float* grads, double* loss_dev) {
  WarmStart& ws = ctx->warm;
  cudaStream_t st = ctx->stream;
  const int n3 = 2 * r;
  ws.act.reserve(sizeof(float) * (size_t)B * (4 * kHidden + 2 * n3 + 2 * kHidden));
  float* Z1 = ws.act.as<float>();
  float* H1 = Z1 + (size_t)B * kHidden;
  float* Z2 = H1 + (size_t)B * kHidden;
  float* H2 = Z2 + (size_t)B * kHidden;
  float* dY = H2 + (size_t)B * kHidden;
  float* dH = dY + (size_t)B * n3;   // reused for dH2 / dZ2 / dH1 / dZ1 (B x 128 each)
  float* dZ = dH + (size_t)B * kHidden;
  ParamView p = view(params, r);
  int64_t& L = ctx->launches;
  layer1_kernel<<<grid_for((int64_t)B * kHidden, 256), 256, 0, st>>>(U, p.W1, p.b1, Z1, H1, B);
  ++L;
  gemm(st, H1, kHidden, 1, p.W2, 1, kHidden, Z2, kHidden, B, kHidden, kHidden, 0.f, L);
  bias_act_kernel<<<grid_for((int64_t)B * kHidden, 256), 256, 0, st>>>(Z2, p.b2, H2, B, kHidden);
  ++L;
  gemm(st, H2, kHidden, 1, p.W3, 1, kHidden, Y, n3, B, n3, kHidden, 0.f, L);
  bias_act_kernel<<<grid_for((int64_t)B * n3, 256), 256, 0, st>>>(Y, p.b3, nullptr, B, n3);
  ++L;
  BEM_LAUNCHED();
  if (!grads) return;
  ParamView g = view(grads, r);
  loss_kernel<<<grid_for((int64_t)B * n3, 256), 256, 0, st>>>(Y, T, dY, B * n3, B, loss_dev);
  ++L;
  gemm(st, dY, 1, n3, H2, kHidden, 1, g.W3, kHidden, n3, kHidden, B, 0.f, L);  // dW3 = dY^T H2
  colsum_kernel<<<grid_for(n3, 128), 128, 0, st>>>(dY, g.b3, B, n3);
  ++L;
  gemm(st, dY, n3, 1, p.W3, kHidden, 1, dH, kHidden, B, kHidden, n3, 0.f, L);   // dH2 = dY W3
  act_back_kernel<<<grid_for((int64_t)B * kHidden, 256), 256, 0, st>>>(dH, Z2, dZ, B * kHidden);
  ++L;
  gemm(st, dZ, 1, kHidden, H1, kHidden, 1, g.W2, kHidden, kHidden, kHidden, B, 0.f, L);  // dW2
  colsum_kernel<<<grid_for(kHidden, 128), 128, 0, st>>>(dZ, g.b2, B, kHidden);
  ++L;
  gemm(st, dZ, kHidden, 1, p.W2, kHidden, 1, dH, kHidden, B, kHidden, kHidden, 0.f, L);  // dH1
  act_back_kernel<<<grid_for((int64_t)B * kHidden, 256), 256, 0, st>>>(dH, Z1, dZ, B * kHidden);
  ++L;
  dw1_kernel<<<grid_for(2 * kHidden, 128), 128, 0, st>>>(dZ, U, g.W1, B);
  colsum_kernel<<<grid_for(kHidden, 128), 128, 0, st>>>(dZ, g.b1, B, kHidden);
  L += 2;
  BEM_LAUNCHED();
}

}  // namespace

// ------------------------------------------------------------------------------- public
void warm_store(bem_ctx* ctx, const double* s, int64_t ns, const cx<double>* x_dev) {
  WarmStart& ws = ctx->warm;
  const int64_t N = 3 * ctx->mesh.ne;
  if (ws.N != N) {
    ws.s.clear();
    ws.N = N;
    ws.trained = false;
  }
  const int64_t old = (int64_t)ws.s.size() / 2;
  const int64_t cap = old + ns;
  DevBuf grown;
  grown.reserve(sizeof(cx<double>) * cap * N);
  if (old) BEM_CUDA(cudaMemcpyAsync(grown.p, ws.X.p, sizeof(cx<double>) * old * N, cudaMemcpyDeviceToDevice, ctx->stream));
  BEM_CUDA(cudaMemcpyAsync(grown.as<cx<double>>() + old * N, x_dev, sizeof(cx<double>) * ns * N,
                           cudaMemcpyDefault, ctx->stream));
  BEM_CUDA(cudaStreamSynchronize(ctx->stream));
  std::swap(ws.X.p, grown.p);
  std::swap(ws.X.bytes, grown.bytes);
  ws.s.insert(ws.s.end(), s, s + 2 * ns);
  // a trained model stays usable: its basis and network describe the solutions stored when it
  // was trained; bem_warm_train refits it to the grown memory
}

void warm_train(bem_ctx* ctx, const bem_warm_params& prm, bem_warm_stats* out) {
  WarmStart& ws = ctx->warm;
  const int64_t N = ws.N;
  const int J = (int)(ws.s.size() / 2);
  BEM_REQUIRE(J >= 2, "the warm-start memory holds fewer than 2 solutions");
  BEM_REQUIRE(J <= 256, "the warm-start memory holds more than 256 solutions");
  cudaStream_t st = ctx->stream;
  const auto t0 = std::chrono::steady_clock::now();
  // POD: Gram matrix on the device, Jacobi on the host
  DevBuf G;
  G.reserve(sizeof(cx<double>) * J * J);
  gram_kernel<<<dim3(J, J), 256, 0, st>>>(ws.X.as<cx<double>>(), N, J, G.as<cx<double>>());
  BEM_LAUNCHED();
  ctx->launches++;
  std::vector<cx<double>> Gh((size_t)J * J);
  copy_out(ctx, Gh.data(), G.p, sizeof(cx<double>) * J * J);
  std::vector<double> w;
  std::vector<cx<double>> V;
  std::vector<cx<double>> Gw(Gh);
  hermitian_jacobi(J, Gw, w, V);
  std::vector<int> order(J);
  for (int i = 0; i < J; ++i) order[i] = i;
  std::sort(order.begin(), order.end(), [&](int a, int b) { return w[a] > w[b]; });
  double total = 0;  // trace(G) = sum_k sigma_k^2
  for (int j = 0; j < J; ++j) total += Gh[(size_t)j * J + j].r;
  std::vector<int> pick;
  double kept = 0;
  for (int idx : order) {
    if ((int)pick.size() >= prm.r_max || w[idx] <= 0.0) break;
    if (total - kept <= prm.energy_tol * total) break;
    pick.push_back(idx);
    kept += w[idx];
  }
  const int r = (int)pick.size();
  BEM_REQUIRE(r >= 1, "POD found no basis vector");
  std::vector<cx<double>> Vs((size_t)J * r);
  for (int k = 0; k < r; ++k) {
    const double sg = std::sqrt(w[pick[k]]);
    for (int j = 0; j < J; ++j) {
      const cx<double> v = V[(size_t)j * J + pick[k]];
      Vs[(size_t)j * r + k] = mk(v.r / sg, v.i / sg);
    }
  }
  DevBuf dV;
  dV.reserve(sizeof(cx<double>) * J * r);
  copy_in(ctx, dV.p, Vs.data(), sizeof(cx<double>) * J * r);
  DevBuf Phi0;
  Phi0.reserve(sizeof(cx<double>) * r * N);
  combine_basis_kernel<<<grid_for(N * r, 256), 256, 0, st>>>(ws.X.as<cx<double>>(), dV.as<cx<double>>(), N, J, r,
                                                              Phi0.as<cx<double>>());
  BEM_LAUNCHED();
  ctx->launches++;
  // The Gram matrix carries rounding ~eps sigma_1^2, so X v_k / sigma_k is orthonormal only to
  // ~eps sigma_1^2 / sigma_r^2.  One Cholesky pass restores it: M = Phi^H Phi = L L^H,
  // Phi <- Phi L^{-H} (same subspace).
  {
    DevBuf dM;
    dM.reserve(sizeof(cx<double>) * r * r);
    gram_kernel<<<dim3(r, r), 256, 0, st>>>(Phi0.as<cx<double>>(), N, r, dM.as<cx<double>>());
    BEM_LAUNCHED();
    ctx->launches++;
    std::vector<cx<double>> M((size_t)r * r), L((size_t)r * r, mk(0.0, 0.0)), Li((size_t)r * r, mk(0.0, 0.0));
    copy_out(ctx, M.data(), dM.p, sizeof(cx<double>) * r * r);
    for (int j = 0; j < r; ++j) {
      double d = M[(size_t)j * r + j].r;
      for (int k = 0; k < j; ++k) d -= L[(size_t)j * r + k].r * L[(size_t)j * r + k].r + L[(size_t)j * r + k].i * L[(size_t)j * r + k].i;
      BEM_REQUIRE(d > 0, "POD basis re-orthonormalisation failed");
      const double ljj = std::sqrt(d);
      L[(size_t)j * r + j] = mk(ljj, 0.0);
      for (int i = j + 1; i < r; ++i) {
        cx<double> v = M[(size_t)i * r + j];
        for (int k = 0; k < j; ++k) v = v - L[(size_t)i * r + k] * conj(L[(size_t)j * r + k]);
        L[(size_t)i * r + j] = mk(v.r / ljj, v.i / ljj);
      }
    }
    for (int c = 0; c < r; ++c)  // columns of L^{-1} by forward substitution
      for (int i = c; i < r; ++i) {
        cx<double> v = mk(i == c ? 1.0 : 0.0, 0.0);
        for (int k = c; k < i; ++k) v = v - L[(size_t)i * r + k] * Li[(size_t)k * r + c];
        const double lii = L[(size_t)i * r + i].r;
        Li[(size_t)i * r + c] = mk(v.r / lii, v.i / lii);
      }
    std::vector<cx<double>> T((size_t)r * r);  // T = L^{-H}: T[j][k] = conj(Li[k][j])
    for (int j = 0; j < r; ++j)
      for (int k = 0; k < r; ++k) T[(size_t)j * r + k] = conj(Li[(size_t)k * r + j]);
    DevBuf dTr;
    dTr.reserve(sizeof(cx<double>) * r * r);
    copy_in(ctx, dTr.p, T.data(), sizeof(cx<double>) * r * r);
    ws.Phi.reserve(sizeof(cx<double>) * r * N);
    combine_basis_kernel<<<grid_for(N * r, 256), 256, 0, st>>>(Phi0.as<cx<double>>(), dTr.as<cx<double>>(), N, r, r,
                                                                ws.Phi.as<cx<double>>());
    BEM_LAUNCHED();
    ctx->launches++;
    BEM_CUDA(cudaStreamSynchronize(st));
  }
  ws.r = r;
  // training set: features and scaled targets
  double omega = 0;
  for (int j = 0; j < J; ++j) omega = std::max(omega, std::fabs(ws.s[2 * j + 1]));
  omega = std::max(omega, std::fabs(ws.s[0]));
  ws.omega = omega;
  std::vector<float> Uh(2 * J);
  for (int j = 0; j < J; ++j) {
    Uh[2 * j] = (float)(ws.s[2 * j] / omega);
    Uh[2 * j + 1] = (float)(ws.s[2 * j + 1] / omega);
  }
  DevBuf dU, dT, dY, dG, dM, dVv, dloss, dC;
  dU.reserve(sizeof(float) * 2 * J);
  dT.reserve(sizeof(float) * 2 * r * J);
  dY.reserve(sizeof(float) * 2 * r * J);
  dC.reserve(sizeof(cx<double>) * r * J);
  copy_in(ctx, dU.p, Uh.data(), sizeof(float) * 2 * J);
  project_kernel<<<dim3(J, r), 256, 0, st>>>(ws.Phi.as<cx<double>>(), ws.X.as<cx<double>>(), N, r,
                                              dC.as<cx<double>>());
  BEM_LAUNCHED();
  ctx->launches++;
  // targets: unit-norm coefficient directions with a real non-negative leading entry
  std::vector<cx<double>> Ch((size_t)r * J);
  copy_out(ctx, Ch.data(), dC.p, sizeof(cx<double>) * r * J);
  std::vector<float> Th((size_t)2 * r * J);
  for (int j = 0; j < J; ++j) {
    const cx<double>* c = &Ch[(size_t)j * r];
    double nrm = 0;
    for (int k = 0; k < r; ++k) nrm += c[k].r * c[k].r + c[k].i * c[k].i;
    nrm = std::sqrt(nrm);
    const double a0 = std::hypot(c[0].r, c[0].i);
    // multiplier conj(c_0) / (|c_0| |c|): unit norm, leading entry real and >= 0
    cx<double> m = mk(nrm > 0 ? 1.0 / nrm : 1.0, 0.0);
    if (a0 > 0 && nrm > 0) m = mk(c[0].r / (a0 * nrm), -c[0].i / (a0 * nrm));
    for (int k = 0; k < r; ++k) {
      const cx<double> t = c[k] * m;
      Th[(size_t)j * 2 * r + k] = (float)t.r;
      Th[(size_t)j * 2 * r + r + k] = (float)t.i;
    }
  }
  copy_in(ctx, dT.p, Th.data(), sizeof(float) * 2 * r * J);
  // parameters: uniform(-1/sqrt(fan_in), 1/sqrt(fan_in)) weights, zero biases, seeded
  const int64_t np = n_params(r);
  std::vector<float> ph(np, 0.f);
  std::mt19937_64 rng(prm.seed);
  ParamView pv = view(ph.data(), r);
  auto fill = [&](float* W, int fo, int fi) {
    std::uniform_real_distribution<double> U(-1.0 / std::sqrt(fi), 1.0 / std::sqrt(fi));
    for (int i = 0; i < fo * fi; ++i) W[i] = (float)U(rng);
  };
  fill(pv.W1, kHidden, 2);
  fill(pv.W2, kHidden, kHidden);
  fill(pv.W3, 2 * r, kHidden);
  ws.params.reserve(sizeof(float) * np);
  copy_in(ctx, ws.params.p, ph.data(), sizeof(float) * np);
  dG.reserve(sizeof(float) * np);
  dM.reserve(sizeof(float) * np);
  dVv.reserve(sizeof(float) * np);
  dloss.reserve(sizeof(double));
  BEM_CUDA(cudaMemsetAsync(dM.p, 0, sizeof(float) * np, st));
  BEM_CUDA(cudaMemsetAsync(dVv.p, 0, sizeof(float) * np, st));
  double first = 0, last = 0;
  const float b1 = 0.9f, b2 = 0.999f;
  for (int it = 1; it <= prm.steps; ++it) {
    BEM_CUDA(cudaMemsetAsync(dloss.p, 0, sizeof(double), st));
    mlp_pass(ctx, ws.params.as<float>(), r, dU.as<float>(), J, dT.as<float>(), dY.as<float>(), dG.as<float>(),
             dloss.as<double>());
    const float c1 = 1.f - std::pow(b1, (float)it), c2 = 1.f - std::pow(b2, (float)it);
    adam_kernel<<<grid_for(np, 256), 256, 0, st>>>(ws.params.as<float>(), dG.as<float>(), dM.as<float>(),
                                                   dVv.as<float>(), (int)np, (float)prm.lr, b1, b2, c1, c2, 1e-8f);
    BEM_LAUNCHED();
    ctx->launches++;
    if (it == 1 || it == prm.steps) {
      double l = 0;
      copy_out(ctx, &l, dloss.p, sizeof(double));
      if (it == 1) first = l;
      last = l;
    }
  }
  ws.trained = true;
  if (out) {
    out->r = r;
    out->n_snapshots = J;
    out->loss_first = first;
    out->loss_last = last;
    out->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  }
}

// Warm-start directions x^[f] (device [F][N]) for the F frequencies s (host, 2F doubles).
void warm_initial(bem_ctx* ctx, int mode, const double* s, int64_t F, cx<double>* x0) {
  WarmStart& ws = ctx->warm;
  const int64_t N = 3 * ctx->mesh.ne;
  BEM_REQUIRE(ws.N == N && !ws.s.empty(), "warm start requested but no stored solutions match the mesh");
  if (mode == BEM_WARM_VF) {
    // weights for exactly these frequencies, else the nearest stored solution
    bool have = ws.vf_J > 0 && (int64_t)ws.vf_s.size() == 2 * F && ws.vf_J <= (int64_t)(ws.s.size() / 2);
    for (int64_t k = 0; have && k < 2 * F; ++k) have = ws.vf_s[k] == s[k];
    if (have) {
      DevBuf dw;
      dw.reserve(sizeof(cx<double>) * F * ws.vf_J);
      copy_in(ctx, dw.p, ws.vf_w.data(), sizeof(cx<double>) * F * ws.vf_J);
      weighted_sum_kernel<<<grid_for(N * F, 256), 256, 0, ctx->stream>>>(dw.as<cx<double>>(), ws.X.as<cx<double>>(),
                                                                          N, ws.vf_J, F, x0);
      BEM_LAUNCHED();
      ctx->launches++;
      BEM_CUDA(cudaStreamSynchronize(ctx->stream));  // dw is released on return
      return;
    }
    mode = BEM_WARM_NEAREST;
  }
  if (mode == BEM_WARM_NEAREST) {
    const int J = (int)(ws.s.size() / 2);
    for (int64_t f = 0; f < F; ++f) {
      const double sr = s[2 * f], si = s[2 * f + 1];
      int best = 0;
      double bd = 1e300;
      for (int j = 0; j < J; ++j) {
        const double d = std::hypot(ws.s[2 * j] - sr, ws.s[2 * j + 1] - si);
        if (d < bd) {
          bd = d;
          best = j;
        }
      }
      BEM_CUDA(cudaMemcpyAsync(x0 + f * N, ws.X.as<cx<double>>() + (int64_t)best * N, sizeof(cx<double>) * N,
                               cudaMemcpyDeviceToDevice, ctx->stream));
    }
    return;
  }
  BEM_REQUIRE(ws.trained, "BEM_WARM_MLP requested before bem_warm_train");
  std::vector<float> Uh(2 * F);
  for (int64_t f = 0; f < F; ++f) {
    Uh[2 * f] = (float)(s[2 * f] / ws.omega);
    Uh[2 * f + 1] = (float)(s[2 * f + 1] / ws.omega);
  }
  DevBuf dU, dY;
  dU.reserve(sizeof(float) * 2 * F);
  dY.reserve(sizeof(float) * 2 * ws.r * F);
  copy_in(ctx, dU.p, Uh.data(), sizeof(float) * 2 * F);
  mlp_pass(ctx, ws.params.as<float>(), ws.r, dU.as<float>(), (int)F, nullptr, dY.as<float>(), nullptr, nullptr);
  expand_kernel<<<grid_for(N * F, 256), 256, 0, ctx->stream>>>(dY.as<float>(), ws.Phi.as<cx<double>>(), N, ws.r,
                                                                (int)F, x0);
  BEM_LAUNCHED();
  ctx->launches++;
}

// Forward / backward with caller parameters (verification).
void mlp_eval(bem_ctx* ctx, int r, const float* params_h, const float* U_h, int B, const float* T_h,
              float* Y_h, float* grads_h, double* loss_h) {
  const int64_t np = n_params(r);
  DevBuf dp, dU, dT, dY, dG, dl;
  dp.reserve(sizeof(float) * np);
  dU.reserve(sizeof(float) * 2 * B);
  dY.reserve(sizeof(float) * 2 * r * B);
  copy_in(ctx, dp.p, params_h, sizeof(float) * np);
  copy_in(ctx, dU.p, U_h, sizeof(float) * 2 * B);
  const bool back = T_h && grads_h;
  if (back) {
    dT.reserve(sizeof(float) * 2 * r * B);
    dG.reserve(sizeof(float) * np);
    dl.reserve(sizeof(double));
    copy_in(ctx, dT.p, T_h, sizeof(float) * 2 * r * B);
    BEM_CUDA(cudaMemsetAsync(dl.p, 0, sizeof(double), ctx->stream));
  }
  mlp_pass(ctx, dp.as<float>(), r, dU.as<float>(), B, back ? dT.as<float>() : nullptr, dY.as<float>(),
           back ? dG.as<float>() : nullptr, back ? dl.as<double>() : nullptr);
  copy_out(ctx, Y_h, dY.p, sizeof(float) * 2 * r * B);
  if (back) {
    copy_out(ctx, grads_h, dG.p, sizeof(float) * np);
    if (loss_h) copy_out(ctx, loss_h, dl.p, sizeof(double));
  }
}

int64_t mlp_n_params(int r) { return n_params(r); }

}  // namespace bem
