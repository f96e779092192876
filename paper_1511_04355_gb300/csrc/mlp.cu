// Learned warm start for the frequency solves (not part of the paper; the paper's adaptive
// sampling of Sec. 3 solves one new frequency at a time, next to frequencies already solved).
//
// Memory: solutions x(s_j) of solved frequencies (FP64 on the device).
// POD:    Phi = the r leading left singular vectors of X = [x(s_1) .. x(s_J)]: Gram matrix
//         G = X^H X on the device (FP64), eigenpairs of G on the host (cyclic Jacobi on the real
//         symmetric embedding [[Re G, -Im G], [Im G, Re G]]), Phi_k = X v_k / sigma_k.
// MLP:    u = (Re s, Im s) / Omega -> 128 -> 128 -> 2r (tanh-GELU), trained on the device to
//         predict c_j = Phi^H x(s_j) (scaled) with MSE loss and Adam: FP32 master weights; the
//         three dense layers' products run on the tensor cores (mma.sync m16n8k16, FP16
//         operands, FP32 accumulation), elementwise parts in FP32.  The products are tiny
//         (at most 256 x 128 x 256), so one warp computes one 16 x 8 output tile.
// Warm start: x0(s) = Phi c(s) (BEM_WARM_MLP) or the stored solution at the nearest solved
//         frequency (BEM_WARM_NEAREST).
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

// x0[f][n] = scale * sum_k (y[f][k] + i y[f][r + k]) Phi[k][n]
__global__ void expand_kernel(const float* y, const cx<double>* Phi, int64_t N, int r, int F, double scale,
                              cx<double>* x0) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= N * F) return;
  const int f = (int)(t / N);
  const int64_t n = t % N;
  cx<double> s = mk(0.0, 0.0);
  for (int k = 0; k < r; ++k)
    s = cfma(mk((double)y[f * 2 * r + k] * scale, (double)y[f * 2 * r + r + k] * scale), Phi[(int64_t)k * N + n], s);
  x0[t] = s;
}

// targets T[j][k] = [Re c, Im c] / scale, c = Phi^H x_j (one block per (j, k))
__global__ void project_kernel(const cx<double>* Phi, const cx<double>* X, int64_t N, int r, double inv_scale,
                               float* T) {
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
  if (threadIdx.x == 0) {
    T[j * 2 * r + k] = (float)(sr[0] * inv_scale);
    T[j * 2 * r + r + k] = (float)(si[0] * inv_scale);
  }
}

// ------------------------------------------------------------------------------- host helpers
namespace {

// Eigen-decomposition of a real symmetric n x n matrix by cyclic Jacobi rotations (row-major);
// returns eigenvalues, eigenvectors in the columns of V.
void jacobi_eig(int n, std::vector<double>& A, std::vector<double>& w, std::vector<double>& V) {
  V.assign((size_t)n * n, 0.0);
  for (int i = 0; i < n; ++i) V[(size_t)i * n + i] = 1.0;
  auto a = [&](int i, int j) -> double& { return A[(size_t)i * n + j]; };
  for (int sweep = 0; sweep < 60; ++sweep) {
    double off = 0, tot = 0;
    for (int i = 0; i < n; ++i)
      for (int j = 0; j < n; ++j) {
        tot += a(i, j) * a(i, j);
        if (i != j) off += a(i, j) * a(i, j);
      }
    if (off <= 1e-30 * tot) break;
    for (int p = 0; p < n - 1; ++p)
      for (int q = p + 1; q < n; ++q) {
        const double apq = a(p, q);
        if (std::fabs(apq) < 1e-300) continue;
        const double theta = (a(q, q) - a(p, p)) / (2.0 * apq);
        const double t = (theta >= 0 ? 1.0 : -1.0) / (std::fabs(theta) + std::sqrt(theta * theta + 1.0));
        const double c = 1.0 / std::sqrt(t * t + 1.0), s = t * c;
        for (int k = 0; k < n; ++k) {  // columns p, q
          const double akp = a(k, p), akq = a(k, q);
          a(k, p) = c * akp - s * akq;
          a(k, q) = s * akp + c * akq;
        }
        for (int k = 0; k < n; ++k) {  // rows p, q
          const double apk = a(p, k), aqk = a(q, k);
          a(p, k) = c * apk - s * aqk;
          a(q, k) = s * apk + c * aqk;
        }
        for (int k = 0; k < n; ++k) {
          const double vkp = V[(size_t)k * n + p], vkq = V[(size_t)k * n + q];
          V[(size_t)k * n + p] = c * vkp - s * vkq;
          V[(size_t)k * n + q] = s * vkp + c * vkq;
        }
      }
  }
  w.resize(n);
  for (int i = 0; i < n; ++i) w[i] = a(i, i);
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
  ws.trained = false;
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
  const int n2 = 2 * J;
  std::vector<double> A((size_t)n2 * n2), w, V;
  for (int a = 0; a < J; ++a)
    for (int b = 0; b < J; ++b) {
      const cx<double> g = Gh[(size_t)a * J + b];
      A[(size_t)a * n2 + b] = g.r;
      A[(size_t)a * n2 + J + b] = -g.i;
      A[(size_t)(J + a) * n2 + b] = g.i;
      A[(size_t)(J + a) * n2 + J + b] = g.r;
    }
  jacobi_eig(n2, A, w, V);
  // each eigenvalue of G appears twice in the embedding; take every other one, descending
  std::vector<int> order(n2);
  for (int i = 0; i < n2; ++i) order[i] = i;
  std::sort(order.begin(), order.end(), [&](int a, int b) { return w[a] > w[b]; });
  std::vector<int> pick;
  std::vector<std::vector<cx<double>>> vecs;
  const double lmax = std::max(w[order[0]], 1e-300);
  for (int idx : order) {
    if ((int)pick.size() >= prm.r_max) break;
    if (w[idx] <= prm.rel_tol * prm.rel_tol * lmax) break;
    std::vector<cx<double>> v(J);
    for (int j = 0; j < J; ++j) v[j] = mk(V[(size_t)j * n2 + idx], V[(size_t)(J + j) * n2 + idx]);
    // drop the partner (i * v) of an eigenvector already taken
    bool dup = false;
    for (const auto& u : vecs) {
      double pr = 0, pi = 0;
      for (int j = 0; j < J; ++j) {
        pr += u[j].r * v[j].r + u[j].i * v[j].i;
        pi += u[j].r * v[j].i - u[j].i * v[j].r;
      }
      if (pr * pr + pi * pi > 0.5) dup = true;
    }
    if (dup) continue;
    double nv = 0;
    for (int j = 0; j < J; ++j) nv += v[j].r * v[j].r + v[j].i * v[j].i;
    nv = std::sqrt(nv);
    for (int j = 0; j < J; ++j) v[j] = mk(v[j].r / nv, v[j].i / nv);
    vecs.push_back(v);
    pick.push_back(idx);
  }
  const int r = (int)pick.size();
  BEM_REQUIRE(r >= 1, "POD found no basis vector");
  std::vector<cx<double>> Vs((size_t)J * r);
  for (int k = 0; k < r; ++k) {
    const double sg = std::sqrt(std::max(w[pick[k]], 1e-300));
    for (int j = 0; j < J; ++j) Vs[(size_t)j * r + k] = mk(vecs[k][j].r / sg, vecs[k][j].i / sg);
  }
  DevBuf dV;
  dV.reserve(sizeof(cx<double>) * J * r);
  copy_in(ctx, dV.p, Vs.data(), sizeof(cx<double>) * J * r);
  ws.Phi.reserve(sizeof(cx<double>) * r * N);
  combine_basis_kernel<<<grid_for(N * r, 256), 256, 0, st>>>(ws.X.as<cx<double>>(), dV.as<cx<double>>(), N, J, r,
                                                              ws.Phi.as<cx<double>>());
  BEM_LAUNCHED();
  ctx->launches++;
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
  // scale: largest coefficient magnitude (sigma_1 bounds |c| per snapshot)
  ws.scale = std::sqrt(std::max(w[pick[0]], 1e-300));
  DevBuf dU, dT, dY, dG, dM, dVv, dloss;
  dU.reserve(sizeof(float) * 2 * J);
  dT.reserve(sizeof(float) * 2 * r * J);
  dY.reserve(sizeof(float) * 2 * r * J);
  copy_in(ctx, dU.p, Uh.data(), sizeof(float) * 2 * J);
  project_kernel<<<dim3(J, r), 256, 0, st>>>(ws.Phi.as<cx<double>>(), ws.X.as<cx<double>>(), N, r, 1.0 / ws.scale,
                                              dT.as<float>());
  BEM_LAUNCHED();
  ctx->launches++;
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

// x0[f] for the frequencies of the current set (device [F][N]).
void warm_initial(bem_ctx* ctx, int mode, cx<double>* x0) {
  WarmStart& ws = ctx->warm;
  const int64_t F = ctx->fs.F, N = 3 * ctx->mesh.ne;
  BEM_REQUIRE(ws.N == N && !ws.s.empty(), "warm start requested but no stored solutions match the mesh");
  if (mode == BEM_WARM_NEAREST) {
    const int J = (int)(ws.s.size() / 2);
    for (int64_t f = 0; f < F; ++f) {
      const double sr = ctx->fs.s[2 * f], si = ctx->fs.s[2 * f + 1];
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
    Uh[2 * f] = (float)(ctx->fs.s[2 * f] / ws.omega);
    Uh[2 * f + 1] = (float)(ctx->fs.s[2 * f + 1] / ws.omega);
  }
  DevBuf dU, dY;
  dU.reserve(sizeof(float) * 2 * F);
  dY.reserve(sizeof(float) * 2 * ws.r * F);
  copy_in(ctx, dU.p, Uh.data(), sizeof(float) * 2 * F);
  mlp_pass(ctx, ws.params.as<float>(), ws.r, dU.as<float>(), (int)F, nullptr, dY.as<float>(), nullptr, nullptr);
  expand_kernel<<<grid_for(N * F, 256), 256, 0, ctx->stream>>>(dY.as<float>(), ws.Phi.as<cx<double>>(), N, ws.r,
                                                                (int)F, ws.scale, x0);
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
