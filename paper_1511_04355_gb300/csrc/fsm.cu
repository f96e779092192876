// Fourier series method (FSM) inverse Laplace transform on the GPU, FP64 (Sec. 2.2,
// Eqs. (invLap), (IDFT-MFT)).
//
// Samples h(s_k) at s_k = eta + i k dw, dw = 2 pi / P, k = 0 .. Nc-1 (N_s = 2 (Nc - 1)), the
// rest of the spectrum following from h(s_{N_s-k}) = conj(h(s_k)).  For any time t:
//   h(t) = e^{eta t} / P [ W_0 Re h_0 + 2 Re sum_{k=1}^{Nc-2} W_k h_k e^{i k dw t}
//                          + W_{Nc-1} Re(h_{Nc-1} e^{i (Nc-1) dw t}) ],
// W_k = (1 + cos(2 pi k / N_s)) / 2 (Hanning) or 1.  The 1/P factor of the trapezoidal rule is
// kept (the printed Eq. (IDFT-MFT) omits it); the Nyquist term is counted once.
// Two kernels: the phase table E[j][k] = c_k W_k e^{i k dw t_j} e^{eta t_j} / P (scratch,
// nt x Nc complex), then out[j][d] = Re sum_k E[j][k] h[k][d] (one thread per output, the
// table row broadcast from shared memory, h read coalesced along d).
#include "kernel_math.cuh"

namespace bem {

__global__ void fsm_table_kernel(const double* t, int64_t nt, int64_t nc, double eta, double period,
                                 int window, cx<double>* E) {
  const int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (q >= nt * nc) return;
  const int64_t j = q / nc, k = q % nc;
  const int64_t ns = 2 * (nc - 1);
  const double dw = 2.0 * kPi / period;
  const double tj = t[j];
  double w = 1.0;
  if (window && ns > 0) w = 0.5 * (1.0 + cos(2.0 * kPi * (double)k / (double)ns));
  const double c = (k == 0 || k == nc - 1) ? 1.0 : 2.0;
  const double amp = c * w * exp(eta * tj) / period;
  double sn, cs;
  sincos((double)k * dw * tj, &sn, &cs);
  E[q] = mk(amp * cs, amp * sn);
}

// out[j][d] = Re sum_k E[j][k] h[k][d]; grid (ceil(m / 128), min(nt, 65535)), each block
// row strides over the times j by gridDim.y (grid y is capped at 65535), the table row of the
// current time in shared memory.
__global__ void fsm_apply_kernel(const cx<double>* E, const cx<double>* h, int64_t nt, int64_t nc,
                                 int64_t m, double* out) {
  extern __shared__ cx<double> row[];
  const int64_t d = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  for (int64_t j = blockIdx.y; j < nt; j += gridDim.y) {
    __syncthreads();  // the previous time's row is no longer read
    for (int64_t k = threadIdx.x; k < nc; k += blockDim.x) row[k] = E[j * nc + k];
    __syncthreads();
    if (d < m) {
      double acc = 0.0;
      for (int64_t k = 0; k < nc; ++k) {
        const cx<double> hv = h[k * m + d];
        acc = fma(row[k].r, hv.r, fma(-row[k].i, hv.i, acc));
      }
      out[j * m + d] = acc;
    }
  }
}

// Launch both kernels with a caller-provided table (nt x nc complex).
void fsm_launch(const cx<double>* h, int64_t nc, int64_t m, double eta, double period,
                const double* t, int64_t nt, int window, double* out, cx<double>* table,
                cudaStream_t st) {
  fsm_table_kernel<<<grid_for(nt * nc, 256), 256, 0, st>>>(t, nt, nc, eta, period, window, table);
  BEM_LAUNCHED();
  const size_t smem = sizeof(cx<double>) * nc;
  if (smem > 48 * 1024)
    BEM_CUDA(cudaFuncSetAttribute(fsm_apply_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  const unsigned gy = (unsigned)std::min<int64_t>(nt, 65535);
  fsm_apply_kernel<<<dim3(grid_for(m, 128), gy), 128, smem, st>>>(table, h, nt, nc, m, out);
  BEM_LAUNCHED();
}

void fsm_check_args(int64_t nc, int64_t m, double eta, double period, int64_t nt, int window) {
  BEM_REQUIRE(nc >= 2, "need at least 2 frequency samples (N_s = 2 (Nc - 1) >= 2)");
  BEM_REQUIRE(m >= 1 && nt >= 1, "need m >= 1 responses and nt >= 1 times");
  BEM_REQUIRE(period > 0 && std::isfinite(period), "period must be > 0");
  BEM_REQUIRE(std::isfinite(eta), "eta must be finite");
  BEM_REQUIRE(window == 0 || window == 1, "window must be 0 (none) or 1 (Hanning)");
  BEM_REQUIRE(nc * (int64_t)sizeof(cx<double>) <= 200 * 1024, "too many frequency samples (max 12800)");
}

// gather out[f][d] = x[f][dofs[d]]
__global__ void gather_kernel(const cx<double>* x, int64_t N, int64_t F, const int64_t* dofs,
                              int64_t nd, cx<double>* out) {
  const int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (q >= F * nd) return;
  const int64_t f = q / nd, d = q % nd;
  out[q] = x[f * N + dofs[d]];
}

void gather_dofs(bem_ctx* ctx, const cx<double>* x, int64_t N, int64_t F, const int64_t* dofs_dev,
                 int64_t nd, cx<double>* out) {
  gather_kernel<<<grid_for(F * nd, 256), 256, 0, ctx->stream>>>(x, N, F, dofs_dev, nd, out);
  BEM_LAUNCHED();
  ctx->launches++;
}

}  // namespace bem
