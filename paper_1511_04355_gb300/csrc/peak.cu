// Measured arithmetic peaks of the device (bem_measure_peak): the denominators of the rooflines
// of the ALU-bound kernels.  The paper has no counterpart; the operator, the refinement residual
// and the plain-FP64 path are bound by the FP32 and FP64 pipes, whose rates are not in the
// table of measured copy and tensor-core peaks, so they are measured here the same way.
//
// Each thread runs kChains independent fused multiply-add chains x <- x * a + b (one FFMA or
// DFMA per step, 2 flops), which is enough independent work per warp to keep the FMA pipes
// issuing every cycle; the grid fills every SM with kBlocksPerSm blocks of kThreads threads.
// The chains' sum is stored only if it equals an impossible value, so the arithmetic cannot be
// removed but nothing is written.  Each launch is timed with CUDA events on the context's
// stream; the best of the timed launches counts.
#include "bem_internal.cuh"

namespace bem {
namespace {

constexpr int kChains = 8;
constexpr int kThreads = 256;
constexpr int kBlocksPerSm = 8;

template <class R>
__global__ void __launch_bounds__(kThreads) fma_chain_kernel(R a, R b, int iters, R* sink) {
  R x[kChains];
#pragma unroll
  for (int c = 0; c < kChains; ++c) x[c] = (R)(threadIdx.x + c) * (R)1e-3;
  for (int it = 0; it < iters; ++it) {
#pragma unroll 16
    for (int u = 0; u < 16; ++u) {
#pragma unroll
      for (int c = 0; c < kChains; ++c) x[c] = fma(x[c], a, b);
    }
  }
  R s = 0;
#pragma unroll
  for (int c = 0; c < kChains; ++c) s += x[c];
  if (s == (R)-1.2345e30) sink[blockIdx.x] = s;
}

// The same chains with the paired FP32 instruction (two fused multiply-adds per thread and
// instruction, __ffma2_rn): whether the FP32 pipes run faster per issued instruction.
__global__ void __launch_bounds__(kThreads) fma2_chain_kernel(float a, float b, int iters, float* sink) {
  float2 x[kChains / 2];
#pragma unroll
  for (int c = 0; c < kChains / 2; ++c) x[c] = make_float2((float)(threadIdx.x + 2 * c) * 1e-3f, (float)(threadIdx.x + 2 * c + 1) * 1e-3f);
  const float2 a2 = make_float2(a, a), b2 = make_float2(b, b);
  for (int it = 0; it < iters; ++it) {
#pragma unroll 16
    for (int u = 0; u < 16; ++u) {
#pragma unroll
      for (int c = 0; c < kChains / 2; ++c) x[c] = __ffma2_rn(x[c], a2, b2);
    }
  }
  float s = 0;
#pragma unroll
  for (int c = 0; c < kChains / 2; ++c) s += x[c].x + x[c].y;
  if (s == -1.2345e30f) sink[blockIdx.x] = s;
}

template <class R, bool PAIRED = false>
void measure(bem_ctx* ctx, int iters, int reps, double* tflops, double* ms_best, int32_t* sms) {
  int n_sm = 0;
  BEM_CUDA(cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, ctx->device));
  const int blocks = n_sm * kBlocksPerSm;
  R* sink = nullptr;
  BEM_CUDA(cudaMalloc(&sink, sizeof(R) * blocks));
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  float best = 0;
  try {
    BEM_CUDA(cudaEventCreate(&e0));
    BEM_CUDA(cudaEventCreate(&e1));
    // a = 1 - 2^-20, b = 2^-20: the chains stay finite and non-constant for any length
    const R a = (R)1 - (R)9.5367431640625e-7, b = (R)9.5367431640625e-7;
    auto launch = [&] {
      if constexpr (PAIRED) fma2_chain_kernel<<<blocks, kThreads, 0, ctx->stream>>>(a, b, iters, sink);
      else fma_chain_kernel<R><<<blocks, kThreads, 0, ctx->stream>>>(a, b, iters, sink);
    };
    launch();  // warm-up
    BEM_LAUNCHED();
    for (int r = 0; r < reps; ++r) {
      BEM_CUDA(cudaEventRecord(e0, ctx->stream));
      launch();
      BEM_LAUNCHED();
      BEM_CUDA(cudaEventRecord(e1, ctx->stream));
      BEM_CUDA(cudaEventSynchronize(e1));
      float ms = 0;
      BEM_CUDA(cudaEventElapsedTime(&ms, e0, e1));
      if (r == 0 || ms < best) best = ms;
    }
  } catch (...) {
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaFree(sink);
    throw;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  BEM_CUDA(cudaFree(sink));
  const double flops = 2.0 * kChains * 16.0 * (double)iters * (double)blocks * kThreads;
  if (tflops) *tflops = best > 0 ? flops / (best * 1e-3) / 1e12 : 0.0;
  if (ms_best) *ms_best = best;
  if (sms) *sms = n_sm;
  ctx->launches += reps + 1;
}

}  // namespace
}  // namespace bem

using namespace bem;

extern "C" int bem_measure_peak(bem_ctx* ctx, int kind, int32_t iters, int32_t reps,
                                double* tflops, double* ms_best, int32_t* sm_count) {
  return guarded_call(ctx, [&] {
    BEM_REQUIRE(kind == BEM_PEAK_FP32 || kind == BEM_PEAK_FP64 || kind == BEM_PEAK_FP32X2,
                "kind must be BEM_PEAK_FP32, BEM_PEAK_FP64 or BEM_PEAK_FP32X2");
    BEM_REQUIRE(iters >= 1 && reps >= 1, "iters and reps must be >= 1");
    if (kind == BEM_PEAK_FP32)
      measure<float>(ctx, iters, reps, tflops, ms_best, sm_count);
    else if (kind == BEM_PEAK_FP32X2)
      measure<float, true>(ctx, iters, reps, tflops, ms_best, sm_count);
    else
      measure<double>(ctx, iters, reps, tflops, ms_best, sm_count);
  });
}
