// Internal declarations of the GB300 BEM library (not part of the ABI).
//
// Layout in device memory (n_e elements, N = 3 n_e unknowns, F frequencies in a batch):
//   element geometry   Elem64[n_e] (FP64 master), float4 SoA copies for the FP32 kernels
//   quadrature points  4-point and 7-point rules: [n_e][q] x (x, y, z, w * area)
//   near lists         CSR int32 (row_ptr[n_e+1], cols[nnz])
//   vectors            [F][n_e][3] complex, (re, im) interleaved, frequency-major so that one
//                      instance's vector is contiguous for the GMRES vector kernels
//   diagonal blocks    [F][n_e][9] complex FP64: own-element H_ii and G_ii
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <cmath>
#include <cstdio>
#include <memory>
#include <stdexcept>
#include <string>
#include <vector>

#include "../../include/bem.h"
#include "hmatrix_host.h"

namespace bem {

// ------------------------------------------------------------------------------- errors
struct Error : std::runtime_error {
  int code;
  Error(int c, const std::string& m) : std::runtime_error(m), code(c) {}
};

#define BEM_CUDA(call)                                                                  \
  do {                                                                                  \
    cudaError_t e_ = (call);                                                            \
    if (e_ != cudaSuccess) {                                                            \
      throw ::bem::Error(e_ == cudaErrorMemoryAllocation ? BEM_ERR_OOM : BEM_ERR_CUDA,  \
                         std::string(#call) + ": " + cudaGetErrorString(e_));           \
    }                                                                                   \
  } while (0)

#define BEM_REQUIRE(cond, msg)                                              \
  do {                                                                      \
    if (!(cond)) throw ::bem::Error(BEM_ERR_INVALID_ARG, std::string(msg)); \
  } while (0)

// launch check: catches configuration errors right after a launch
#define BEM_LAUNCHED() BEM_CUDA(cudaGetLastError())

// ------------------------------------------------------------------------------- complex
template <class R>
struct cx {
  R r, i;
};
template <class R>
__host__ __device__ __forceinline__ cx<R> mk(R r, R i) {
  cx<R> z;
  z.r = r;
  z.i = i;
  return z;
}
template <class R>
__host__ __device__ __forceinline__ cx<R> operator+(cx<R> a, cx<R> b) { return mk(a.r + b.r, a.i + b.i); }
template <class R>
__host__ __device__ __forceinline__ cx<R> operator-(cx<R> a, cx<R> b) { return mk(a.r - b.r, a.i - b.i); }
template <class R>
__host__ __device__ __forceinline__ cx<R> operator*(cx<R> a, cx<R> b) {
  return mk(a.r * b.r - a.i * b.i, a.r * b.i + a.i * b.r);
}
template <class R>
__host__ __device__ __forceinline__ cx<R> operator*(R a, cx<R> b) { return mk(a * b.r, a * b.i); }
template <class R>
__host__ __device__ __forceinline__ cx<R> conj(cx<R> a) { return mk(a.r, -a.i); }
// a + k * b with real k
template <class R>
__host__ __device__ __forceinline__ cx<R> axpy(R k, cx<R> b, cx<R> a) {
  return mk(fma(k, b.r, a.r), fma(k, b.i, a.i));
}
// a + b * c (complex)
template <class R>
__host__ __device__ __forceinline__ cx<R> cfma(cx<R> b, cx<R> c, cx<R> a) {
  return mk(fma(b.r, c.r, fma(-b.i, c.i, a.r)), fma(b.r, c.i, fma(b.i, c.r, a.i)));
}

// ------------------------------------------------------------------------------- constants
constexpr int kSeriesMax = 20;         // max Taylor terms of the small-|z| branch
constexpr int kSeriesF32 = 9;          // terms used by the FP32 kernels (|z| < 1/2)
constexpr int kSeriesF64 = 18;         // terms used by the FP64 kernels (|z| < 1/2)
constexpr double kZSeries2 = 0.25;     // |z_s|^2 below which the series is used
constexpr double kNearFactor = 2.0;    // near source: |x_i - c_e| < 2 h_e
constexpr int kDuffyN = 13;            // Gauss-Legendre points per Duffy direction

// Material constants used by the kernels (host computes them in FP64).
template <class R>
struct MatC {
  R mu;        // shear modulus
  R inv_cs;    // 1 / c_s
  R beta;      // c_s / c_p
  R beta2;     // (c_s / c_p)^2
  R c1m2b2;    // 1 - 2 beta^2
  R inv4pimu;  // 1 / (4 pi mu)
  R d[kSeriesMax];  // Taylor coefficients of J(z) = beta^2 h(beta z) - h(z)
};

// Per-frequency constants.
template <class R>
struct FreqC {
  cx<R> a;       // s / c_s
  cx<R> inv_a2;  // 1 / a^2
  R a_abs2;      // |a|^2
  R pad;
  // phase slopes Im(s)/c_s and Im(s)/c_p as (hi, lo) pairs: the FP32 kernels form the phase
  // omega r / c in float-float so that it carries ~1e-7 absolute error at |phase| ~ 60
  R ai_hi, ai_lo, bi_hi, bi_lo;
};

// A far-kernel CTA's frequencies: entries [start, start + count) of the staged frequency list.
// In an equally spaced group (recurrence kernel) s_j = s_0 + j i delta, and (ws, wp) are the
// phase slopes of one step, delta / c_s and beta delta / c_s, as float-float pairs.
struct FarGroup {
  int32_t start, count;
  float ws_hi, ws_lo, wp_hi, wp_lo;
};

// Shape of an FP32 far-field launch (see bem_tune_entry): frequencies per CTA, source tiles a
// CTA sums before its FP64 atomic add, and the grid's target in waves of resident CTAs.
struct FarShape {
  int ft = 12, tiles = 2, waves = 4;
};

// Four packed doubles (centroid + h, normal + area, quadrature point + weight).
struct alignas(32) D4 {
  double x, y, z, w;
};

// Element geometry, FP64 master.
struct Elem64 {
  double c[3];  // centroid (collocation point)
  double n[3];  // unit normal (out of the elastic domain)
  double area;
  double h;     // longest edge
};

// ------------------------------------------------------------------------------- buffers
struct DevBuf {
  void* p = nullptr;
  size_t bytes = 0;
  DevBuf() = default;
  DevBuf(const DevBuf&) = delete;
  DevBuf& operator=(const DevBuf&) = delete;
  ~DevBuf() { release(); }
  void release() {
    if (p) cudaFree(p);
    p = nullptr;
    bytes = 0;
  }
  // grow-only: keeps the allocation when it is large enough
  void reserve(size_t n) {
    if (n <= bytes) return;
    release();
    if (n == 0) return;
    cudaError_t e = cudaMalloc(&p, n);
    if (e != cudaSuccess) {
      p = nullptr;
      throw Error(BEM_ERR_OOM, "cudaMalloc of " + std::to_string(n) + " bytes failed: " +
                                   cudaGetErrorString(e));
    }
    bytes = n;
  }
  template <class T>
  T* as() const { return reinterpret_cast<T*>(p); }
};

// ------------------------------------------------------------------------------- context
struct Mesh {
  int64_t ne = 0;
  std::vector<double> verts;   // nv x 3
  std::vector<int32_t> tris;   // ne x 3
  DevBuf elem64;               // Elem64[ne]
  DevBuf tri64;                // double[ne][9] vertices
  DevBuf c32, n32;             // float4[ne]: (centroid, h), (normal, area)
  DevBuf c64, n64;             // D4[ne]:     (centroid, h), (normal, area)
  DevBuf q4_64, q7_64;         // double4-like [ne][4|7][4]
  DevBuf q4_32, q7_32;         // float4 [ne][4|7]
  DevBuf q4_32lo, c32lo;       // float4: low parts (x - (float)x) of the 4-point rule points and
                               // of the centroids, for float-float source-target distances
  DevBuf near_ptr, near_col;   // int32 CSR
  int64_t nnz = 0;
  std::vector<int32_t> h_near_ptr, h_near_col;
  double diam = 0;             // bounding-box diagonal (bounds every source-target distance)
  DevBuf self_pts;             // SelfPt[ne][3 kDuffyN^2]: own-element Duffy points (float-float)
};

// One Duffy point of an element's own integral (frequency independent): distance r, unit
// direction rh and weight w, each as a float-float pair (hi, lo).
struct SelfPt {
  float4 a;  // r_hi, r_lo, rh0_hi, rh0_lo
  float4 b;  // rh1_hi, rh1_lo, rh2_hi, rh2_lo
  float2 c;  // w_hi, w_lo
};

struct Material {
  double mu = 0, nu = 0, rho = 0;
  bool set = false;
};

struct BC {
  bool set = false;
  int profile = BEM_PROFILE_STEP;
  std::vector<int8_t> type;    // per element
  std::vector<double> value;   // ne x 3
  DevBuf d_type;               // int8[ne]
  DevBuf d_value;              // double[ne][3]
};

// Frequency-set data: constants and own-element blocks for a batch of frequencies.
struct FreqSet {
  int64_t F = 0;
  std::vector<double> s;       // 2F
  DevBuf fc64, fc32;           // FreqC<double/float>[F]
  DevBuf Tself, Gself;         // cx<double>[F][ne][9]
  DevBuf Minv64;               // cx<double>[F][ne][9] inverse of A_ii
  DevBuf Minv32;               // cx<float>[F][ne][9]
  DevBuf pfac;                 // cx<double>[F] profile factor
  DevBuf fcdf;                 // float-float frequency constants for the df64 residual
  bool valid = false;
};

// Optional CUDA-event timing of kernel classes (enabled by bem_profile).
enum ProfKind { PK_FAR32 = 0, PK_FAR64, PK_NEAR32, PK_NEAR64, PK_SELF, PK_VEC, PK_RES64, PK_HAPPLY, PK_HBUILD, PK_COUNT };
struct ProfRec {
  int kind;
  cudaEvent_t a, b;
  int64_t work;  // frequencies covered by the launch
};

// Learned / nearest warm start: stored solutions, POD basis and MLP parameters.
struct WarmStart {
  int64_t N = 0;              // unknowns of the stored solutions
  std::vector<double> s;      // 2J: frequencies of the stored solutions
  DevBuf X;                   // cx<double>[J][N]
  DevBuf Phi;                 // cx<double>[r][N] POD basis
  int r = 0;
  DevBuf params;              // float MLP parameters (W1, b1, W2, b2, W3, b3)
  DevBuf act;                 // activations scratch
  double omega = 1;
  bool trained = false;
  // rational-prediction weights (BEM_WARM_VF, set by the AFS driver for its next solve):
  // x(vf_s[f]) ~ sum_j vf_w[f][j] X[j] over the first vf_J stored solutions
  std::vector<double> vf_s;         // 2F: frequencies the weights are for
  std::vector<cx<double>> vf_w;     // [F][vf_J]
  int64_t vf_J = 0;
};

// H-matrix far field (hmatrix.cu): structure of the current mesh and parameters, and the
// FP32 low-rank factors of the current frequency set.
struct HMat {
  bem_hmatrix_params prm{};     // enable = 0: off
  bool have_structure = false;  // tree, partition and their device copies are current
  hm::Tree tree;
  hm::Partition part;
  DevBuf perm;                  // int32[ne]: tree position -> element
  DevBuf lr;                    // int4[n_lr]: low-rank block (t0, tn, s0, sn) as tree positions
  DevBuf tgrp;                  // int4[n_tg]: target cluster (t0, tn, first, count <= 4) of tblk
  DevBuf tblk;                  // int32[n_lr]: low-rank blocks grouped by target cluster
  DevBuf dgrp;                  // int4[n_dg]: target leaf (t0, tn, first, count <= 4) of dsrc
  DevBuf dsrc;                  // int2[n_dn]: dense blocks' source leaves (s0, sn), grouped
  int64_t n_lr = 0, n_tg = 0, n_dg = 0, n_dn = 0, lr_pairs = 0, dn_pairs = 0;
  int max_lr = 0;               // largest side (elements) of a low-rank block
  int max_leaf = 0;             // largest leaf
  bool built = false;           // factors for the current frequency set
  int64_t F = 0;
  DevBuf rank;                  // int32[F][n_lr]
  DevBuf fptr;                  // (float2*)[F][n_lr]: U (3 tn x k) then V (3 sn x k) of a block
  std::vector<std::unique_ptr<DevBuf>> chunks;  // factor storage
  DevBuf scratch, items, dst, capped, brank;
  bem_hmatrix_info info{};
};

}  // namespace bem

struct bem_ctx {
  int device = 0;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  std::string err;
  bem_options opt{};
  bem::Mesh mesh;
  bem::Material mat;
  bem::BC bc;
  bem::FreqSet fs;
  bem::WarmStart warm;
  bem::HMat hm;
  // scratch buffers for vectors (grow-only)
  bem::DevBuf io_a, io_b;       // staging for ABI copies
  bem::DevBuf io_c, io_d, io_e; // staging for the FSM calls (samples, times, output, dofs)
  bem::DevBuf fsm_table;        // FSM phase table [nt][nc] complex
  bem::DevBuf active;           // int32[F] per-frequency active flags
  bem::DevBuf flist_d;          // int32 frequency list of the current operator launch
  std::vector<int32_t> flist_h;
  bem::DevBuf groups_d;         // FarGroup per CTA frequency group of the current far launches
  std::vector<bem::FarGroup> groups_h;
  int64_t rec_entries = 0;      // leading list entries in equally spaced runs (FP32 recurrence)
  bem::DevBuf zero_pfac;        // zero profile factors: the residual sweep as an operator
  bool fp64_op_df = false;      // FP64 GMRES applies the float-float operator (mixed fallback)
  bem::DevBuf yacc;             // FP64 far-field accumulator [F][ne][3] complex
  int64_t launches = 0;         // kernels launched (accumulated, reset per call)
  int64_t f32_applies = 0, f64_applies = 0;
  std::vector<bem_tune_entry> tune;  // FP32 far-field launch shapes (empty: FarShape defaults)
  bool tune_forced = false;          // the autotuner's trial shape overrides the table
  bem::FarShape tune_force;
  int n_sm = 0;                      // multiprocessors of the device
  int64_t warm_learned_gains = 0; // frequencies of the last solve whose learned start, combined with
                                  // the nearest solution, beat that solution alone by >= 10 %
  // kernel timing
  bool prof = false;
  std::vector<bem::ProfRec> prof_recs;
  std::vector<cudaEvent_t> prof_pool;
  double prof_ms[bem::PK_COUNT] = {0};
  int64_t prof_n[bem::PK_COUNT] = {0};
  int64_t prof_work[bem::PK_COUNT] = {0};
};

namespace bem {

// ------------------------------------------------------------------------------- host API
// geometry.cu
void build_geometry(bem_ctx* ctx);
void build_near_lists(bem_ctx* ctx);
MatC<double> mat_constants64(const Material& m);
MatC<float> mat_constants32(const Material& m);
// df_self: form the own-element Duffy sums in float-float (mixed-precision solves, whose
// FP64-class residual tolerates ~1e-12 block errors); else in FP64 (FP64 solves, parity checks).
void prepare_frequencies(bem_ctx* ctx, const double* s_host, int64_t F, bool df_self = false);
void element_blocks(bem_ctx* ctx, double sr, double si, const int32_t* rows,
                    const int32_t* cols, int64_t npairs, cx<double>* H, cx<double>* G);

// operator.cu
// y[f] = Op(s_f) x[f] for the frequencies in flist (null = all).
// which = BEM_APPLY_A or BEM_APPLY_K.  x, y device pointers [F][ne][3] complex.
void apply_operator64(bem_ctx* ctx, const cx<double>* x, cx<double>* y, int which,
                      const std::vector<int32_t>* flist);
void apply_operator32(bem_ctx* ctx, const cx<float>* x, cx<float>* y, int which,
                      const std::vector<int32_t>* flist);
// r[f] = K(s_f) k_f - A(s_f) x[f] in FP64 in one sweep (k = profile(s) * known data)
void residual64(bem_ctx* ctx, const cx<double>* x, cx<double>* r, const std::vector<int32_t>* flist);
// the same with the far field in float-float arithmetic on the FP32 pipes (resid_df.cu)
void residual_df(bem_ctx* ctx, const cx<double>* x, cx<double>* r, const std::vector<int32_t>* flist,
                 const cx<double>* pfac_override = nullptr);
// y = A(s) x with the float-float sweeps (FP64-class, ~1e-10 relative) for the listed frequencies
void apply_operator_df(bem_ctx* ctx, const cx<double>* x, cx<double>* y, const std::vector<int32_t>* flist);
void build_freq_df(bem_ctx* ctx, const double* s, int64_t F);
// own-element Duffy sums in float-float: out[F][ne][13] = (psi, chi rh rh (6), T remainder a (3),
// b (3)) per frequency and element (resid_df.cu)
void self_sums_df(bem_ctx* ctx, cx<double>* out);
// helpers shared by the far kernels: stage the frequency list + zero the FP64 accumulator, and
// the FP64 near-field/own-element pass of the residual
int64_t stage_flist(bem_ctx* ctx, const std::vector<int32_t>* flist, int rec_ft);
void near_residual64(bem_ctx* ctx, const cx<double>* x, cx<double>* r, int64_t nfl);
void apply_precond64(bem_ctx* ctx, const cx<double>* x, cx<double>* y, const int32_t* active);
void apply_precond32(bem_ctx* ctx, const cx<float>* x, cx<float>* y, const int32_t* active);
void known_data(bem_ctx* ctx, cx<double>* out);  // profile(s_f) * bc_value, [F][ne][3]

// gmres.cu
void solve_batch(bem_ctx* ctx, cx<double>* x_dev, bem_solve_stats* st,
                 std::vector<int32_t>& iters, std::vector<int32_t>& refines,
                 std::vector<double>& resid, std::vector<int32_t>& status);

// kernel timing: brackets the launches issued between begin and end with two events
struct ProfScope {
  bem_ctx* c;
  int kind;
  cudaEvent_t a = nullptr, b = nullptr;
  int64_t work;
  ProfScope(bem_ctx* ctx, int k, int64_t w = 0);
  ~ProfScope();
};
void prof_collect(bem_ctx* ctx);  // synchronises and folds finished records into totals

// afs.cu: solve a frequency list (prepared inside) with the context's options, including the
// two-pass sweep of BEM_WARM_SWEEP; per-frequency statistics in list order
void solve_frequency_list(bem_ctx* ctx, const double* s_host, int64_t ns, cx<double>* x_dev,
                          std::vector<int32_t>& it, std::vector<int32_t>& rf, std::vector<double>& res,
                          std::vector<int32_t>& status);

// tune.cu: the shape of an FP32 far-field launch of nfl frequencies on the context's mesh
FarShape far32_shape(bem_ctx* ctx, int64_t nfl);

// hmatrix.cu: H-matrix far field.  hm_active: enabled for the context's mesh.  hm_far32: the
// far-field sums of the listed (staged) frequencies into the FP64 accumulator, building the
// factors first when the frequency set changed.  hm_invalidate: drop the factors (and, with
// structure = true, the tree and partition).
bool hm_active(bem_ctx* ctx);
void hm_far32(bem_ctx* ctx, const cx<float>* x, int64_t nfl);
void hm_invalidate(bem_ctx* ctx, bool structure);

// fsm.cu
void fsm_check_args(int64_t nc, int64_t m, double eta, double period, int64_t nt, int window);
void fsm_launch(const cx<double>* h, int64_t nc, int64_t m, double eta, double period,
                const double* t, int64_t nt, int window, double* out, cx<double>* table,
                cudaStream_t st);
void gather_dofs(bem_ctx* ctx, const cx<double>* x, int64_t N, int64_t F, const int64_t* dofs_dev,
                 int64_t nd, cx<double>* out);

// error handling shared by the entry points: runs fn, turns exceptions into codes + messages
void set_global_error(const std::string& m);
template <class Fn>
int guarded_call(bem_ctx* ctx, Fn&& fn) {
  try {
    if (!ctx) throw Error(BEM_ERR_INVALID_ARG, "null context");
    BEM_CUDA(cudaSetDevice(ctx->device));
    ctx->launches = 0;
    fn();
    return BEM_OK;
  } catch (const Error& e) {
    if (ctx) ctx->err = e.what();
    return e.code;
  } catch (const std::exception& e) {
    if (ctx) ctx->err = e.what();
    return BEM_ERR_INVALID_ARG;
  }
}
void need_problem(bem_ctx* ctx);  // mesh, material and boundary conditions set

// mlp.cu
void warm_store(bem_ctx* ctx, const double* s, int64_t ns, const cx<double>* x_dev);
void warm_train(bem_ctx* ctx, const bem_warm_params& prm, bem_warm_stats* out);
void warm_initial(bem_ctx* ctx, int mode, const double* s, int64_t F, cx<double>* x0);
void mlp_eval(bem_ctx* ctx, int r, const float* params_h, const float* U_h, int B, const float* T_h,
              float* Y_h, float* grads_h, double* loss_h);
int64_t mlp_n_params(int r);

// helpers
inline int grid_for(int64_t n, int block) { return (int)((n + block - 1) / block); }
bool is_device_ptr(const void* p);
void narrow_array(bem_ctx* ctx, const cx<double>* a, cx<float>* b, int64_t n);
void widen_array(bem_ctx* ctx, const cx<float>* a, cx<double>* b, int64_t n);
void copy_in(bem_ctx* ctx, void* dst_dev, const void* src, size_t bytes);
void copy_out(bem_ctx* ctx, void* dst, const void* src_dev, size_t bytes);

}  // namespace bem
