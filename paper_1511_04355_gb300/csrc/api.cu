// extern "C" entry points of the library: argument checking, host/device marshalling and
// orchestration of the kernels in geometry.cu, operator.cu and gmres.cu.  Every C++ exception
// is turned into a BEM_ERR_* code plus a message (bem_last_error), so no error escapes the ABI.
#include <algorithm>
#include <chrono>
#include <cstring>
#include <mutex>

#include "kernel_math.cuh"

namespace bem {

bool is_device_ptr(const void* p) {
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();  // clear
    return false;
  }
  return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

// Copies between any host pointer and any device pointer of the context (unified addressing).
void copy_in(bem_ctx* ctx, void* dst_dev, const void* src, size_t bytes) {
  if (!bytes) return;
  BEM_CUDA(cudaMemcpyAsync(dst_dev, src, bytes, cudaMemcpyDefault, ctx->stream));
  BEM_CUDA(cudaStreamSynchronize(ctx->stream));
}
void copy_out(bem_ctx* ctx, void* dst, const void* src, size_t bytes) {
  if (!bytes) return;
  BEM_CUDA(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDefault, ctx->stream));
  BEM_CUDA(cudaStreamSynchronize(ctx->stream));
}

static cudaEvent_t prof_event(bem_ctx* c) {
  if (!c->prof_pool.empty()) {
    cudaEvent_t e = c->prof_pool.back();
    c->prof_pool.pop_back();
    return e;
  }
  cudaEvent_t e;
  BEM_CUDA(cudaEventCreate(&e));
  return e;
}

ProfScope::ProfScope(bem_ctx* ctx, int k, int64_t w) : c(ctx), kind(k), work(w) {
  if (!c->prof) return;
  a = prof_event(c);
  b = prof_event(c);
  cudaEventRecord(a, c->stream);
}

ProfScope::~ProfScope() {
  if (!c->prof || !a) return;
  cudaEventRecord(b, c->stream);
  c->prof_recs.push_back(ProfRec{kind, a, b, work});
}

void prof_collect(bem_ctx* c) {
  for (const ProfRec& r : c->prof_recs) {
    float ms = 0;
    cudaEventSynchronize(r.b);
    if (cudaEventElapsedTime(&ms, r.a, r.b) == cudaSuccess) {
      c->prof_ms[r.kind] += ms;
      c->prof_n[r.kind] += 1;
      c->prof_work[r.kind] += r.work;
    }
    c->prof_pool.push_back(r.a);
    c->prof_pool.push_back(r.b);
  }
  c->prof_recs.clear();
}

__global__ void narrow_kernel(const cx<double>* a, cx<float>* b, int64_t n) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t < n) b[t] = mk((float)a[t].r, (float)a[t].i);
}
__global__ void widen_kernel(const cx<float>* a, cx<double>* b, int64_t n) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t < n) b[t] = mk((double)a[t].r, (double)a[t].i);
}

void narrow_array(bem_ctx* ctx, const cx<double>* a, cx<float>* b, int64_t n) {
  narrow_kernel<<<grid_for(n, 256), 256, 0, ctx->stream>>>(a, b, n);
  BEM_LAUNCHED();
  ctx->launches++;
}
void widen_array(bem_ctx* ctx, const cx<float>* a, cx<double>* b, int64_t n) {
  widen_kernel<<<grid_for(n, 256), 256, 0, ctx->stream>>>(a, b, n);
  BEM_LAUNCHED();
  ctx->launches++;
}

}  // namespace bem

using namespace bem;

namespace {
std::mutex g_err_mu;
std::string g_create_err;

template <class Fn>
int guarded(bem_ctx* ctx, Fn&& fn) {
  return guarded_call(ctx, std::forward<Fn>(fn));
}

void need_mesh(bem_ctx* ctx) {
  if (ctx->mesh.ne <= 0) throw Error(BEM_ERR_NO_MESH, "bem_set_mesh has not been called");
  if (!ctx->mat.set) throw Error(BEM_ERR_INVALID_ARG, "bem_set_material has not been called");
}

void need_bc(bem_ctx* ctx) {
  if (!ctx->bc.set) throw Error(BEM_ERR_INVALID_ARG, "bem_set_bc has not been called");
}
}  // namespace

namespace bem {
void set_global_error(const std::string& m) {
  std::lock_guard<std::mutex> lk(g_err_mu);
  g_create_err = m;
}
void need_problem(bem_ctx* ctx) {
  need_mesh(ctx);
  need_bc(ctx);
}
}  // namespace bem

extern "C" {

int bem_default_options(bem_options* o) {
  if (!o) return BEM_ERR_INVALID_ARG;
  std::memset(o, 0, sizeof *o);
  o->precision = BEM_PREC_MIXED;
  o->restart = 50;
  o->max_iters = 500;
  o->max_refine = 8;
  o->tol = 1e-6;
  o->inner_tol = 1e-6;
  o->warm_start = BEM_WARM_ZERO;
  o->residual_mode = BEM_RESID_DF64;
  return BEM_OK;
}

int bem_create(bem_ctx** out, int device, void* stream) {
  if (!out) return BEM_ERR_INVALID_ARG;
  *out = nullptr;
  bem_ctx* c = nullptr;
  try {
    int n = 0;
    BEM_CUDA(cudaGetDeviceCount(&n));
    if (device < 0 || device >= n) throw Error(BEM_ERR_INVALID_ARG, "device index out of range");
    BEM_CUDA(cudaSetDevice(device));
    c = new bem_ctx();
    c->device = device;
    BEM_CUDA(cudaDeviceGetAttribute(&c->n_sm, cudaDevAttrMultiProcessorCount, device));
    bem_default_options(&c->opt);
    if (stream) {
      c->stream = (cudaStream_t)stream;
    } else {
      BEM_CUDA(cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking));
      c->own_stream = true;
    }
    *out = c;
    return BEM_OK;
  } catch (const Error& e) {
    std::lock_guard<std::mutex> lk(g_err_mu);
    g_create_err = e.what();
    delete c;
    return e.code;
  }
}

int bem_profile(bem_ctx* ctx, int enable) {
  return guarded(ctx, [&] {
    prof_collect(ctx);
    ctx->prof = enable != 0;
    for (int k = 0; k < PK_COUNT; ++k) {
      ctx->prof_ms[k] = 0;
      ctx->prof_n[k] = 0;
      ctx->prof_work[k] = 0;
    }
  });
}

int bem_kernel_time(bem_ctx* ctx, int kind, int64_t* launches, double* ms, int64_t* freq_launches) {
  return guarded(ctx, [&] {
    BEM_REQUIRE(kind >= 0 && kind < PK_COUNT, "unknown kernel class");
    prof_collect(ctx);
    if (launches) *launches = ctx->prof_n[kind];
    if (ms) *ms = ctx->prof_ms[kind];
    if (freq_launches) *freq_launches = ctx->prof_work[kind];
  });
}

int bem_destroy(bem_ctx* ctx) {
  if (!ctx) return BEM_OK;
  cudaSetDevice(ctx->device);
  if (ctx->stream) cudaStreamSynchronize(ctx->stream);
  prof_collect(ctx);
  for (cudaEvent_t e : ctx->prof_pool) cudaEventDestroy(e);
  if (ctx->own_stream && ctx->stream) cudaStreamDestroy(ctx->stream);
  delete ctx;
  return BEM_OK;
}

const char* bem_last_error(const bem_ctx* ctx) {
  if (!ctx) {
    std::lock_guard<std::mutex> lk(g_err_mu);
    return g_create_err.c_str();
  }
  return ctx->err.c_str();
}

int bem_set_options(bem_ctx* ctx, const bem_options* o) {
  return guarded(ctx, [&] {
    BEM_REQUIRE(o, "null options");
    BEM_REQUIRE(o->precision == BEM_PREC_FP64 || o->precision == BEM_PREC_MIXED,
                "precision must be BEM_PREC_FP64 or BEM_PREC_MIXED");
    BEM_REQUIRE(o->restart >= 1 && o->restart <= 512, "restart must be in [1, 512]");
    BEM_REQUIRE(o->max_iters >= 1, "max_iters must be >= 1");
    BEM_REQUIRE(o->tol > 0 && o->tol < 1, "tol must be in (0, 1)");
    BEM_REQUIRE(o->inner_tol > 0 && o->inner_tol < 1, "inner_tol must be in (0, 1)");
    BEM_REQUIRE(o->warm_start >= BEM_WARM_ZERO && o->warm_start <= BEM_WARM_SWEEP, "bad warm_start");
    BEM_REQUIRE(o->residual_mode == BEM_RESID_DF64 || o->residual_mode == BEM_RESID_FP64,
                "residual_mode must be BEM_RESID_DF64 or BEM_RESID_FP64");
    ctx->opt = *o;
  });
}

int bem_set_mesh(bem_ctx* ctx, const double* verts, int64_t nv, const int32_t* tris, int64_t ne) {
  return guarded(ctx, [&] {
    BEM_REQUIRE(verts && tris, "null mesh array");
    BEM_REQUIRE(nv >= 3 && ne >= 1, "mesh needs nv >= 3 and ne >= 1");
    BEM_REQUIRE(ne < (int64_t)1 << 28, "too many elements");
    for (int64_t k = 0; k < 3 * ne; ++k)
      BEM_REQUIRE(tris[k] >= 0 && tris[k] < nv, "triangle vertex index out of range");
    for (int64_t k = 0; k < 3 * nv; ++k) BEM_REQUIRE(std::isfinite(verts[k]), "non-finite vertex");
    Mesh& m = ctx->mesh;
    m.ne = 0;
    m.verts.assign(verts, verts + 3 * nv);
    m.tris.assign(tris, tris + 3 * ne);
    m.ne = ne;
    double lo[3] = {verts[0], verts[1], verts[2]}, hi[3] = {verts[0], verts[1], verts[2]};
    for (int64_t k = 0; k < nv; ++k)
      for (int c = 0; c < 3; ++c) {
        lo[c] = std::min(lo[c], verts[3 * k + c]);
        hi[c] = std::max(hi[c], verts[3 * k + c]);
      }
    m.diam = std::sqrt((hi[0] - lo[0]) * (hi[0] - lo[0]) + (hi[1] - lo[1]) * (hi[1] - lo[1]) +
                       (hi[2] - lo[2]) * (hi[2] - lo[2]));
    ctx->bc.set = false;
    ctx->fs.valid = false;
    hm_invalidate(ctx, true);
    try {
      build_geometry(ctx);
      build_near_lists(ctx);
    } catch (...) {
      m.ne = 0;
      throw;
    }
  });
}

int bem_set_material(bem_ctx* ctx, double mu, double nu, double rho) {
  return guarded(ctx, [&] {
    BEM_REQUIRE(mu > 0 && std::isfinite(mu), "mu must be > 0");
    BEM_REQUIRE(rho > 0 && std::isfinite(rho), "rho must be > 0");
    BEM_REQUIRE(nu > -1.0 && nu < 0.5, "nu must be in (-1, 0.5)");
    ctx->mat.mu = mu;
    ctx->mat.nu = nu;
    ctx->mat.rho = rho;
    ctx->mat.set = true;
    ctx->fs.valid = false;
    hm_invalidate(ctx, false);
  });
}

int bem_set_bc(bem_ctx* ctx, const int8_t* type, const double* value, int profile) {
  return guarded(ctx, [&] {
    if (ctx->mesh.ne <= 0) throw Error(BEM_ERR_NO_MESH, "bem_set_mesh has not been called");
    BEM_REQUIRE(type && value, "null boundary-condition array");
    BEM_REQUIRE(profile == BEM_PROFILE_STEP || profile == BEM_PROFILE_CONSTANT, "unknown time profile");
    const int64_t ne = ctx->mesh.ne;
    for (int64_t e = 0; e < ne; ++e)
      BEM_REQUIRE(type[e] == BEM_BC_TRACTION || type[e] == BEM_BC_DISPLACEMENT, "unknown bc type");
    for (int64_t k = 0; k < 3 * ne; ++k) BEM_REQUIRE(std::isfinite(value[k]), "non-finite bc value");
    BC& b = ctx->bc;
    b.type.assign(type, type + ne);
    b.value.assign(value, value + 3 * ne);
    b.profile = profile;
    b.d_type.reserve(ne);
    b.d_value.reserve(sizeof(double) * 3 * ne);
    copy_in(ctx, b.d_type.p, b.type.data(), ne);
    copy_in(ctx, b.d_value.p, b.value.data(), sizeof(double) * 3 * ne);
    b.set = true;
    ctx->fs.valid = false;
    hm_invalidate(ctx, false);
  });
}

int bem_geometry(bem_ctx* ctx, double* out) {
  return guarded(ctx, [&] {
    if (ctx->mesh.ne <= 0) throw Error(BEM_ERR_NO_MESH, "bem_set_mesh has not been called");
    BEM_REQUIRE(out, "null output");
    static_assert(sizeof(Elem64) == 8 * sizeof(double), "Elem64 layout");
    copy_out(ctx, out, ctx->mesh.elem64.p, sizeof(Elem64) * ctx->mesh.ne);
  });
}

int bem_near_lists(bem_ctx* ctx, int64_t* row_ptr, int32_t* cols, int64_t cap, int64_t* nnz) {
  return guarded(ctx, [&] {
    if (ctx->mesh.ne <= 0) throw Error(BEM_ERR_NO_MESH, "bem_set_mesh has not been called");
    const Mesh& m = ctx->mesh;
    if (nnz) *nnz = m.nnz;
    if (row_ptr)
      for (int64_t i = 0; i <= m.ne; ++i) row_ptr[i] = m.h_near_ptr[i];
    if (cols) {
      BEM_REQUIRE(cap >= m.nnz, "cols capacity smaller than the number of near pairs");
      std::memcpy(cols, m.h_near_col.data(), sizeof(int32_t) * m.nnz);
    }
  });
}

int bem_element_blocks(bem_ctx* ctx, double s_re, double s_im, const int32_t* rows,
                       const int32_t* cols, int64_t npairs, double* H_out, double* G_out) {
  return guarded(ctx, [&] {
    need_mesh(ctx);
    BEM_REQUIRE(rows && cols && H_out && G_out, "null pointer");
    BEM_REQUIRE(npairs >= 1, "npairs must be >= 1");
    BEM_REQUIRE(s_re > 0 && std::isfinite(s_re) && std::isfinite(s_im), "need 0 < Re s");
    element_blocks(ctx, s_re, s_im, rows, cols, npairs, reinterpret_cast<cx<double>*>(H_out),
                   reinterpret_cast<cx<double>*>(G_out));
  });
}

int bem_apply(bem_ctx* ctx, const double* s, int64_t ns, const double* x, double* y,
              int precision, int which) {
  return guarded(ctx, [&] {
    need_mesh(ctx);
    BEM_REQUIRE(s && x && y, "null pointer");
    BEM_REQUIRE(ns >= 1, "ns must be >= 1");
    BEM_REQUIRE(precision == BEM_PREC_FP64 || precision == BEM_PREC_FP32, "precision must be FP64 or FP32");
    BEM_REQUIRE(which == BEM_APPLY_A || which == BEM_APPLY_K, "which must be BEM_APPLY_A or _K");
    std::vector<double> sh(2 * ns);
    copy_out(ctx, sh.data(), s, sizeof(double) * 2 * ns);
    prepare_frequencies(ctx, sh.data(), ns);
    const int64_t n = ns * 3 * ctx->mesh.ne;
    ctx->io_a.reserve(sizeof(cx<double>) * n);
    ctx->io_b.reserve(sizeof(cx<double>) * n);
    copy_in(ctx, ctx->io_a.p, x, sizeof(cx<double>) * n);
    if (precision == BEM_PREC_FP64) {
      apply_operator64(ctx, ctx->io_a.as<cx<double>>(), ctx->io_b.as<cx<double>>(), which, nullptr);
      BEM_CUDA(cudaStreamSynchronize(ctx->stream));
    } else {
      DevBuf xf, yf;
      xf.reserve(sizeof(cx<float>) * n);
      yf.reserve(sizeof(cx<float>) * n);
      narrow_kernel<<<grid_for(n, 256), 256, 0, ctx->stream>>>(ctx->io_a.as<cx<double>>(), xf.as<cx<float>>(), n);
      apply_operator32(ctx, xf.as<cx<float>>(), yf.as<cx<float>>(), which, nullptr);
      widen_kernel<<<grid_for(n, 256), 256, 0, ctx->stream>>>(yf.as<cx<float>>(), ctx->io_b.as<cx<double>>(), n);
      ctx->launches += 2;
      BEM_LAUNCHED();
      BEM_CUDA(cudaStreamSynchronize(ctx->stream));
    }
    copy_out(ctx, y, ctx->io_b.p, sizeof(cx<double>) * n);
  });
}

int bem_rhs(bem_ctx* ctx, const double* s, int64_t ns, double* b_out) {
  return guarded(ctx, [&] {
    need_mesh(ctx);
    need_bc(ctx);
    BEM_REQUIRE(s && b_out && ns >= 1, "bad argument");
    std::vector<double> sh(2 * ns);
    copy_out(ctx, sh.data(), s, sizeof(double) * 2 * ns);
    prepare_frequencies(ctx, sh.data(), ns);
    const int64_t n = ns * 3 * ctx->mesh.ne;
    ctx->io_a.reserve(sizeof(cx<double>) * n);
    ctx->io_b.reserve(sizeof(cx<double>) * n);
    known_data(ctx, ctx->io_a.as<cx<double>>());
    apply_operator64(ctx, ctx->io_a.as<cx<double>>(), ctx->io_b.as<cx<double>>(), BEM_APPLY_K, nullptr);
    copy_out(ctx, b_out, ctx->io_b.p, sizeof(cx<double>) * n);
  });
}

int bem_default_warm_params(bem_warm_params* p) {
  if (!p) return BEM_ERR_INVALID_ARG;
  std::memset(p, 0, sizeof *p);
  p->r_max = 32;
  p->energy_tol = 1e-10;
  p->steps = 2000;
  p->lr = 1e-3;
  p->seed = 20151113ull;
  return BEM_OK;
}

int bem_warm_store(bem_ctx* ctx, const double* s, int64_t ns, const double* x) {
  return guarded(ctx, [&] {
    if (ctx->mesh.ne <= 0) throw Error(BEM_ERR_NO_MESH, "bem_set_mesh has not been called");
    BEM_REQUIRE(s && x && ns >= 1, "bad argument");
    warm_store(ctx, s, ns, reinterpret_cast<const cx<double>*>(x));
  });
}

int bem_warm_clear(bem_ctx* ctx) {
  return guarded(ctx, [&] {
    ctx->warm.s.clear();
    ctx->warm.trained = false;
    ctx->warm.r = 0;
  });
}

int bem_warm_train(bem_ctx* ctx, const bem_warm_params* p, bem_warm_stats* st) {
  return guarded(ctx, [&] {
    BEM_REQUIRE(p, "null parameters");
    BEM_REQUIRE(p->r_max >= 1 && p->r_max <= 64 && p->steps >= 1 && p->lr > 0 && p->energy_tol >= 0 && p->energy_tol < 1,
                "bad warm-start parameters");
    warm_train(ctx, *p, st);
  });
}

int bem_warm_predict(bem_ctx* ctx, int32_t mode, const double* s, int64_t ns, double* x_out) {
  return guarded(ctx, [&] {
    need_mesh(ctx);
    BEM_REQUIRE(s && x_out && ns >= 1, "bad argument");
    BEM_REQUIRE(mode == BEM_WARM_NEAREST || mode == BEM_WARM_MLP, "mode must be BEM_WARM_NEAREST or BEM_WARM_MLP");
    std::vector<double> sh(2 * ns);
    copy_out(ctx, sh.data(), s, sizeof(double) * 2 * ns);
    const int64_t n = ns * 3 * ctx->mesh.ne;
    ctx->io_a.reserve(sizeof(cx<double>) * n);
    warm_initial(ctx, mode, sh.data(), ns, ctx->io_a.as<cx<double>>());
    copy_out(ctx, x_out, ctx->io_a.p, sizeof(cx<double>) * n);
  });
}

int bem_warm_basis(bem_ctx* ctx, double* phi, int32_t* r) {
  return guarded(ctx, [&] {
    BEM_REQUIRE(ctx->warm.trained, "no trained warm start");
    if (r) *r = ctx->warm.r;
    if (phi) copy_out(ctx, phi, ctx->warm.Phi.p, sizeof(cx<double>) * ctx->warm.r * ctx->warm.N);
  });
}

int bem_mlp_eval(bem_ctx* ctx, int32_t r, const float* params, const float* U, int32_t B,
                 const float* T, float* y, float* grads, double* loss) {
  return guarded(ctx, [&] {
    BEM_REQUIRE(params && U && y && r >= 1 && r <= 64 && B >= 1 && B <= 4096, "bad argument");
    BEM_REQUIRE(!T || grads, "targets given without a gradient buffer");
    mlp_eval(ctx, r, params, U, B, T, y, grads, loss);
  });
}

int bem_residual(bem_ctx* ctx, const double* s, int64_t ns, const double* x, double* r, int mode) {
  return guarded(ctx, [&] {
    need_mesh(ctx);
    need_bc(ctx);
    BEM_REQUIRE(s && x && r && ns >= 1, "bad argument");
    BEM_REQUIRE(mode == BEM_RESID_DF64 || mode == BEM_RESID_FP64, "bad residual mode");
    std::vector<double> sh(2 * ns);
    copy_out(ctx, sh.data(), s, sizeof(double) * 2 * ns);
    prepare_frequencies(ctx, sh.data(), ns);
    const int64_t n = ns * 3 * ctx->mesh.ne;
    ctx->io_a.reserve(sizeof(cx<double>) * n);
    ctx->io_b.reserve(sizeof(cx<double>) * n);
    copy_in(ctx, ctx->io_a.p, x, sizeof(cx<double>) * n);
    if (mode == BEM_RESID_DF64) residual_df(ctx, ctx->io_a.as<cx<double>>(), ctx->io_b.as<cx<double>>(), nullptr);
    else residual64(ctx, ctx->io_a.as<cx<double>>(), ctx->io_b.as<cx<double>>(), nullptr);
    copy_out(ctx, r, ctx->io_b.p, sizeof(cx<double>) * n);
  });
}

int bem_precond_apply(bem_ctx* ctx, const double* s, int64_t ns, const double* x, double* y) {
  return guarded(ctx, [&] {
    need_mesh(ctx);
    BEM_REQUIRE(s && x && y && ns >= 1, "bad argument");
    std::vector<double> sh(2 * ns);
    copy_out(ctx, sh.data(), s, sizeof(double) * 2 * ns);
    prepare_frequencies(ctx, sh.data(), ns);
    const int64_t n = ns * 3 * ctx->mesh.ne;
    ctx->io_a.reserve(sizeof(cx<double>) * n);
    ctx->io_b.reserve(sizeof(cx<double>) * n);
    copy_in(ctx, ctx->io_a.p, x, sizeof(cx<double>) * n);
    apply_precond64(ctx, ctx->io_a.as<cx<double>>(), ctx->io_b.as<cx<double>>(), nullptr);
    copy_out(ctx, y, ctx->io_b.p, sizeof(cx<double>) * n);
  });
}

int bem_fsm_eval(bem_ctx* ctx, const double* h, int64_t nc, int64_t m, double eta, double period,
                 const double* t, int64_t nt, int window, double* out) {
  return guarded(ctx, [&] {
    BEM_REQUIRE(h && t && out, "null pointer");
    fsm_check_args(nc, m, eta, period, nt, window);
    ctx->io_c.reserve(sizeof(cx<double>) * nc * m);
    ctx->io_d.reserve(sizeof(double) * nt);
    ctx->io_e.reserve(sizeof(double) * nt * m);
    ctx->fsm_table.reserve(sizeof(cx<double>) * nt * nc);
    copy_in(ctx, ctx->io_c.p, h, sizeof(cx<double>) * nc * m);
    copy_in(ctx, ctx->io_d.p, t, sizeof(double) * nt);
    fsm_launch(ctx->io_c.as<cx<double>>(), nc, m, eta, period, ctx->io_d.as<double>(), nt, window,
               ctx->io_e.as<double>(), ctx->fsm_table.as<cx<double>>(), ctx->stream);
    ctx->launches += 2;
    copy_out(ctx, out, ctx->io_e.p, sizeof(double) * nt * m);
  });
}

int bem_fsm(bem_ctx* ctx, double period, double eta, int64_t nc, const double* t, int64_t nt,
            const int64_t* dofs, int64_t ndofs, double* resp_out, bem_solve_stats* stats) {
  int not_conv = 0;
  const int rc = guarded(ctx, [&] {
    need_mesh(ctx);
    need_bc(ctx);
    BEM_REQUIRE(t && dofs && resp_out, "null pointer");
    fsm_check_args(nc, ndofs, eta, period, nt, 1);
    BEM_REQUIRE(eta > 0, "eta must be > 0");
    const int64_t N = 3 * ctx->mesh.ne;
    std::vector<int64_t> hd(ndofs);
    copy_out(ctx, hd.data(), dofs, sizeof(int64_t) * ndofs);
    for (int64_t d = 0; d < ndofs; ++d) BEM_REQUIRE(hd[d] >= 0 && hd[d] < N, "dof index out of range");
    std::vector<double> s(2 * nc);
    for (int64_t k = 0; k < nc; ++k) {
      s[2 * k] = eta;
      s[2 * k + 1] = 2.0 * kPi * (double)k / period;
    }
    ctx->f32_applies = ctx->f64_applies = 0;
    ctx->io_a.reserve(sizeof(cx<double>) * nc * N);
    std::vector<int32_t> it, rf, status;
    std::vector<double> res;
    solve_frequency_list(ctx, s.data(), nc, ctx->io_a.as<cx<double>>(), it, rf, res, status);
    for (int64_t f = 0; f < nc; ++f) not_conv |= (status[f] != 0);
    DevBuf ddofs;
    ddofs.reserve(sizeof(int64_t) * ndofs);
    copy_in(ctx, ddofs.p, hd.data(), sizeof(int64_t) * ndofs);
    ctx->io_c.reserve(sizeof(cx<double>) * nc * ndofs);
    gather_dofs(ctx, ctx->io_a.as<cx<double>>(), N, nc, ddofs.as<int64_t>(), ndofs, ctx->io_c.as<cx<double>>());
    ctx->io_d.reserve(sizeof(double) * nt);
    ctx->io_e.reserve(sizeof(double) * nt * ndofs);
    ctx->fsm_table.reserve(sizeof(cx<double>) * nt * nc);
    copy_in(ctx, ctx->io_d.p, t, sizeof(double) * nt);
    fsm_launch(ctx->io_c.as<cx<double>>(), nc, ndofs, eta, period, ctx->io_d.as<double>(), nt, 1,
               ctx->io_e.as<double>(), ctx->fsm_table.as<cx<double>>(), ctx->stream);
    ctx->launches += 2;
    copy_out(ctx, resp_out, ctx->io_e.p, sizeof(double) * nt * ndofs);
    if (stats) {
      if (stats->iterations) std::memcpy(stats->iterations, it.data(), sizeof(int32_t) * nc);
      if (stats->refinements) std::memcpy(stats->refinements, rf.data(), sizeof(int32_t) * nc);
      if (stats->residual) std::memcpy(stats->residual, res.data(), sizeof(double) * nc);
      if (stats->status) std::memcpy(stats->status, status.data(), sizeof(int32_t) * nc);
      stats->fp32_operator_applies = ctx->f32_applies;
      stats->fp64_operator_applies = ctx->f64_applies;
      stats->kernel_launches = ctx->launches;
    }
  });
  if (rc != BEM_OK) return rc;
  if (not_conv) {
    ctx->err = "some frequencies did not reach the tolerance (see stats.status)";
    return BEM_ERR_NOT_CONVERGED;
  }
  return BEM_OK;
}

int bem_solve_frequencies(bem_ctx* ctx, const double* s, int64_t ns, double* x_out,
                          bem_solve_stats* stats) {
  int not_conv = 0;
  const int rc = guarded(ctx, [&] {
    const auto t0 = std::chrono::steady_clock::now();
    need_mesh(ctx);
    need_bc(ctx);
    BEM_REQUIRE(s && ns >= 1, "bad frequency list");
    ctx->f32_applies = ctx->f64_applies = 0;
    std::vector<double> sh(2 * ns);
    copy_out(ctx, sh.data(), s, sizeof(double) * 2 * ns);
    const int64_t n = ns * 3 * ctx->mesh.ne;
    ctx->io_a.reserve(sizeof(cx<double>) * n);
    std::vector<int32_t> it, rf, status;
    std::vector<double> res;
    solve_frequency_list(ctx, sh.data(), ns, ctx->io_a.as<cx<double>>(), it, rf, res, status);
    if (x_out) copy_out(ctx, x_out, ctx->io_a.p, sizeof(cx<double>) * n);
    for (int64_t f = 0; f < ns; ++f) not_conv |= (status[f] != 0);
    if (stats) {
      if (stats->iterations) std::memcpy(stats->iterations, it.data(), sizeof(int32_t) * ns);
      if (stats->refinements) std::memcpy(stats->refinements, rf.data(), sizeof(int32_t) * ns);
      if (stats->residual) std::memcpy(stats->residual, res.data(), sizeof(double) * ns);
      if (stats->status) std::memcpy(stats->status, status.data(), sizeof(int32_t) * ns);
      stats->fp32_operator_applies = ctx->f32_applies;
      stats->fp64_operator_applies = ctx->f64_applies;
      stats->kernel_launches = ctx->launches;
      stats->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    }
  });
  if (rc != BEM_OK) return rc;
  if (not_conv) {
    ctx->err = "some frequencies did not reach the tolerance (see stats.status)";
    return BEM_ERR_NOT_CONVERGED;
  }
  return BEM_OK;
}

}  // extern "C"
