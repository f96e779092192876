// Adaptive frequency sampling driver (Sec. 3, Algorithm AFS) and the C ABI of vector fitting.
//
// The driver runs on the host; every BEM analysis it requests is one batched GPU solve
// (bem_solve_frequencies' machinery) whose observed unknowns are gathered back to the host.
//   init     J0 frequencies s_j = eta + i Omega [1 - cos(j pi / (2 (J0 - 1)))] (the printed
//            cosine argument lacks the pi; read as above)
//   step     VF fits of orders M_H = floor(J / alpha_H) and M_L = floor(J / alpha_L)
//            (Eq. (fit-ords)) on the ORFs (each scaled by its largest sample), residues of all
//            observed unknowns; e_k = max|f_kH - f_kL| / max|f_kH| on a uniform grid of
//            n_grid frequencies in [0, Omega] (Eq. (ferr)); s_new = grid argmax of
//            |f_kH - f_kL| for the ORF k with the largest e_k (Eqs. (snew), (snew1)), skipping
//            grid points within 1.5 spacings of a sample (batch > 1, a variant: further
//            argmaxes of the same curve after masking +-Omega/(2J) around each pick, kept while
//            >= 0.1 of the first, all solved in one batch); E1 (Eq. (stop-E1), trapezoidal on nt
//            times in [0, T], E1 = inf at the first step) and E2 = max e_k over the test
//            unknowns (Eq. (stop-E2))
//   stop     when E1 < E1bar and E2 < E2bar at a step and at the J_c steps that follow
//            (Eq. (converge) and the validation stage)
//   output   time responses of the observed unknowns by Eq. (vf-td) with the final M_H fit.
// Time responses sum Eq. (vf-td) over the fitted poles left of the sampling line Re s = eta
// only: the Bromwich integral of Eq. (invLap) along the contour the samples lie on (placed to
// the right of every singularity, Sec. 2.2) collects exactly those residues, so a fitted pole
// right of the line is outside the region the data describe and would otherwise blow up as
// e^{a t}.
#include <chrono>
#include <cstring>
#include <future>
#include <limits>

#include "kernel_math.cuh"
#include "vf_host.h"

using bem::vfit::cd;

namespace bem {

namespace {

double trapz(const std::vector<double>& y, const std::vector<double>& t, int K, int k) {
  double acc = 0;
  for (size_t j = 1; j < t.size(); ++j) acc += 0.5 * (t[j] - t[j - 1]) * (y[j * K + k] + y[(j - 1) * K + k]);
  return acc;
}

struct StepOut {
  vfit::Model H;
  std::vector<double> e;     // per observed unknown
  std::vector<double> diff;  // grid x n_obs |fH - fL|
  std::vector<double> h;     // nt x n_obs time response of the H fit
};

StepOut afs_step(const std::vector<cd>& s, const std::vector<cd>& F, int nobs, int K,
                 const bem_afs_params& p, const std::vector<cd>& grid, const std::vector<double>& t) {
  const int J = (int)s.size();
  const int MH = (int)std::floor(J / p.alpha_H), ML = (int)std::floor(J / p.alpha_L);
  // ORF columns scaled by their largest sample for pole identification
  std::vector<cd> Fo((size_t)J * K);
  for (int k = 0; k < K; ++k) {
    double mx = 0;
    for (int j = 0; j < J; ++j) mx = std::max(mx, std::abs(F[(size_t)j * nobs + k]));
    if (mx == 0) mx = 1;
    for (int j = 0; j < J; ++j) Fo[(size_t)j * K + k] = F[(size_t)j * nobs + k] / mx;
  }
  std::vector<int> cols(K);
  for (int k = 0; k < K; ++k) cols[k] = k;
  // the two fits are independent: f_L on a second host thread (its exceptions rethrown here)
  auto fut_L = std::async(std::launch::async,
                          [&] { return vfit::fit_poles(s, Fo, K, cols, ML, p.omega_max, p.vf_iters, 1e-10); });
  const vfit::Poles PH = vfit::fit_poles(s, Fo, K, cols, MH, p.omega_max, p.vf_iters, 1e-10);
  const vfit::Poles PL = fut_L.get();
  StepOut o;
  o.H = vfit::residues(s, F, nobs, PH);
  const vfit::Model L = vfit::residues(s, F, nobs, PL);
  std::vector<cd> fH, fL;
  vfit::evaluate(o.H, grid, fH);
  vfit::evaluate(L, grid, fL);
  o.e.assign(nobs, 0.0);
  o.diff.assign(grid.size() * nobs, 0.0);
  std::vector<double> mxH(nobs, 0.0);
  for (size_t g = 0; g < grid.size(); ++g)
    for (int k = 0; k < nobs; ++k) {
      const double d = std::abs(fH[g * nobs + k] - fL[g * nobs + k]);
      o.diff[g * nobs + k] = d;
      o.e[k] = std::max(o.e[k], d);
      mxH[k] = std::max(mxH[k], std::abs(fH[g * nobs + k]));
    }
  for (int k = 0; k < nobs; ++k) o.e[k] /= std::max(mxH[k], 1e-300);
  vfit::time_response(o.H, t, o.h, p.eta);
  return o;
}

}  // namespace

// Rational-prediction weights (BEM_WARM_VF).  With the fit's poles a_m, the residues of every
// unknown follow by least squares over the stored solutions x_j = x(s_j) (the paper's residue
// identification, Sec. 2.3): min |Phi R - X| with Phi[j][m] = 1/(s_j - a_m).  The prediction at
// s*, phi*^T R = phi*^T Phi^+ X, is a combination of the stored solutions with weights
// w = conj(Q) u, where Phi D^{-1} = Q R' (modified Gram-Schmidt on the unit-scaled columns D) and
// R'^T u = D^{-1} phi*.  Columns whose pivot falls below 1e-12 of the largest are dropped.
// Returns false (no weights) when fewer solutions than poles are stored.
bool vf_weights(const std::vector<cd>& poles, const std::vector<double>& s_stored, int64_t J,
                const std::vector<cd>& targets, std::vector<cx<double>>& w) {
  const int M = (int)poles.size();
  if (M < 1 || J < M + 1) return false;
  std::vector<cd> Q((size_t)J * M), R((size_t)M * M, cd(0, 0));
  std::vector<double> d(M);
  for (int m = 0; m < M; ++m) {
    double nrm = 0;
    for (int64_t j = 0; j < J; ++j) {
      const cd v = 1.0 / (cd(s_stored[2 * j], s_stored[2 * j + 1]) - poles[m]);
      Q[(size_t)j * M + m] = v;
      nrm += std::norm(v);
    }
    d[m] = nrm > 0 ? std::sqrt(nrm) : 1.0;
    for (int64_t j = 0; j < J; ++j) Q[(size_t)j * M + m] /= d[m];
  }
  for (int m = 0; m < M; ++m) {  // modified Gram-Schmidt
    for (int k = 0; k < m; ++k) {
      cd dot(0, 0);
      for (int64_t j = 0; j < J; ++j) dot += std::conj(Q[(size_t)j * M + k]) * Q[(size_t)j * M + m];
      R[(size_t)k * M + m] = dot;
      for (int64_t j = 0; j < J; ++j) Q[(size_t)j * M + m] -= dot * Q[(size_t)j * M + k];
    }
    double nrm = 0;
    for (int64_t j = 0; j < J; ++j) nrm += std::norm(Q[(size_t)j * M + m]);
    nrm = std::sqrt(nrm);
    R[(size_t)m * M + m] = nrm;
    if (nrm > 0)
      for (int64_t j = 0; j < J; ++j) Q[(size_t)j * M + m] /= nrm;
  }
  double rmax = 0;
  for (int m = 0; m < M; ++m) rmax = std::max(rmax, std::abs(R[(size_t)m * M + m]));
  w.assign(targets.size() * (size_t)J, mk(0.0, 0.0));
  for (size_t f = 0; f < targets.size(); ++f) {
    std::vector<cd> u(M, cd(0, 0));
    for (int m = 0; m < M; ++m) {
      const double rmm = std::abs(R[(size_t)m * M + m]);
      if (rmm <= 1e-12 * rmax) continue;  // dependent column: dropped
      cd acc = 1.0 / (targets[f] - poles[m]) / d[m];
      for (int k = 0; k < m; ++k) acc -= R[(size_t)k * M + m] * u[k];
      u[m] = acc / R[(size_t)m * M + m];
    }
    for (int64_t j = 0; j < J; ++j) {
      cd acc(0, 0);
      for (int m = 0; m < M; ++m) acc += u[m] * std::conj(Q[(size_t)j * M + m]);
      w[f * J + j] = mk(acc.real(), acc.imag());
    }
  }
  return true;
}


// The frequency sweep of BEM_WARM_SWEEP: every other frequency first (zero start), a vector fit
// of order J/2 (Eq. (fit-ords) with alpha 2) to K = 8 unknowns spread over the mesh at those J
// frequencies, then the remaining frequencies from the fit's rational prediction combined with
// the nearest solved frequency (BEM_WARM_VF).  The tolerance and the certification of every
// frequency are unchanged.  Fewer than 8 frequencies, or a failed fit: one batch, zero start.
void solve_frequency_list(bem_ctx* ctx, const double* sh, int64_t ns, cx<double>* x_dev,
                          std::vector<int32_t>& it, std::vector<int32_t>& rf, std::vector<double>& res,
                          std::vector<int32_t>& status) {
  const bool mixed = ctx->opt.precision == BEM_PREC_MIXED;
  const int wmode = ctx->opt.warm_start;
  if (wmode != BEM_WARM_SWEEP || ns < 8) {
    const int saved = ctx->opt.warm_start;
    if (wmode == BEM_WARM_SWEEP) ctx->opt.warm_start = BEM_WARM_ZERO;
    // with the H-matrix far field, at most max_freqs frequencies' factors at a time
    const int64_t chunk = hm_active(ctx) && ctx->hm.prm.max_freqs > 0 ? ctx->hm.prm.max_freqs : ns;
    it.assign(ns, 0);
    rf.assign(ns, 0);
    res.assign(ns, 0.0);
    status.assign(ns, 0);
    try {
      for (int64_t c0 = 0; c0 < ns; c0 += chunk) {
        const int64_t nc = std::min(chunk, ns - c0);
        prepare_frequencies(ctx, sh + 2 * c0, nc, mixed);
        std::vector<int32_t> it_c, rf_c, st_c;
        std::vector<double> res_c;
        solve_batch(ctx, x_dev + c0 * 3 * ctx->mesh.ne, nullptr, it_c, rf_c, res_c, st_c);
        for (int64_t k = 0; k < nc; ++k) {
          it[c0 + k] = it_c[k];
          rf[c0 + k] = rf_c[k];
          res[c0 + k] = res_c[k];
          status[c0 + k] = st_c[k];
        }
      }
    } catch (...) {
      ctx->opt.warm_start = saved;
      throw;
    }
    ctx->opt.warm_start = saved;
    return;
  }
  const int64_t N = 3 * ctx->mesh.ne;
  std::vector<int64_t> idx[2];
  for (int64_t f = 0; f < ns; ++f) idx[f % 2].push_back(f);
  it.assign(ns, 0);
  rf.assign(ns, 0);
  res.assign(ns, 0.0);
  status.assign(ns, 0);
  DevBuf part;
  WarmStart& ws = ctx->warm;
  const int saved = ctx->opt.warm_start;
  try {
    for (int pass = 0; pass < 2; ++pass) {
      const std::vector<int64_t>& I = idx[pass];
      const int64_t F = (int64_t)I.size();
      std::vector<double> sp(2 * F);
      for (int64_t k = 0; k < F; ++k) {
        sp[2 * k] = sh[2 * I[k]];
        sp[2 * k + 1] = sh[2 * I[k] + 1];
      }
      part.reserve(sizeof(cx<double>) * F * N);
      ctx->opt.warm_start = pass == 0 ? BEM_WARM_ZERO : BEM_WARM_VF;
      prepare_frequencies(ctx, sp.data(), F, mixed);
      std::vector<int32_t> it_p, rf_p, st_p;
      std::vector<double> res_p;
      solve_batch(ctx, part.as<cx<double>>(), nullptr, it_p, rf_p, res_p, st_p);
      for (int64_t k = 0; k < F; ++k) {
        it[I[k]] = it_p[k];
        rf[I[k]] = rf_p[k];
        res[I[k]] = res_p[k];
        status[I[k]] = st_p[k];
        BEM_CUDA(cudaMemcpyAsync(x_dev + I[k] * N, part.as<cx<double>>() + k * N, sizeof(cx<double>) * N,
                                 cudaMemcpyDeviceToDevice, ctx->stream));
      }
      if (pass == 1) break;
      // the fit of the first pass and the prediction weights of the second
      ws.s.clear();
      ws.trained = false;
      ws.r = 0;
      ws.vf_J = 0;
      ws.vf_s.clear();
      warm_store(ctx, sp.data(), F, part.as<cx<double>>());
      constexpr int K = 8;
      std::vector<int64_t> dofs(K);
      for (int k = 0; k < K; ++k) dofs[k] = 3 * ((2 * k + 1) * ctx->mesh.ne / (2 * K)) + (k % 3);
      DevBuf ddofs, obs;
      ddofs.reserve(sizeof(int64_t) * K);
      obs.reserve(sizeof(cx<double>) * F * K);
      copy_in(ctx, ddofs.p, dofs.data(), sizeof(int64_t) * K);
      gather_dofs(ctx, part.as<cx<double>>(), N, F, ddofs.as<int64_t>(), K, obs.as<cx<double>>());
      std::vector<cx<double>> hv((size_t)F * K);
      copy_out(ctx, hv.data(), obs.p, sizeof(cx<double>) * F * K);
      std::vector<cd> sv(F), Fo((size_t)F * K);
      double wmax = 0;
      for (int64_t k = 0; k < F; ++k) {
        sv[k] = cd(sp[2 * k], sp[2 * k + 1]);
        wmax = std::max(wmax, std::fabs(sp[2 * k + 1]));
      }
      for (int c = 0; c < K; ++c) {
        double mx = 0;
        for (int64_t k = 0; k < F; ++k) mx = std::max(mx, std::hypot(hv[k * K + c].r, hv[k * K + c].i));
        if (mx == 0) mx = 1;
        for (int64_t k = 0; k < F; ++k) Fo[(size_t)k * K + c] = cd(hv[k * K + c].r, hv[k * K + c].i) / mx;
      }
      std::vector<int> cols(K);
      for (int c = 0; c < K; ++c) cols[c] = c;
      std::vector<cd> targets;
      for (int64_t f : idx[1]) targets.emplace_back(sh[2 * f], sh[2 * f + 1]);
      try {
        const vfit::Poles PH = vfit::fit_poles(sv, Fo, K, cols, (int)(F / 2), std::max(wmax, 1.0), 20, 1e-10);
        const vfit::Model md = vfit::residues(sv, Fo, K, PH);
        if (vf_weights(md.poles, ws.s, F, targets, ws.vf_w)) {
          ws.vf_J = F;
          for (const cd& z : targets) {
            ws.vf_s.push_back(z.real());
            ws.vf_s.push_back(z.imag());
          }
        }
      } catch (const std::exception&) {
        // no prediction: the second pass starts from the nearest solved frequency
      }
    }
  } catch (...) {
    ctx->opt.warm_start = saved;
    throw;
  }
  ctx->opt.warm_start = saved;
  BEM_CUDA(cudaStreamSynchronize(ctx->stream));
}

}  // namespace bem

using namespace bem;

extern "C" {

int bem_default_afs_params(bem_afs_params* p) {
  if (!p) return BEM_ERR_INVALID_ARG;
  std::memset(p, 0, sizeof *p);
  p->J0 = 16;
  p->alpha_H = 2.0;
  p->alpha_L = 2.3;
  p->E1bar = 1e-4;
  p->E2bar = 2e-3;
  p->Jc = 3;
  p->n_grid = 4096;
  p->nt = 512;
  p->max_samples = 400;
  p->batch = 1;
  p->vf_iters = 20;
  return BEM_OK;
}

int bem_vf_fit(const double* s, int64_t J, const double* F, int64_t K, const int32_t* fit_cols,
               int32_t n_fit_cols, int32_t M, double omega_max, int32_t n_iter, double* poles,
               double* residues) {
  try {
    BEM_REQUIRE(s && F && poles && residues, "null pointer");
    BEM_REQUIRE(J >= 1 && K >= 1 && M >= 1 && M <= J, "need 1 <= M <= J and K >= 1");
    BEM_REQUIRE(omega_max > 0 && n_iter >= 1, "omega_max > 0 and n_iter >= 1 required");
    std::vector<cd> sv(J), Fv((size_t)J * K);
    for (int64_t j = 0; j < J; ++j) sv[j] = cd(s[2 * j], s[2 * j + 1]);
    for (int64_t q = 0; q < J * K; ++q) Fv[q] = cd(F[2 * q], F[2 * q + 1]);
    std::vector<int> cols;
    if (fit_cols) {
      for (int32_t c = 0; c < n_fit_cols; ++c) {
        BEM_REQUIRE(fit_cols[c] >= 0 && fit_cols[c] < K, "fit column out of range");
        cols.push_back(fit_cols[c]);
      }
    } else {
      for (int64_t k = 0; k < K; ++k) cols.push_back((int)k);
    }
    BEM_REQUIRE(!cols.empty(), "no response selected for pole identification");
    const vfit::Poles P = vfit::fit_poles(sv, Fv, (int)K, cols, M, omega_max, n_iter, 1e-10);
    const vfit::Model md = vfit::residues(sv, Fv, (int)K, P);
    for (int m = 0; m < M; ++m) {
      poles[2 * m] = md.poles[m].real();
      poles[2 * m + 1] = md.poles[m].imag();
    }
    for (int64_t q = 0; q < K * M; ++q) {
      residues[2 * q] = md.R[q].real();
      residues[2 * q + 1] = md.R[q].imag();
    }
    return BEM_OK;
  } catch (const Error& e) {
    set_global_error(e.what());
    return e.code;
  } catch (const std::exception& e) {
    set_global_error(e.what());
    return BEM_ERR_BREAKDOWN;
  }
}

int bem_vf_eval(const double* poles, int32_t M, const double* residues, int64_t K, const double* s,
                int64_t n, double* out) {
  try {
    BEM_REQUIRE(poles && residues && s && out && M >= 1 && K >= 1 && n >= 0, "bad argument");
    vfit::Model md;
    md.K = (int)K;
    for (int m = 0; m < M; ++m) md.poles.emplace_back(poles[2 * m], poles[2 * m + 1]);
    for (int64_t q = 0; q < K * M; ++q) md.R.emplace_back(residues[2 * q], residues[2 * q + 1]);
    std::vector<cd> sv(n), f;
    for (int64_t j = 0; j < n; ++j) sv[j] = cd(s[2 * j], s[2 * j + 1]);
    vfit::evaluate(md, sv, f);
    for (size_t q = 0; q < f.size(); ++q) {
      out[2 * q] = f[q].real();
      out[2 * q + 1] = f[q].imag();
    }
    return BEM_OK;
  } catch (const Error& e) {
    set_global_error(e.what());
    return e.code;
  }
}

int bem_vf_time(const double* poles, int32_t M, const double* residues, int64_t K, const double* t,
                int64_t nt, double eta, double* out) {
  try {
    BEM_REQUIRE(poles && residues && t && out && M >= 1 && K >= 1 && nt >= 0, "bad argument");
    vfit::Model md;
    md.K = (int)K;
    for (int m = 0; m < M; ++m) md.poles.emplace_back(poles[2 * m], poles[2 * m + 1]);
    for (int64_t q = 0; q < K * M; ++q) md.R.emplace_back(residues[2 * q], residues[2 * q + 1]);
    std::vector<double> tv(t, t + nt), h;
    vfit::time_response(md, tv, h, eta);
    std::memcpy(out, h.data(), sizeof(double) * h.size());
    return BEM_OK;
  } catch (const Error& e) {
    set_global_error(e.what());
    return e.code;
  }
}

int bem_afs(bem_ctx* ctx, const bem_afs_params* prm, const int64_t* orf, int64_t K,
            const int64_t* test, int64_t Kt, const double* t_out, int64_t nt_out, double* resp_out,
            bem_afs_stats* st) {
  return guarded_call(ctx, [&] {
    need_problem(ctx);
    BEM_REQUIRE(prm && orf && K >= 1 && Kt >= 0 && (Kt == 0 || test), "bad observation lists");
    const bem_afs_params p = *prm;
    BEM_REQUIRE(p.eta > 0 && p.omega_max > 0 && p.T > 0, "eta, omega_max and T must be > 0");
    BEM_REQUIRE(p.J0 >= 3 && p.alpha_H > 0 && p.alpha_L > p.alpha_H, "need J0 >= 3, 0 < alpha_H < alpha_L");
    BEM_REQUIRE(p.Jc >= 0 && p.n_grid >= 16 && p.nt >= 2 && p.max_samples >= p.J0 && p.vf_iters >= 1,
                "bad AFS parameters");
    BEM_REQUIRE(p.batch >= 1 && p.batch <= 64, "batch must be in [1, 64]");
    const int64_t N = 3 * ctx->mesh.ne;
    const int nobs = (int)(K + Kt);
    std::vector<int64_t> dofs(nobs);
    for (int64_t k = 0; k < K; ++k) dofs[k] = orf[k];
    for (int64_t k = 0; k < Kt; ++k) dofs[K + k] = test[k];
    for (int64_t d : dofs) BEM_REQUIRE(d >= 0 && d < N, "observed unknown out of range");
    DevBuf ddofs, obs;
    ddofs.reserve(sizeof(int64_t) * nobs);
    copy_in(ctx, ddofs.p, dofs.data(), sizeof(int64_t) * nobs);
    double t_solve = 0, t_fit = 0, t_train = 0;
    std::vector<int32_t> solve_iters;
    // warm start: the memory holds this run's own samples only
    const int wmode = ctx->opt.warm_start == BEM_WARM_SWEEP ? BEM_WARM_VF : ctx->opt.warm_start;
    const int retrain = p.warm_retrain > 0 ? p.warm_retrain : 4;
    constexpr int kWarmCap = 256;  // solutions the network can be trained on
    int warm_trainings = 0, last_train = 0;
    int64_t learned_gains = 0;
    if (wmode != BEM_WARM_ZERO) {
      ctx->warm.s.clear();
      ctx->warm.trained = false;
      ctx->warm.r = 0;
    }
    bem_warm_params wprm;
    bem_default_warm_params(&wprm);
    // one batched solve of the listed frequencies, observed unknowns back to the host
    auto solve = [&](const std::vector<cd>& sl, std::vector<cd>& Fout) {
      const auto t0 = std::chrono::steady_clock::now();
      const int64_t F = (int64_t)sl.size();
      std::vector<double> sr(2 * F);
      for (int64_t f = 0; f < F; ++f) {
        sr[2 * f] = sl[f].real();
        sr[2 * f + 1] = sl[f].imag();
      }
      prepare_frequencies(ctx, sr.data(), F, ctx->opt.precision == BEM_PREC_MIXED);
      ctx->io_a.reserve(sizeof(cx<double>) * F * N);
      std::vector<int32_t> it, rf, status;
      std::vector<double> res;
      solve_batch(ctx, ctx->io_a.as<cx<double>>(), nullptr, it, rf, res, status);
      for (int64_t f = 0; f < F; ++f)
        if (status[f] != 0) throw Error(BEM_ERR_NOT_CONVERGED, "AFS: a frequency solve did not converge");
      obs.reserve(sizeof(cx<double>) * F * nobs);
      gather_dofs(ctx, ctx->io_a.as<cx<double>>(), N, F, ddofs.as<int64_t>(), nobs, obs.as<cx<double>>());
      std::vector<cx<double>> h(F * nobs);
      copy_out(ctx, h.data(), obs.p, sizeof(cx<double>) * F * nobs);
      Fout.resize(F * nobs);
      for (int64_t q = 0; q < F * nobs; ++q) Fout[q] = cd(h[q].r, h[q].i);
      for (int64_t f = 0; f < F; ++f) solve_iters.push_back(it[f]);
      learned_gains += ctx->warm_learned_gains;
      if (wmode != BEM_WARM_ZERO) {
        const int64_t room = kWarmCap - (int64_t)ctx->warm.s.size() / 2;
        if (room > 0) warm_store(ctx, sr.data(), std::min(F, room), ctx->io_a.as<cx<double>>());
      }
      t_solve += std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
      // the learned start: train after the initial frequencies, then every `retrain` samples
      const int J = (int)(ctx->warm.s.size() / 2);
      if (wmode == BEM_WARM_MLP && J >= 2 && (warm_trainings == 0 || J - last_train >= retrain)) {
        const auto t1 = std::chrono::steady_clock::now();
        warm_train(ctx, wprm, nullptr);
        t_train += std::chrono::duration<double>(std::chrono::steady_clock::now() - t1).count();
        ++warm_trainings;
        last_train = J;
      }
    };
    std::vector<cd> s, F;
    for (int j = 0; j < p.J0; ++j)
      s.emplace_back(p.eta, p.omega_max * (1.0 - std::cos(j * kPi / (2.0 * (p.J0 - 1)))));
    solve(s, F);
    std::vector<cd> grid(p.n_grid);
    for (int g = 0; g < p.n_grid; ++g) grid[g] = cd(p.eta, p.omega_max * g / (p.n_grid - 1));
    const double dgrid = p.omega_max / (p.n_grid - 1);
    std::vector<double> t(p.nt);
    for (int j = 0; j < p.nt; ++j) t[j] = p.T * j / (p.nt - 1);
    std::vector<double> E1s, E2s, h_prev;
    int ok_run = 0;
    StepOut so;
    while (true) {
      const auto t0 = std::chrono::steady_clock::now();
      so = afs_step(s, F, nobs, (int)K, p, grid, t);
      double E1 = std::numeric_limits<double>::infinity();
      if (!h_prev.empty()) {
        E1 = 0;
        for (int64_t k = K; k < nobs; ++k) {
          std::vector<double> d2(t.size()), f2(t.size());
          for (size_t j = 0; j < t.size(); ++j) {
            const double a = so.h[j * nobs + k], b = h_prev[j * nobs + k];
            d2[j] = (a - b) * (a - b);
            f2[j] = a * a;
          }
          const double num = trapz(d2, t, 1, 0), den = trapz(f2, t, 1, 0);
          E1 = std::max(E1, num / std::max(den, 1e-300));
        }
      }
      double E2 = 0;
      for (int64_t k = K; k < nobs; ++k) E2 = std::max(E2, so.e[k]);
      E1s.push_back(E1);
      E2s.push_back(E2);
      h_prev = so.h;
      ok_run = (E1 < p.E1bar && E2 < p.E2bar) ? ok_run + 1 : 0;
      t_fit += std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
      if (ok_run >= p.Jc + 1 || (int)s.size() >= p.max_samples) break;
      int kmax = 0;
      for (int k = 1; k < K; ++k)
        if (so.e[k] > so.e[kmax]) kmax = k;
      // discrepancy curve of that ORF, grid points within 1.5 spacings of a sample excluded
      std::vector<double> d(p.n_grid);
      for (int g = 0; g < p.n_grid; ++g) {
        d[g] = so.diff[(size_t)g * nobs + kmax];
        for (const cd& sj : s)
          if (std::fabs(grid[g].imag() - sj.imag()) < 1.5 * dgrid) {
            d[g] = -1.0;
            break;
          }
      }
      // the paper's s_new; with batch > 1 further argmaxes after masking +-Omega/(2J) around
      // each pick, kept while at least 0.1 of the first pick's discrepancy
      const int want = std::min(p.batch, p.max_samples - (int)s.size());
      const double half = p.omega_max / (2.0 * (double)s.size());
      std::vector<cd> picks;
      double first = 0;
      for (int b = 0; b < want; ++b) {
        int gbest = 0;
        for (int g = 1; g < p.n_grid; ++g)
          if (d[g] > d[gbest]) gbest = g;
        if (b == 0) first = d[gbest];
        else if (d[gbest] < 0.1 * first || d[gbest] < 0) break;
        picks.push_back(grid[gbest]);
        const double wb = grid[gbest].imag();
        for (int g = 0; g < p.n_grid; ++g)
          if (std::fabs(grid[g].imag() - wb) <= half) d[g] = -1.0;
      }
      if (wmode == BEM_WARM_VF) {
        // the next solve starts from the current fit's rational prediction (and the nearest
        // stored solution): weights over the stored solutions for each pick
        WarmStart& ws = ctx->warm;
        const int64_t Js = (int64_t)(ws.s.size() / 2);
        ws.vf_J = 0;
        ws.vf_s.clear();
        if (vf_weights(so.H.poles, ws.s, Js, picks, ws.vf_w)) {
          ws.vf_J = Js;
          for (const cd& z : picks) {
            ws.vf_s.push_back(z.real());
            ws.vf_s.push_back(z.imag());
          }
        }
      }
      std::vector<cd> Fn;
      solve(picks, Fn);
      s.insert(s.end(), picks.begin(), picks.end());
      F.insert(F.end(), Fn.begin(), Fn.end());
    }
    if (resp_out && t_out && nt_out > 0) {
      std::vector<double> tv(nt_out), h;
      copy_out(ctx, tv.data(), t_out, sizeof(double) * nt_out);
      vfit::time_response(so.H, tv, h, p.eta);
      copy_out(ctx, resp_out, h.data(), sizeof(double) * h.size());
    }
    if (st) {
      st->n_samples = (int64_t)s.size();
      st->n_steps = (int64_t)E1s.size();
      st->n_poles = (int32_t)so.H.poles.size();
      st->seconds_solve = t_solve;
      st->seconds_fit = t_fit;
      st->seconds_train = t_train;
      st->warm_trainings = warm_trainings;
      st->warm_learned_gains = (int32_t)learned_gains;
      const int64_t cap = st->capacity;
      for (int64_t j = 0; j < (int64_t)s.size() && j < cap; ++j) {
        if (st->s) {
          st->s[2 * j] = s[j].real();
          st->s[2 * j + 1] = s[j].imag();
        }
        if (st->gmres_iters) st->gmres_iters[j] = solve_iters[j];
      }
      for (int64_t j = 0; j < (int64_t)E1s.size() && j < cap; ++j) {
        if (st->E1) st->E1[j] = E1s[j];
        if (st->E2) st->E2[j] = E2s[j];
      }
      for (int64_t m = 0; m < (int64_t)so.H.poles.size() && m < cap; ++m)
        if (st->poles) {
          st->poles[2 * m] = so.H.poles[m].real();
          st->poles[2 * m + 1] = so.H.poles[m].imag();
        }
    }
  });
}

}  // extern "C"
