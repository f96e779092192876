// Vector fitting on the host, FP64 (Sec. 2.3, Eqs. (vf-f), (vf-td)): the small dense linear
// algebra of the method (J <= a few hundred samples, K <= ~10 responses, M <= ~150 poles) is
// latency-bound, so it runs in native C++ next to the GPU solver that produces its samples.
//
// Model: f_k(s) = sum_m r_{k,m} / (s - a_m), common poles, no constant/linear term.
// Pole identification (repeated): with current poles abar, least squares for
//   sum_m c_{k,m} phi_m(s_j) - f_k(s_j) sum_m ct_m phi_m(s_j) = f_k(s_j)
// in the real-coefficient basis phi (pair a: 1/(s-a) + 1/(s-conj a), i/(s-a) - i/(s-conj a);
// real a: 1/(s-a)), real and imaginary parts stacked.  The c_k are eliminated response by
// response: a Householder QR of each block [Phi | -diag(f_k) Phi] leaves, in its last M rows,
// the equations that involve ct alone; these are stacked over k and solved for ct (the
// "fast" arrangement of the same least-squares problem).  The new poles are the eigenvalues of
// A - b ct^T (real realisation of sigma(s) = 1 + ct^T (sI - A)^{-1} b; pair block
// [[Re a, Im a], [-Im a, Re a]] with b = (2, 0)), computed by Hessenberg reduction and
// Francis double-shift QR.  Unstable poles are kept.
// Residue identification: one QR of Phi, all responses as right-hand sides.
// The per-response eliminations are independent and run on host threads (each response's
// arithmetic is unchanged, so the result does not depend on the thread count).
#include <algorithm>
#include <cmath>
#include <complex>
#include <exception>
#include <stdexcept>
#include <thread>
#include <vector>

#include "vf_host.h"

namespace bem {
namespace vfit {

namespace {

// Worker threads for the per-response eliminations: half the host's hardware threads (the two
// fits of an AFS step run side by side), at least one.
int host_threads() {
  const unsigned h = std::thread::hardware_concurrency();
  return std::max(1, (int)(h / 2));
}

// Column-major dense helpers ------------------------------------------------------------------
struct Mat {
  int m = 0, n = 0;
  std::vector<double> a;  // column-major
  Mat() = default;
  Mat(int m_, int n_) : m(m_), n(n_), a((size_t)m_ * n_, 0.0) {}
  double& operator()(int i, int j) { return a[(size_t)j * m + i]; }
  double operator()(int i, int j) const { return a[(size_t)j * m + i]; }
};

// Householder QR of A (m x n, m >= n) applied to B (m x r): on return the upper triangle of A
// holds R and B holds Q^T B.
void householder_qr(Mat& A, Mat& B) {
  const int m = A.m, n = A.n;
  std::vector<double> v(m);
  for (int k = 0; k < n && k < m; ++k) {
    double nrm = 0;
    for (int i = k; i < m; ++i) nrm += A(i, k) * A(i, k);
    nrm = std::sqrt(nrm);
    if (nrm == 0.0) continue;
    const double alpha = A(k, k) > 0 ? -nrm : nrm;
    double vv = 0;
    for (int i = k; i < m; ++i) {
      v[i] = A(i, k) - (i == k ? alpha : 0.0);
      vv += v[i] * v[i];
    }
    if (vv == 0.0) continue;
    const double beta = 2.0 / vv;
    for (int j = k; j < n; ++j) {
      double d = 0;
      for (int i = k; i < m; ++i) d += v[i] * A(i, j);
      d *= beta;
      for (int i = k; i < m; ++i) A(i, j) -= d * v[i];
    }
    for (int j = 0; j < B.n; ++j) {
      double d = 0;
      for (int i = k; i < m; ++i) d += v[i] * B(i, j);
      d *= beta;
      for (int i = k; i < m; ++i) B(i, j) -= d * v[i];
    }
    A(k, k) = alpha;
    for (int i = k + 1; i < m; ++i) A(i, k) = 0.0;
  }
}

// Least squares min ||A x - B|| (columns scaled to unit norm first); returns X (n x r).
Mat lstsq(Mat A, Mat B) {
  const int n = A.n;
  std::vector<double> sc(n, 1.0);
  for (int j = 0; j < n; ++j) {
    double s = 0;
    for (int i = 0; i < A.m; ++i) s += A(i, j) * A(i, j);
    s = std::sqrt(s);
    sc[j] = s > 0 ? s : 1.0;
    for (int i = 0; i < A.m; ++i) A(i, j) /= sc[j];
  }
  householder_qr(A, B);
  Mat X(n, B.n);
  for (int c = 0; c < B.n; ++c)
    for (int i = n - 1; i >= 0; --i) {
      double acc = B(i, c);
      for (int j = i + 1; j < n; ++j) acc -= A(i, j) * X(j, c);
      const double d = A(i, i);
      X(i, c) = (std::fabs(d) > 1e-300) ? acc / d : 0.0;
    }
  for (int j = 0; j < n; ++j)
    for (int c = 0; c < B.n; ++c) X(j, c) /= sc[j];
  return X;
}

// Eigenvalues of a real n x n matrix: Householder reduction to upper Hessenberg form, then
// Francis double-shift QR steps with deflation on small subdiagonals.
std::vector<cd> eig_real(Mat H) {
  const int n = H.n;
  std::vector<cd> ev;
  ev.reserve(n);
  // Hessenberg reduction
  std::vector<double> v(n);
  for (int k = 0; k + 2 < n; ++k) {
    double nrm = 0;
    for (int i = k + 1; i < n; ++i) nrm += H(i, k) * H(i, k);
    nrm = std::sqrt(nrm);
    if (nrm == 0) continue;
    const double alpha = H(k + 1, k) > 0 ? -nrm : nrm;
    double vv = 0;
    for (int i = k + 1; i < n; ++i) {
      v[i] = H(i, k) - (i == k + 1 ? alpha : 0.0);
      vv += v[i] * v[i];
    }
    if (vv == 0) continue;
    const double beta = 2.0 / vv;
    for (int j = 0; j < n; ++j) {  // rows: H = P H
      double d = 0;
      for (int i = k + 1; i < n; ++i) d += v[i] * H(i, j);
      d *= beta;
      for (int i = k + 1; i < n; ++i) H(i, j) -= d * v[i];
    }
    for (int i = 0; i < n; ++i) {  // columns: H = H P
      double d = 0;
      for (int j = k + 1; j < n; ++j) d += H(i, j) * v[j];
      d *= beta;
      for (int j = k + 1; j < n; ++j) H(i, j) -= d * v[j];
    }
    for (int i = k + 2; i < n; ++i) H(i, k) = 0.0;
  }
  const double eps = 2.220446049250313e-16;
  int hi = n - 1, iter = 0, total = 0;
  while (hi >= 0) {
    int l = hi;
    while (l > 0) {
      const double s = std::fabs(H(l - 1, l - 1)) + std::fabs(H(l, l));
      if (std::fabs(H(l, l - 1)) <= eps * (s > 0 ? s : 1.0)) {
        H(l, l - 1) = 0.0;
        break;
      }
      --l;
    }
    if (l == hi) {
      ev.emplace_back(H(hi, hi), 0.0);
      --hi;
      iter = 0;
      continue;
    }
    if (l == hi - 1) {
      const double a = H(hi - 1, hi - 1), b = H(hi - 1, hi), c = H(hi, hi - 1), d = H(hi, hi);
      const double tr = a + d, det = a * d - b * c, disc = 0.25 * tr * tr - det;
      if (disc >= 0) {
        const double r = std::sqrt(disc);
        const double l1 = 0.5 * tr + (tr >= 0 ? r : -r);
        const double l2 = (l1 != 0.0) ? det / l1 : 0.5 * tr - (tr >= 0 ? r : -r);
        ev.emplace_back(l1, 0.0);
        ev.emplace_back(l2, 0.0);
      } else {
        const double im = std::sqrt(-disc);
        ev.emplace_back(0.5 * tr, im);
        ev.emplace_back(0.5 * tr, -im);
      }
      hi -= 2;
      iter = 0;
      continue;
    }
    if (++total > 200 * n) throw std::runtime_error("eigenvalue iteration did not converge");
    ++iter;
    double s, t;
    if (iter % 10 == 0) {  // exceptional shift
      const double w = std::fabs(H(hi, hi - 1)) + std::fabs(H(hi - 1, hi - 2));
      s = 1.5 * w;
      t = w * w;
    } else {
      s = H(hi - 1, hi - 1) + H(hi, hi);
      t = H(hi - 1, hi - 1) * H(hi, hi) - H(hi - 1, hi) * H(hi, hi - 1);
    }
    double x = H(l, l) * H(l, l) + H(l, l + 1) * H(l + 1, l) - s * H(l, l) + t;
    double y = H(l + 1, l) * (H(l, l) + H(l + 1, l + 1) - s);
    double z = H(l + 1, l) * H(l + 2, l + 1);
    for (int k = l; k <= hi - 1; ++k) {
      const int nr = (k < hi - 1) ? 3 : 2;  // reflector size
      double u[3] = {x, y, nr == 3 ? z : 0.0};
      const double nrm = std::sqrt(u[0] * u[0] + u[1] * u[1] + u[2] * u[2]);
      if (nrm != 0.0) {
        const double alpha = u[0] > 0 ? -nrm : nrm;
        u[0] -= alpha;
        const double uu = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
        const double beta = 2.0 / uu;
        const int c0 = std::max(l, k - 1);
        for (int j = c0; j <= hi; ++j) {  // rows k..k+nr-1
          double d = 0;
          for (int q = 0; q < nr; ++q) d += u[q] * H(k + q, j);
          d *= beta;
          for (int q = 0; q < nr; ++q) H(k + q, j) -= d * u[q];
        }
        const int r1 = std::min(hi, k + 3);
        for (int i = l; i <= r1; ++i) {  // columns k..k+nr-1
          double d = 0;
          for (int q = 0; q < nr; ++q) d += H(i, k + q) * u[q];
          d *= beta;
          for (int q = 0; q < nr; ++q) H(i, k + q) -= d * u[q];
        }
      }
      if (k < hi - 1) {
        x = H(k + 1, k);
        y = H(k + 2, k);
        if (k < hi - 2) z = H(k + 3, k);
      }
    }
  }
  return ev;
}

void basis_row(cd s, const Poles& P, std::vector<cd>& row) {
  row.clear();
  for (const cd& a : P.pairs) {
    const cd u = 1.0 / (s - a), w = 1.0 / (s - std::conj(a));
    row.push_back(u + w);
    row.push_back(cd(0, 1) * u - cd(0, 1) * w);
  }
  for (double a : P.reals) row.push_back(1.0 / (s - a));
}

}  // namespace

Poles initial_poles(int M, double omega_max) {
  Poles P;
  const int np = M / 2;
  for (int m = 1; m <= np; ++m) {
    const double b = omega_max * m / std::max(np, 1);
    P.pairs.emplace_back(-b / 100.0, b);
  }
  if (M % 2) P.reals.push_back(-omega_max / 100.0);
  return P;
}

Poles split_poles(const std::vector<cd>& z) {
  double scale = 1.0;
  for (const cd& v : z) scale = std::max(scale, std::abs(v));
  Poles P;
  for (const cd& v : z) {
    if (std::fabs(v.imag()) <= 1e-12 * scale) P.reals.push_back(v.real());
    else if (v.imag() > 0) P.pairs.push_back(v);
  }
  std::sort(P.reals.begin(), P.reals.end());
  std::sort(P.pairs.begin(), P.pairs.end(), [](const cd& a, const cd& b) { return a.imag() < b.imag(); });
  return P;
}

Poles relocate(const std::vector<cd>& s, const std::vector<cd>& F, int K, const std::vector<int>& cols,
               const Poles& P) {
  const int J = (int)s.size();
  const int M = 2 * (int)P.pairs.size() + (int)P.reals.size();
  const int Kc = (int)cols.size();
  // basis and common column scaling
  std::vector<std::vector<cd>> Phi(J);
  for (int j = 0; j < J; ++j) basis_row(s[j], P, Phi[j]);
  std::vector<double> sc(M, 0.0);
  for (int j = 0; j < J; ++j)
    for (int m = 0; m < M; ++m) sc[m] += std::norm(Phi[j][m]);
  for (int m = 0; m < M; ++m) sc[m] = sc[m] > 0 ? std::sqrt(2.0 * sc[m]) : 1.0;
  Mat Rs(Kc * M, M), Ys(Kc * M, 1);
  auto eliminate = [&](int kk) {
    const int k = cols[kk];
    Mat A(2 * J, 2 * M), B(2 * J, 1);
    for (int j = 0; j < J; ++j) {
      const cd f = F[(size_t)j * K + k];
      for (int m = 0; m < M; ++m) {
        const cd p = Phi[j][m] / sc[m];
        const cd q = -f * p;
        A(j, m) = p.real();
        A(J + j, m) = p.imag();
        A(j, M + m) = q.real();
        A(J + j, M + m) = q.imag();
      }
      B(j, 0) = f.real();
      B(J + j, 0) = f.imag();
    }
    householder_qr(A, B);
    for (int r = 0; r < M; ++r) {
      for (int c = 0; c < M; ++c) Rs(kk * M + r, c) = (M + r <= M + c) ? A(M + r, M + c) : 0.0;
      Ys(kk * M + r, 0) = B(M + r, 0);
    }
  };
  // responses on host threads once the eliminations are large enough to pay for a thread
  const int nt = ((double)J * M * M < 2e5) ? 1 : std::min(Kc, host_threads());
  if (nt <= 1) {
    for (int kk = 0; kk < Kc; ++kk) eliminate(kk);
  } else {
    // a worker's exception (e.g. an allocation failure) is carried back and rethrown here
    std::vector<std::exception_ptr> err(nt);
    std::vector<std::thread> pool;
    for (int w = 0; w < nt; ++w)
      pool.emplace_back([&, w] {
        try {
          for (int kk = w; kk < Kc; kk += nt) eliminate(kk);
        } catch (...) {
          err[w] = std::current_exception();
        }
      });
    for (auto& th : pool) th.join();
    for (auto& e : err)
      if (e) std::rethrow_exception(e);
  }
  Mat ct = lstsq(Rs, Ys);
  Mat H(M, M);
  std::vector<double> b(M, 0.0);
  int c = 0;
  for (const cd& a : P.pairs) {
    H(c, c) = a.real();
    H(c, c + 1) = a.imag();
    H(c + 1, c) = -a.imag();
    H(c + 1, c + 1) = a.real();
    b[c] = 2.0;
    c += 2;
  }
  for (double a : P.reals) {
    H(c, c) = a;
    b[c] = 1.0;
    ++c;
  }
  for (int i = 0; i < M; ++i)
    for (int j = 0; j < M; ++j) H(i, j) -= b[i] * ct(j, 0) / sc[j];
  return split_poles(eig_real(H));
}

Model residues(const std::vector<cd>& s, const std::vector<cd>& F, int K, const Poles& P) {
  const int J = (int)s.size();
  const int M = 2 * (int)P.pairs.size() + (int)P.reals.size();
  Mat A(2 * J, M), B(2 * J, K);
  std::vector<cd> row;
  for (int j = 0; j < J; ++j) {
    basis_row(s[j], P, row);
    for (int m = 0; m < M; ++m) {
      A(j, m) = row[m].real();
      A(J + j, m) = row[m].imag();
    }
    for (int k = 0; k < K; ++k) {
      B(j, k) = F[(size_t)j * K + k].real();
      B(J + j, k) = F[(size_t)j * K + k].imag();
    }
  }
  const Mat X = lstsq(A, B);
  Model out;
  out.K = K;
  for (const cd& a : P.pairs) {
    out.poles.push_back(a);
    out.poles.push_back(std::conj(a));
  }
  for (double a : P.reals) out.poles.emplace_back(a, 0.0);
  out.R.assign((size_t)K * M, cd(0, 0));
  for (int k = 0; k < K; ++k) {
    int c = 0;
    for (size_t p = 0; p < P.pairs.size(); ++p) {
      const cd r(X(c, k), X(c + 1, k));
      out.R[(size_t)k * M + 2 * p] = r;
      out.R[(size_t)k * M + 2 * p + 1] = std::conj(r);
      c += 2;
    }
    for (size_t q = 0; q < P.reals.size(); ++q, ++c) out.R[(size_t)k * M + 2 * P.pairs.size() + q] = cd(X(c, k), 0.0);
  }
  return out;
}

// A relocated pole closer than 1e-6 Omega to a sample s_j moves to s_j - 1e-6 Omega (same
// imaginary part, left of the sampling line).  The samples lie right of the physical poles
// (Re s = eta > 0) and unstable poles are kept, so with noisy data a surplus pole can settle on
// a sample, where the next step's basis 1/(s - a) is infinite; the paper is silent on this case.
static void keep_off_samples(const std::vector<cd>& s, Poles& P, double omega_max) {
  const double gap = 1e-6 * omega_max;
  auto nearest = [&](cd a) {
    size_t jb = 0;
    for (size_t j = 1; j < s.size(); ++j)
      if (std::abs(s[j] - a) < std::abs(s[jb] - a)) jb = j;
    return s[jb];
  };
  for (cd& a : P.pairs) {
    const cd sj = nearest(a);
    if (std::abs(sj - a) < gap) a = sj - gap;
  }
  for (double& a : P.reals) {
    const cd sj = nearest(cd(a, 0.0));
    if (std::abs(sj - cd(a, 0.0)) < gap) a = sj.real() - gap;
  }
}

Poles fit_poles(const std::vector<cd>& s, const std::vector<cd>& F, int K, const std::vector<int>& cols,
                int M, double omega_max, int n_iter, double tol) {
  Poles P = initial_poles(M, omega_max);
  for (int it = 0; it < n_iter; ++it) {
    Poles Q = relocate(s, F, K, cols, P);
    keep_off_samples(s, Q, omega_max);
    double change = 0.0;
    const bool same = Q.pairs.size() == P.pairs.size() && Q.reals.size() == P.reals.size();
    if (same) {
      for (size_t i = 0; i < Q.pairs.size(); ++i) change = std::max(change, std::abs(Q.pairs[i] - P.pairs[i]));
      for (size_t i = 0; i < Q.reals.size(); ++i) change = std::max(change, std::fabs(Q.reals[i] - P.reals[i]));
    }
    P = Q;
    if (same && change <= tol * omega_max) break;
  }
  return P;
}

void evaluate(const Model& md, const std::vector<cd>& s, std::vector<cd>& out) {
  const int M = (int)md.poles.size();
  out.assign(s.size() * md.K, cd(0, 0));
  std::vector<cd> w(M);
  for (size_t j = 0; j < s.size(); ++j) {
    for (int m = 0; m < M; ++m) w[m] = 1.0 / (s[j] - md.poles[m]);
    for (int k = 0; k < md.K; ++k) {
      cd acc(0, 0);
      for (int m = 0; m < M; ++m) acc += md.R[(size_t)k * M + m] * w[m];
      out[j * md.K + k] = acc;
    }
  }
}

void time_response(const Model& md, const std::vector<double>& t, std::vector<double>& out, double eta) {
  const int M = (int)md.poles.size();
  out.assign(t.size() * md.K, 0.0);
  std::vector<cd> e(M);
  for (size_t j = 0; j < t.size(); ++j) {
    for (int m = 0; m < M; ++m) e[m] = (md.poles[m].real() < eta) ? std::exp(md.poles[m] * t[j]) : cd(0, 0);
    for (int k = 0; k < md.K; ++k) {
      cd acc(0, 0);
      for (int m = 0; m < M; ++m) acc += md.R[(size_t)k * M + m] * e[m];
      out[j * md.K + k] = acc.real();
    }
  }
}

}  // namespace vfit
}  // namespace bem
