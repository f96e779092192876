// Host-side vector fitting and adaptive frequency sampling (vf.cpp, afs.cpp).
#pragma once

#include <complex>
#include <vector>

namespace bem {
namespace vfit {

using cd = std::complex<double>;

// Poles of a real model: complex pairs by their member with Im > 0, and real poles.
struct Poles {
  std::vector<cd> pairs;
  std::vector<double> reals;
};

// f_k(s) = sum_m R[k][m] / (s - poles[m]) with pairs expanded (a, conj a adjacent).
struct Model {
  std::vector<cd> poles;  // M
  std::vector<cd> R;      // K x M row-major
  int K = 0;
};

Poles initial_poles(int M, double omega_max);
Poles split_poles(const std::vector<cd>& z);
// one pole relocation from the responses F (J x K row-major) restricted to the columns `cols`
Poles relocate(const std::vector<cd>& s, const std::vector<cd>& F, int K, const std::vector<int>& cols,
               const Poles& P);
Poles fit_poles(const std::vector<cd>& s, const std::vector<cd>& F, int K, const std::vector<int>& cols,
                int M, double omega_max, int n_iter, double tol);
Model residues(const std::vector<cd>& s, const std::vector<cd>& F, int K, const Poles& P);
void evaluate(const Model& md, const std::vector<cd>& s, std::vector<cd>& out);            // J x K
// nt x K; only poles with Re a < eta contribute (the Bromwich contour Re s = eta of the samples)
void time_response(const Model& md, const std::vector<double>& t, std::vector<double>& out, double eta);

}  // namespace vfit
}  // namespace bem
