// Host-side FP64 tables of the plan (filters, deapodisation, twiddles).
#pragma once

#include <vector>

namespace pdgb {

// Low-pass filter of db_p, largest tap first, sum sqrt(2).
std::vector<double> daubechies(int p);
// pi sqrt((J/2)^2 (3/2)^2 - 0.8): Kaiser-Bessel shape for 2x oversampling.
double kb_beta_default(int J);
// c[i] = 1 / phi_hat((i - n/2) / K) for a J-wide Kaiser-Bessel kernel.
std::vector<double> deapodisation(int n, int K, int J, double beta);
// interleaved (cos, -sin)(2 pi k / K), k in [0, K)
std::vector<double> twiddles(int K);
// Monomial coefficients (in x = 2 f - 1, f in [0, 1)) of the degree-`deg` Chebyshev
// interpolant of tap a's weight phi(f + J/2 - 1 - a), for a = 0..J-1: [J][deg + 1].
std::vector<double> kb_tap_polynomials(int J, double beta, int deg);

}  // namespace pdgb
