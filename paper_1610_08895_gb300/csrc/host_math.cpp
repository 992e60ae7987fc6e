// Host-side tables of the plan: Daubechies filters, Kaiser-Bessel deapodisation
// and FFT twiddles, all computed in FP64.
#include "host_math.hpp"

#include <cmath>
#include <complex>
#include <vector>

namespace pdgb {

using cd = std::complex<double>;

// Roots of a polynomial with real coefficients a[0] x^n + ... + a[n] by the
// Weierstrass (Durand-Kerner) simultaneous iteration, polished by Newton steps.
static std::vector<cd> poly_roots(const std::vector<double>& a) {
    const int n = (int)a.size() - 1;
    std::vector<cd> z(n);
    if (n <= 0) return z;
    std::vector<double> m(a.size());
    for (size_t i = 0; i < a.size(); ++i) m[i] = a[i] / a[0];
    auto eval = [&](cd x) {
        cd v = 1.0;
        for (int i = 1; i <= n; ++i) v = v * x + m[i];
        return v;
    };
    auto deriv = [&](cd x) {
        cd v = (double)n;
        for (int i = 1; i < n; ++i) v = v * x + (double)(n - i) * m[i];
        return v;
    };
    const cd seed(0.4, 0.9);
    cd w = 1.0;
    for (int i = 0; i < n; ++i) { z[i] = w; w *= seed; }
    for (int it = 0; it < 2000; ++it) {
        double change = 0.0;
        for (int i = 0; i < n; ++i) {
            cd den = 1.0;
            for (int j = 0; j < n; ++j)
                if (j != i) den *= (z[i] - z[j]);
            const cd step = eval(z[i]) / den;
            z[i] -= step;
            change = std::max(change, std::abs(step));
        }
        if (change < 1e-15) break;
    }
    for (int i = 0; i < n; ++i)
        for (int k = 0; k < 3; ++k) {
            const cd d = deriv(z[i]);
            if (std::abs(d) > 0) z[i] -= eval(z[i]) / d;
        }
    return z;
}

static double binom(int n, int k) {
    double r = 1.0;
    for (int i = 1; i <= k; ++i) r = r * (n - k + i) / i;
    return r;
}

// db_p low-pass filter: minimum-phase spectral factor of the maximally flat
// half-band polynomial P(y) = sum_{k<p} C(p-1+k, k) y^k (Daubechies 1988).
std::vector<double> daubechies(int p) {
    std::vector<cd> zeros;
    for (int i = 0; i < p; ++i) zeros.push_back(cd(-1.0, 0.0));
    if (p > 1) {
        std::vector<double> coef(p);   // decreasing powers of y
        for (int k = 0; k < p; ++k) coef[p - 1 - k] = binom(p - 1 + k, k);
        for (const cd& y : poly_roots(coef)) {
            // y = (2 - z - 1/z)/4  <=>  z^2 - (2 - 4y) z + 1 = 0; keep the root inside the unit circle
            const cd c = 1.0 - 2.0 * y;
            const cd s = std::sqrt(c * c - 1.0);
            const cd z1 = c + s, z2 = c - s;
            zeros.push_back(std::abs(z1) < 1.0 ? z1 : z2);
        }
    }
    // expand prod (z - zero) in decreasing powers
    std::vector<cd> poly(1, cd(1.0, 0.0));
    for (const cd& r : zeros) {
        std::vector<cd> nxt(poly.size() + 1, cd(0.0, 0.0));
        for (size_t i = 0; i < poly.size(); ++i) {
            nxt[i] += poly[i];
            nxt[i + 1] -= r * poly[i];
        }
        poly.swap(nxt);
    }
    std::vector<double> h(poly.size());
    double sum = 0.0;
    for (size_t i = 0; i < poly.size(); ++i) { h[i] = poly[i].real(); sum += h[i]; }
    for (double& v : h) v *= std::sqrt(2.0) / sum;
    return h;
}

double kb_beta_default(int J) {
    const double a = 2.0;
    return M_PI * std::sqrt((J / a) * (J / a) * (a - 0.5) * (a - 0.5) - 0.8);
}

// Fourier transform of the Kaiser-Bessel window of width J (cycles per cell).
static double kb_hat(double xi, int J, double beta) {
    const double z2 = beta * beta - (M_PI * J * xi) * (M_PI * J * xi);
    if (z2 > 0) { const double z = std::sqrt(z2); return J * std::sinh(z) / z; }
    if (z2 < 0) { const double z = std::sqrt(-z2); return J * std::sin(z) / z; }
    return J;
}

std::vector<double> deapodisation(int n, int K, int J, double beta) {
    std::vector<double> c(n);
    for (int i = 0; i < n; ++i) c[i] = 1.0 / kb_hat((i - n / 2) / (double)K, J, beta);
    return c;
}

std::vector<double> twiddles(int K) {
    std::vector<double> t(2 * K);
    for (int k = 0; k < K; ++k) {
        const double a = 2.0 * M_PI * (double)k / (double)K;
        t[2 * k] = std::cos(a);
        t[2 * k + 1] = -std::sin(a);
    }
    return t;
}

// Kaiser-Bessel weight I0(beta sqrt(1 - (2t/J)^2)), |t| <= J/2.
static double kb_phi(double t, int J, double beta) {
    const double u = 2.0 * t / J;
    const double arg = 1.0 - u * u;
    return arg >= 0 ? std::cyl_bessel_i(0.0, beta * std::sqrt(arg)) : 0.0;
}

// Chebyshev interpolation at the deg + 1 Chebyshev points of the first kind,
// then conversion of sum_j c_j T_j(x) to monomials with T_{j+1} = 2 x T_j - T_{j-1}.
std::vector<double> kb_tap_polynomials(int J, double beta, int deg) {
    const int n = deg + 1;
    std::vector<double> out((size_t)J * n, 0.0);
    for (int a = 0; a < J; ++a) {
        std::vector<double> fx(n), cheb(n, 0.0);
        for (int k = 0; k < n; ++k) {
            const double xk = std::cos(M_PI * (k + 0.5) / n);
            fx[k] = kb_phi((xk + 1.0) / 2.0 + J / 2 - 1 - a, J, beta);
        }
        for (int j = 0; j < n; ++j) {
            double acc = 0.0;
            for (int k = 0; k < n; ++k) acc += fx[k] * std::cos(M_PI * j * (k + 0.5) / n);
            cheb[j] = (j == 0 ? 1.0 : 2.0) * acc / n;
        }
        std::vector<double> tm1(n, 0.0), t0(n, 0.0), mono(n, 0.0);
        t0[0] = 1.0;                                   // T_0
        for (int j = 0; j < n; ++j) {
            for (int i = 0; i < n; ++i) mono[i] += cheb[j] * t0[i];
            std::vector<double> t1(n, 0.0);            // T_{j+1} = 2 x T_j - T_{j-1}
            for (int i = 0; i + 1 < n; ++i) t1[i + 1] += 2.0 * t0[i];
            if (j == 0) { t1.assign(n, 0.0); if (n > 1) t1[1] = 1.0; }
            else for (int i = 0; i < n; ++i) t1[i] -= tm1[i];
            tm1 = t0;
            t0 = t1;
        }
        for (int i = 0; i < n; ++i) out[(size_t)a * n + i] = mono[i];
    }
    return out;
}

}  // namespace pdgb
