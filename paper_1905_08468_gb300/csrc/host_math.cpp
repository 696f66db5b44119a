// Host-side FP64 tables of the MUFFIN library: Daubechies scaling filters
// (Sec. 4.2.1: the union of the first 8 Daubechies bases) and the
// orthonormal DCT-II (W_lambda).  Written from the mathematics:
//
// Daubechies' spectral factorisation.  The extremal-phase scaling filter of
// db<p> has p zeros at z = -1 and one zero inside the unit circle for every
// root y_j of P(y) = sum_{k<p} C(p-1+k, k) y^k, namely the root of
// z^2 - (2 - 4 y_j) z + 1 = 0 with |z| < 1.  The roots of P are found with
// the Weierstrass (Durand-Kerner) simultaneous iteration polished by Newton
// steps; h is the coefficient list of (z+1)^p prod_j (z - z_j) in descending
// powers, scaled to sum sqrt(2).
#include <cmath>
#include <complex>
#include <vector>

#include "host_math.h"

namespace muffin {

using cd = std::complex<double>;

static cd poly_eval(const std::vector<double> &c_desc, cd z) {
  cd r = 0.0;
  for (double c : c_desc) r = r * z + c;
  return r;
}

static cd poly_deriv(const std::vector<double> &c_desc, cd z) {
  cd r = 0.0;
  const size_t d = c_desc.size() - 1;
  for (size_t i = 0; i < d; ++i) r = r * z + c_desc[i] * double(d - i);
  return r;
}

// roots of a real polynomial given in descending powers
static std::vector<cd> poly_roots(const std::vector<double> &c_desc) {
  const size_t d = c_desc.size() - 1;
  std::vector<cd> r(d);
  if (d == 0) return r;
  std::vector<double> m(c_desc);
  for (double &v : m) v /= c_desc[0];
  const cd seed(0.4, 0.9);
  cd s = 1.0;
  for (size_t i = 0; i < d; ++i) { r[i] = s; s *= seed; }
  for (int it = 0; it < 5000; ++it) {
    double delta = 0.0;
    for (size_t i = 0; i < d; ++i) {
      cd den = 1.0;
      for (size_t j = 0; j < d; ++j)
        if (j != i) den *= (r[i] - r[j]);
      const cd step = poly_eval(m, r[i]) / den;
      r[i] -= step;
      delta = std::fmax(delta, std::abs(step));
    }
    if (delta < 1e-15) break;
  }
  for (size_t i = 0; i < d; ++i)
    for (int k = 0; k < 3; ++k) {
      const cd dv = poly_deriv(m, r[i]);
      if (std::abs(dv) > 0) r[i] -= poly_eval(m, r[i]) / dv;
    }
  return r;
}

void daubechies_lowpass(int p, double *h) {
  std::vector<cd> zeros(p, cd(-1.0, 0.0));
  if (p > 1) {
    std::vector<double> P_desc(p);
    for (int k = 0; k < p; ++k) {
      // C(p-1+k, k)
      double c = 1.0;
      for (int i = 1; i <= k; ++i) c = c * double(p - 1 + i) / double(i);
      P_desc[p - 1 - k] = c;
    }
    for (const cd &y : poly_roots(P_desc)) {
      const cd b = 2.0 - 4.0 * y;
      const cd disc = std::sqrt(b * b - 4.0);
      const cd z1 = (b + disc) / 2.0, z2 = (b - disc) / 2.0;
      zeros.push_back(std::abs(z1) < 1.0 ? z1 : z2);
    }
  }
  std::vector<cd> poly(1, cd(1.0, 0.0));   // descending coefficients
  for (const cd &z : zeros) {
    std::vector<cd> nx(poly.size() + 1, cd(0.0, 0.0));
    for (size_t i = 0; i < poly.size(); ++i) {
      nx[i] += poly[i];
      nx[i + 1] -= z * poly[i];
    }
    poly.swap(nx);
  }
  double sum = 0.0;
  for (int i = 0; i < 2 * p; ++i) sum += poly[i].real();
  const double sc = std::sqrt(2.0) / sum;
  for (int i = 0; i < 2 * p; ++i) h[i] = poly[i].real() * sc;
}

void dct2_matrix(int L, double *C) {
  const double pi = 3.14159265358979323846;
  for (int k = 0; k < L; ++k) {
    const double ck = k == 0 ? std::sqrt(1.0 / L) : std::sqrt(2.0 / L);
    for (int l = 0; l < L; ++l)
      C[(size_t)k * L + l] = ck * std::cos(pi * (2.0 * l + 1.0) * k / (2.0 * L));
  }
}

double iuwt_norm2(int n, int J) {
  const double pi = 3.14159265358979323846;
  // 1D transfer function of the B3 spline at dilation d: (1 + cos w d)^2 / 4
  std::vector<std::vector<double>> h(J, std::vector<double>(n));
  for (int j = 0; j < J; ++j)
    for (int k = 0; k < n; ++k) {
      const double c = std::cos(2.0 * pi * (double)(k << j) / n);
      h[j][k] = (1.0 + c) * (1.0 + c) / 4.0;
    }
  double best = 0.0;
  for (int ky = 0; ky < n; ++ky)
    for (int kx = 0; kx < n; ++kx) {
      double a = 1.0, s = 0.0;
      for (int j = 0; j < J; ++j) {
        const double an = a * h[j][ky] * h[j][kx];
        s += (a - an) * (a - an);
        a = an;
      }
      s += a * a;
      if (s > best) best = s;
    }
  return best;
}

}  // namespace muffin
