// Tensorised Gauss-Legendre x uniform-azimuth quadrature on the upper
// hemisphere (Sec. 4.1 normalisation, product rule named in Sec. 5.1.1).
//
// Gauss-Legendre nodes: roots of P_n on [-1, 1] by Newton's method with the
// three-term recurrence (k+1) P_{k+1} = (2k+1) x P_k - k P_{k-1} and
// P_n'(x) = n (x P_n - P_{n-1}) / (x^2 - 1); weights 2 / ((1 - x^2) P_n'(x)^2).
// Initial guesses cos(pi (i + 3/4) / (n + 1/2)) (Tricomi's asymptotic form).
#include <cmath>

#include "host_common.h"

namespace rtk {

// P_n(z) and P_{n-1}(z) by the three-term recurrence (n >= 1).
static void legendre_pair(int n, double z, double* pn, double* pm) {
  double a = 1.0, b = z;   // P_0, P_1
  for (int k = 1; k < n; ++k) {
    const double c = ((2.0 * k + 1.0) * z * b - k * a) / (k + 1.0);
    a = b;
    b = c;
  }
  *pn = b;
  *pm = a;
}

static void gauss_legendre(int n, double* x, double* w) {
  for (int i = 0; i < n; ++i) {
    double z = std::cos(M_PI * (i + 0.75) / (n + 0.5));
    double pn, pm, dp;
    for (int it = 0; it < 100; ++it) {
      legendre_pair(n, z, &pn, &pm);
      dp = n * (z * pn - pm) / (z * z - 1.0);
      const double dz = pn / dp;
      z -= dz;
      if (std::fabs(dz) < 1e-16) break;
    }
    legendre_pair(n, z, &pn, &pm);
    dp = n * (z * pn - pm) / (z * z - 1.0);
    // store ascending: the guesses run from the largest root down
    x[n - 1 - i] = z;
    w[n - 1 - i] = 2.0 / ((1.0 - z * z) * dp * dp);
  }
}

}  // namespace rtk

extern "C" rt_status rt_quad_product(int32_t n_p, int32_t n_phi, double* xi, double* eta, double* mu, double* w) {
  rtk::clear_error();
  if (n_p < 1 || n_p > 64 || n_phi < 1 || n_phi > 4096 || !xi || !eta || !w) {
    rtk::set_error("rt_quad_product: need 1 <= n_p <= 64, 1 <= n_phi <= 4096 and output arrays");
    return RT_EINVAL;
  }
  double gx[64], gw[64];
  if (n_p == 1) {
    gx[0] = 0.0;
    gw[0] = 2.0;
  } else {
    rtk::gauss_legendre(n_p, gx, gw);
  }
  for (int a = 0; a < n_phi; ++a) {
    const double ph = (a + 0.5) * (2.0 * M_PI / n_phi);
    const double c = std::cos(ph), s = std::sin(ph);
    for (int p = 0; p < n_p; ++p) {
      const int k = a * n_p + p;
      const double m = 0.5 * (gx[p] + 1.0);   // map [-1,1] -> [0,1]
      const double r = std::sqrt(1.0 - m * m);
      xi[k] = r * c;
      eta[k] = r * s;
      if (mu) mu[k] = m;
      w[k] = 0.5 * gw[p] * (2.0 * M_PI / n_phi);
    }
  }
  return RT_OK;
}

namespace {

struct Vec3 {
  double x, y, z;
};
Vec3 add(Vec3 a, Vec3 b) { return {a.x + b.x, a.y + b.y, a.z + b.z}; }
Vec3 scale(Vec3 a, double s) { return {a.x * s, a.y * s, a.z * s}; }
double dot(Vec3 a, Vec3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
Vec3 unit(Vec3 a) { return scale(a, 1.0 / std::sqrt(dot(a, a))); }

// Area of the spherical triangle with unit corners a, b, c: twice the angle of
// the complex number (1 + a.b + b.c + c.a) + i |a.(b x c)|.
double excess(Vec3 a, Vec3 b, Vec3 c) {
  const Vec3 bc = {b.y * c.z - b.z * c.y, b.z * c.x - b.x * c.z, b.x * c.y - b.y * c.x};
  const double num = std::fabs(dot(a, bc));
  const double den = 1.0 + dot(a, b) + dot(b, c) + dot(c, a);
  return 2.0 * std::atan2(num, den);
}

}  // namespace

extern "C" rt_status rt_quad_tessellation(int32_t N, double* xi, double* eta, double* mu, double* w) {
  rtk::clear_error();
  if (N < 1 || N > 128 || !xi || !eta || !w) {
    rtk::set_error("rt_quad_tessellation: need 1 <= N <= 128 and output arrays");
    return RT_EINVAL;
  }
  // upper faces of the octahedron, one per azimuth quadrant: corners A, B, pole
  const Vec3 corner[5] = {{1, 0, 0}, {0, 1, 0}, {-1, 0, 0}, {0, -1, 0}, {1, 0, 0}};
  const Vec3 pole = {0, 0, 1};
  int k = 0;
  for (int f = 0; f < 4; ++f) {
    const Vec3 A = corner[f], B = corner[f + 1];
    auto P = [&](int i, int j) {   // A + (B - A) i/N + (pole - A) j/N
      const double u = (double)i / N, v = (double)j / N;
      return add(add(scale(A, 1.0 - u - v), scale(B, u)), scale(pole, v));
    };
    auto emit = [&](Vec3 p, Vec3 q, Vec3 r) {
      const Vec3 c = unit(scale(add(add(p, q), r), 1.0 / 3.0));
      xi[k] = c.x;
      eta[k] = c.y;
      if (mu) mu[k] = c.z;
      w[k] = excess(unit(p), unit(q), unit(r));
      ++k;
    };
    for (int j = 0; j < N; ++j)
      for (int i = 0; i < N - j; ++i) {
        emit(P(i, j), P(i + 1, j), P(i, j + 1));
        if (i < N - 1 - j) emit(P(i + 1, j), P(i + 1, j + 1), P(i, j + 1));
      }
  }
  return RT_OK;
}
