// Host-side FP64 construction of the preconditioning polynomial and of the
// quadrature rule used by the small projected solve.
#include <cmath>
#include <vector>

#include "internal.h"

// Chebyshev polynomial for z^{-1/2} on [a,b] (Sec. 5.1).  The coefficient
// integrals c_i = (2/pi) int w(z) f(z) T_i^{[a,b]}(z) dz (c_0 with 1/pi) are
// evaluated with the (degree+1)-point Gauss-Chebyshev rule, which makes q the
// interpolant of z^{-1/2} at the first-kind Chebyshev nodes of [a,b].  This
// is the reading under which the worked example of Sec. 3.2 (50 x 50
// Laplacian, d = 32) gives the printed kappa_pre = 1.5153.
std::vector<double> cheb_interp_coeffs(double a, double b, int degree) {
  const int d = degree + 1;
  std::vector<double> fz(d), c(d, 0.0);
  for (int k = 0; k < d; ++k) {
    const double t = M_PI * (k + 0.5) / d;
    const double z = 0.5 * (a + b) + 0.5 * (b - a) * std::cos(t);
    fz[k] = 1.0 / std::sqrt(z);
  }
  for (int i = 0; i < d; ++i) {
    double s = 0.0;
    for (int k = 0; k < d; ++k) s += fz[k] * std::cos(i * M_PI * (k + 0.5) / d);
    c[i] = (i == 0 ? 1.0 : 2.0) * s / d;
  }
  return c;
}

// Scalar Clenshaw evaluation of q(z) = sum c_i T_i((2z - a - b)/(b - a)).
double cheb_eval(const std::vector<double> &c, double a, double b, double z) {
  const double x = (2.0 * z - a - b) / (b - a);
  double b1 = 0.0, b2 = 0.0;
  for (int i = (int)c.size() - 1; i >= 1; --i) {
    const double b0 = 2.0 * x * b1 - b2 + c[i];
    b2 = b1;
    b1 = b0;
  }
  return x * b1 - b2 + c[0];
}

// Dense scan of [a,b] (uniform and geometric points, endpoints included) for
// the positivity check of Sec. 5.1 and the image interval of z q(z)^2.
void cheb_scan(const std::vector<double> &c, double a, double b, double *qmin, double *img_lo,
               double *img_hi) {
  const int N = 20001;
  double qm = INFINITY, lo = INFINITY, hi = -INFINITY;
  for (int pass = 0; pass < 2; ++pass) {
    for (int k = 0; k < N; ++k) {
      const double f = (double)k / (N - 1);
      const double z = pass == 0 ? a + (b - a) * f : a * std::pow(b / a, f);
      const double q = cheb_eval(c, a, b, z);
      const double p = z * q * q;
      qm = std::fmin(qm, q);
      lo = std::fmin(lo, p);
      hi = std::fmax(hi, p);
    }
  }
  *qmin = qm;
  *img_lo = lo;
  *img_hi = hi;
}

// Trapezoid rule for z^{-1/2} = (2/pi) int_{-inf}^{inf} e^u / (e^{2u} + z) du.
// The integrand is analytic in the strip |Im u| < (pi - |arg z|)/2, so the
// trapezoid error is about 2 exp(-2 pi d / h); d is taken as 0.9 of the strip
// half-width for |arg z| <= theta_max.  The two tails are cut where their
// relative contribution (2/pi) e^{u} z^{-1/2} (left) and (2/pi) e^{-u} z^{1/2}
// (right) falls below tau for z in [lo, hi].
void invsqrt_quadrature(double lo, double hi, double tau, double theta_max, std::vector<double> *sig,
                        std::vector<double> *wt) {
  const double d = 0.9 * 0.5 * (M_PI - theta_max);
  const double h = 2.0 * M_PI * d / std::log(2.0 / tau);
  const double umin = std::log(tau * M_PI / 2.0) + 0.5 * std::log(lo);
  const double umax = -std::log(tau * M_PI / 2.0) + 0.5 * std::log(hi);
  const int K = (int)std::ceil((umax - umin) / h) + 1;
  sig->resize(K);
  wt->resize(K);
  for (int k = 0; k < K; ++k) {
    const double u = umin + k * h;
    (*sig)[k] = std::exp(2.0 * u);
    (*wt)[k] = (2.0 * h / M_PI) * std::exp(u);
  }
}
