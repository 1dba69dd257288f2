// Host-side FP64 construction of the preconditioning polynomial and of the
// quadrature rule used by the small projected solve.
#include <algorithm>
#include <cmath>
#include <complex>
#include <functional>
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

// Quadrature for z^{-1/2} = (2/pi) int_{-inf}^{inf} e^u / (e^{2u} + z) du, the
// small solve's sum over shifted systems: z^{-1/2} ~ sum_k wt_k / (sig_k + z).
//
// The plain trapezoid rule in u: the integrand is analytic in the strip
// |Im u| < (pi - |arg z|)/2, so the rule's error is about 2 exp(-2 pi d / h);
// d is taken as 0.9 of the strip half-width for |arg z| <= theta_max.  The
// two tails are cut where their relative contribution (2/pi) e^{u} z^{-1/2}
// (left) and (2/pi) e^{-u} z^{1/2} (right) falls below tau for z in [lo, hi].
// The integrand decays only like e^{-|u|}, so most nodes sit in the tails.
static void trapezoid_rule(double lo, double hi, double tau, double theta_max, std::vector<double> *sig,
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

// The same integral after u = uc + a sinh(w), uc = (log lo + log hi)/4: the
// integrand decays double-exponentially in w, so the tails take few nodes (a
// sinh-type double-exponential substitution of the Takahasi-Mori kind).
// Nodes whose u lies beyond the plain rule's tail cuts are left out (their
// terms are below tau).
static void sinh_rule(double lo, double hi, double tau, double a, double hw, std::vector<double> *sig,
                      std::vector<double> *wt) {
  const double uc = 0.25 * (std::log(lo) + std::log(hi));
  const double umin = std::log(tau * M_PI / 2.0) + 0.5 * std::log(lo) - 1.0;
  const double umax = -std::log(tau * M_PI / 2.0) + 0.5 * std::log(hi) + 1.0;
  const int n = (int)std::ceil(std::asinh(std::fmax(umax - uc, uc - umin) / a) / hw);
  sig->clear();
  wt->clear();
  for (int k = -n; k <= n; ++k) {
    const double w = k * hw, u = uc + a * std::sinh(w);
    if (u < umin || u > umax) continue;
    sig->push_back(std::exp(2.0 * u));
    wt->push_back((2.0 * hw / M_PI) * a * std::cosh(w) * std::exp(u));
  }
}

// Largest relative error of a rule over z = r e^{i phi}, kR radii log-spaced
// in [lo, hi], phi in {0, +-theta/2, +-theta}; the sum in real arithmetic
// (w / (s + x + i y) = w (s + x - i y) / ((s + x)^2 + y^2)).
static double rule_error(const std::vector<double> &sig, const std::vector<double> &wt, double lo, double hi,
                         double theta, int kR) {
  const double phis[3] = {0.0, 0.5 * theta, theta};
  double worst = 0.0;
  for (int i = 0; i < kR; ++i) {
    const double r = std::exp(std::log(lo) + (std::log(hi) - std::log(lo)) * i / (kR - 1));
    for (int j = 0; j < (theta > 0.0 ? 3 : 1); ++j) {
      // z and its conjugate give conjugate sums: one angle sign suffices
      const double x = r * std::cos(phis[j]), y = r * std::sin(phis[j]);
      double re = 0.0, im = 0.0;
      for (size_t k = 0; k < sig.size(); ++k) {
        const double sx = sig[k] + x, inv = wt[k] / (sx * sx + y * y);
        re += sx * inv;
        im -= y * inv;
      }
      const std::complex<double> sq = std::sqrt(std::complex<double>(x, y));
      const double e = std::abs(std::complex<double>(re, im) * sq - 1.0);
      if (!(e <= worst)) worst = e;  // NaN propagates as the worst
    }
  }
  return worst;
}

void invsqrt_quadrature(double lo, double hi, double tau, double theta_max, std::vector<double> *sig,
                        std::vector<double> *wt) {
  trapezoid_rule(lo, hi, tau, theta_max, sig, wt);
  // the sinh-mapped rule with the fewest nodes whose error on the sector
  // stays at the rounding level of the sums, 3e-15, or at twice the plain
  // rule's: for each scale a, the largest step hw that keeps it on a coarse
  // sample (bisection), then the winner checked on a fine sample, its step
  // reduced until it passes there
  constexpr int kCoarse = 64, kFine = 512;
  const double target = std::fmax(2.0 * rule_error(*sig, *wt, lo, hi, theta_max, kFine), 3e-15);
  std::vector<double> ts, tw;
  double best_a = 0.0, best_h = 0.0;
  size_t best_k = sig->size();
  for (double a : {1.0, 2.0, 4.0}) {
    double lo_h = 0.01, hi_h = 0.3;
    sinh_rule(lo, hi, tau, a, lo_h, &ts, &tw);
    if (!(rule_error(ts, tw, lo, hi, theta_max, kCoarse) <= target)) continue;
    for (int it = 0; it < 8; ++it) {
      const double mid = std::sqrt(lo_h * hi_h);
      sinh_rule(lo, hi, tau, a, mid, &ts, &tw);
      if (rule_error(ts, tw, lo, hi, theta_max, kCoarse) <= target)
        lo_h = mid;
      else
        hi_h = mid;
    }
    sinh_rule(lo, hi, tau, a, lo_h, &ts, &tw);
    if (ts.size() < best_k) {
      best_k = ts.size();
      best_a = a;
      best_h = lo_h;
    }
  }
  for (int it = 0; best_a > 0.0 && it < 6; ++it, best_h *= 0.9) {
    sinh_rule(lo, hi, tau, best_a, best_h, &ts, &tw);
    if (ts.size() >= sig->size()) break;
    if (rule_error(ts, tw, lo, hi, theta_max, kFine) <= target) {
      *sig = ts;
      *wt = tw;
      break;
    }
  }
}

// ---- interpolation at (harmonic) Ritz values (Sec. 5.2) ----

using cplx = std::complex<double>;

// Leja order: a node of largest modulus first, then each time the remaining
// node whose product of distances to the nodes already taken is largest
// (compared as sums of logarithms; ties go to the earlier node).  Nodes of a
// real problem come as real values or conjugate pairs: only the member with
// Im > 0 of a pair is a candidate, and its conjugate follows it at once.
// pairs = false (a complex operator): every node is a candidate on its own.
static std::vector<cplx> leja_order(const std::vector<cplx> &nodes, bool pairs = true) {
  std::vector<cplx> rest, out;
  for (const cplx &z : nodes)
    if (!pairs || z.imag() >= 0.0) rest.push_back(z);
  auto take = [&](size_t i) {
    const cplx z = rest[i];
    rest.erase(rest.begin() + (long)i);
    out.push_back(z);
    if (pairs && z.imag() > 0.0) out.push_back(std::conj(z));
  };
  size_t first = 0;
  for (size_t i = 1; i < rest.size(); ++i)
    if (std::abs(rest[i]) > std::abs(rest[first])) first = i;
  take(first);
  while (!rest.empty()) {
    size_t best = 0;
    double best_s = -INFINITY;
    for (size_t i = 0; i < rest.size(); ++i) {
      double s = 0.0;
      for (const cplx &x : out) s += rest[i] == x ? -INFINITY : std::log(std::abs(rest[i] - x));
      if (s > best_s) {
        best_s = s;
        best = i;
      }
    }
    take(best);
  }
  return out;
}

bool newton_form(const std::vector<cplx> &nodes, NewtonForm *F) {
  return newton_form_fn(nodes, [](cplx z) { return 1.0 / std::sqrt(z); }, F);
}

bool newton_form_fn(const std::vector<cplx> &nodes, const std::function<cplx(cplx)> &f, NewtonForm *F) {
  // Newton form with the nodes in reverse Leja order (a pair stays a pair,
  // Im > 0 first): the Horner scheme applies the factor of the last node
  // first, so the factors go on in Leja order.  With the Leja order itself
  // Horner lost the consistency of q(A) on non-normal operators (degree 15 on
  // a graph Laplacian: 156 Krylov steps and error 3e-4 against 20 steps and
  // 9e-9), while the reversed order matches the term-by-term Newton sum.
  const std::vector<cplx> lj = leja_order(nodes);
  if (lj.empty() || lj.size() != nodes.size()) return false;  // a pair without its conjugate
  std::vector<cplx> x;
  for (size_t e = lj.size(); e > 0;) {
    if (e >= 2 && lj[e - 1].imag() < 0.0) {  // a pair (z, conj z), z with Im > 0
      x.push_back(lj[e - 2]);
      x.push_back(lj[e - 1]);
      e -= 2;
    } else {
      x.push_back(lj[e - 1]);
      e -= 1;
    }
  }
  const size_t d = x.size();
  // divided differences a_i = f[x_0, ..., x_i]
  std::vector<cplx> col(d), a(d);
  for (size_t i = 0; i < d; ++i) col[i] = f(x[i]);
  a[0] = col[0];
  for (size_t k = 1; k < d; ++k) {
    for (size_t i = 0; i + k < d; ++i) col[i] = (col[i + 1] - col[i]) / (x[i + k] - x[i]);
    a[k] = col[0];
  }
  // scaling: a quarter of the diameter of the node set (the capacity of an interval)
  double diam = 0.0;
  for (size_t i = 0; i < d; ++i)
    for (size_t j = i + 1; j < d; ++j) diam = std::fmax(diam, std::abs(x[i] - x[j]));
  F->cap = diam > 0.0 ? 0.25 * diam : 1.0;
  // scaled Newton coefficients ah_i = a_i cap^i of the basis N_i = prod_{l<i} (z - x_l)/cap
  std::vector<cplx> ah(d);
  double p = 1.0;
  for (size_t i = 0; i < d; ++i) {
    ah[i] = a[i] * p;
    p *= F->cap;
  }
  // real basis: R_0 = 1; a real node x_i: R_{i+1} = ((z - x_i)/cap) R_i; a pair
  // (x_i, conj x_i): R_{i+1} = ((z - Re x_i)/cap) R_i and R_{i+2} = ((z - Re x_i)/cap)
  // R_{i+1} + (Im x_i/cap)^2 R_i.  N_i = R_i at the start of a pair, N_{i+1} =
  // R_{i+1} - i (Im x_i/cap) R_i, so q = sum b_i R_i with b_i = ah_i - i (Im x_i/cap)
  // ah_{i+1}, b_{i+1} = ah_{i+1} (real for a conjugation-closed node set).
  F->re.resize(d);
  F->im.resize(d);
  F->b.assign(d, 0.0);
  F->c.assign(d, 0.0);
  F->e.assign(d, 0.0);
  for (size_t i = 0; i < d; ++i) {
    F->re[i] = x[i].real();
    F->im[i] = x[i].imag();
  }
  for (size_t i = 0; i < d;) {
    F->c[i] = x[i].real();
    if (x[i].imag() > 0.0) {
      if (i + 1 >= d) return false;
      const double s = x[i].imag() / F->cap;
      F->b[i] = (ah[i] - cplx(0.0, s) * ah[i + 1]).real();
      F->b[i + 1] = ah[i + 1].real();
      F->c[i + 1] = x[i].real();
      F->e[i + 1] = s * s;
      i += 2;
    } else {
      F->b[i] = ah[i].real();
      i += 1;
    }
  }
  for (size_t i = 0; i < d; ++i)
    if (!std::isfinite(F->b[i])) return false;
  return true;
}

// Complex operator: the interpolant of f (default z^{-1/2}) at complex nodes
// with no conjugate symmetry, in Newton form at the nodes in reverse Leja
// order (as in newton_form_fn), basis N_i = prod_{l<i} (z - x_l)/cap,
// coefficients b_i = f[x_0..x_i] cap^i.
bool newton_form_cx_fn(const std::vector<cplx> &nodes, const std::function<cplx(cplx)> &f, NewtonForm *F) {
  const std::vector<cplx> lj = leja_order(nodes, false);
  if (lj.empty() || lj.size() != nodes.size()) return false;
  const std::vector<cplx> x(lj.rbegin(), lj.rend());
  const size_t d = x.size();
  std::vector<cplx> col(d), a(d);
  for (size_t i = 0; i < d; ++i) col[i] = f(x[i]);
  a[0] = col[0];
  for (size_t k = 1; k < d; ++k) {
    for (size_t i = 0; i + k < d; ++i) col[i] = (col[i + 1] - col[i]) / (x[i + k] - x[i]);
    a[k] = col[0];
  }
  double diam = 0.0;
  for (size_t i = 0; i < d; ++i)
    for (size_t j = i + 1; j < d; ++j) diam = std::fmax(diam, std::abs(x[i] - x[j]));
  F->cap = diam > 0.0 ? 0.25 * diam : 1.0;
  F->cx = true;
  F->re.resize(d);
  F->im.resize(d);
  F->b.resize(d);
  F->bi.resize(d);
  F->c.resize(d);
  F->ci.resize(d);
  F->e.assign(d, 0.0);
  double p = 1.0;
  for (size_t i = 0; i < d; ++i) {
    const cplx bh = a[i] * p;
    p *= F->cap;
    F->re[i] = F->c[i] = x[i].real();
    F->im[i] = F->ci[i] = x[i].imag();
    F->b[i] = bh.real();
    F->bi[i] = bh.imag();
    if (!std::isfinite(F->b[i]) || !std::isfinite(F->bi[i])) return false;
  }
  return true;
}

bool newton_form_cx(const std::vector<cplx> &nodes, NewtonForm *F) {
  return newton_form_cx_fn(nodes, [](cplx z) { return 1.0 / std::sqrt(z); }, F);
}

// q(z) by the backward recurrence of the basis: u_{k+1} = u_{k+2} = 0,
// u_i = b_i + ((z - c_i)/cap) u_{i+1} + e_{i+1} u_{i+2}, q(z) = u_0.
cplx newton_form_eval(const NewtonForm &F, cplx z) {
  const int k = (int)F.b.size() - 1;
  cplx u1 = 0.0, u2 = 0.0;
  if (F.cx) {
    for (int i = k; i >= 0; --i) u1 = cplx(F.b[i], F.bi[i]) + (z - cplx(F.c[i], F.ci[i])) / F.cap * u1;
    return u1;
  }
  for (int i = k; i >= 0; --i) {
    const cplx u0 = F.b[i] + (z - F.c[i]) / F.cap * u1 + (i + 1 <= k ? F.e[i + 1] : 0.0) * u2;
    u2 = u1;
    u1 = u0;
  }
  return u1;
}

// Positivity check and image of z q(z)^2 for a Newton-form q: the points of
// cheb_scan on [lo, hi] (q real there; skipped when hi <= lo), the nodes
// themselves and the extra points.  qmin is the smallest real part of q over
// the points, img_lo / img_hi the extremes of |z q(z)^2|.
void newton_scan(const NewtonForm &F, double lo, double hi, const std::vector<cplx> *extra, double *qmin,
                 double *img_lo, double *img_hi) {
  const int N = 20001;
  double qm = INFINITY, l = INFINITY, h = -INFINITY;
  auto visit = [&](cplx z) {
    const cplx q = newton_form_eval(F, z);
    const double p = std::abs(z * q * q);
    qm = std::fmin(qm, q.real());
    l = std::fmin(l, p);
    h = std::fmax(h, p);
  };
  if (hi > lo && lo > 0.0)
    for (int pass = 0; pass < 2; ++pass)
      for (int k = 0; k < N; ++k) {
        const double f = (double)k / (N - 1);
        visit(pass == 0 ? lo + (hi - lo) * f : lo * std::pow(hi / lo, f));
      }
  for (size_t i = 0; i < F.re.size(); ++i) visit(cplx(F.re[i], F.im[i]));
  if (extra)
    for (const cplx &z : *extra) visit(z);
  *qmin = qm;
  *img_lo = l;
  *img_hi = h;
}

// Eigenvalues of a complex upper Hessenberg matrix (n x n, row-major) by the
// shifted QR iteration with Givens rotations (Golub & Van Loan, Sec. 7.5,
// the single-shift form for complex matrices): Wilkinson shift from the
// trailing 2 x 2 block of the active window, an exceptional shift every 10
// iterations without deflation, deflation when |h_{k,k-1}| <= eps (|h_kk| +
// |h_{k-1,k-1}|).  Only the active window is transformed.  false if an
// eigenvalue has not converged after 60 n iterations.
bool zhess_eigvals(std::vector<cplx> H, int n, std::vector<cplx> *w) {
  auto h = [&](int i, int j) -> cplx & { return H[(size_t)i * n + j]; };
  w->assign(n, 0.0);
  const double eps = 0x1p-52;
  int hi = n - 1, iter = 0, total = 0;
  std::vector<cplx> cs(n), sn(n);
  while (hi >= 0) {
    int l = hi;
    while (l > 0) {
      const double s = std::abs(h(l - 1, l - 1)) + std::abs(h(l, l));
      if (std::abs(h(l, l - 1)) <= eps * (s > 0.0 ? s : 1.0)) break;
      --l;
    }
    if (l > 0) h(l, l - 1) = 0.0;
    if (l == hi) {
      (*w)[hi] = h(hi, hi);
      --hi;
      iter = 0;
      continue;
    }
    if (++total > 60 * n) return false;
    ++iter;
    cplx mu;
    if (iter % 10 == 0) {
      mu = h(hi, hi) + 0.75 * std::abs(h(hi, hi - 1));
    } else {
      const cplx a = h(hi - 1, hi - 1), b = h(hi - 1, hi), c = h(hi, hi - 1), d = h(hi, hi);
      const cplx half = 0.5 * (a - d);
      const cplx disc = std::sqrt(half * half + b * c);
      const cplx m1 = 0.5 * (a + d) + disc, m2 = 0.5 * (a + d) - disc;
      mu = std::abs(m1 - d) < std::abs(m2 - d) ? m1 : m2;
    }
    for (int k = l; k <= hi; ++k) h(k, k) -= mu;
    // H - mu I = QR: rotations G_k = [[conj c, conj s], [-s, c]] on rows k, k+1
    for (int k = l; k < hi; ++k) {
      const cplx x = h(k, k), y = h(k + 1, k);
      const double r = std::hypot(std::abs(x), std::abs(y));
      cs[k] = r > 0.0 ? x / r : cplx(1.0);
      sn[k] = r > 0.0 ? y / r : cplx(0.0);
      for (int j = k; j <= hi; ++j) {
        const cplx t1 = h(k, j), t2 = h(k + 1, j);
        h(k, j) = std::conj(cs[k]) * t1 + std::conj(sn[k]) * t2;
        h(k + 1, j) = -sn[k] * t1 + cs[k] * t2;
      }
    }
    // RQ + mu I: G_k^* on columns k, k+1
    for (int k = l; k < hi; ++k) {
      const int rmax = std::min(k + 1, hi);
      for (int i = l; i <= rmax; ++i) {
        const cplx t1 = h(i, k), t2 = h(i, k + 1);
        h(i, k) = t1 * cs[k] + t2 * sn[k];
        h(i, k + 1) = -t1 * std::conj(sn[k]) + t2 * std::conj(cs[k]);
      }
    }
    for (int k = l; k <= hi; ++k) h(k, k) += mu;
  }
  return true;
}

// f = M^{-*} e_n: Gaussian elimination with partial pivoting on M^* (complex).
bool zsolve_adjoint_last(const std::vector<cplx> &M, int n, std::vector<cplx> *f) {
  std::vector<cplx> A((size_t)n * n);
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) A[(size_t)i * n + j] = std::conj(M[(size_t)j * n + i]);
  std::vector<cplx> r(n, 0.0);
  r[n - 1] = 1.0;
  for (int k = 0; k < n; ++k) {
    int p = k;
    for (int i = k + 1; i < n; ++i)
      if (std::abs(A[(size_t)i * n + k]) > std::abs(A[(size_t)p * n + k])) p = i;
    if (!(std::abs(A[(size_t)p * n + k]) > 0.0)) return false;
    if (p != k) {
      for (int j = 0; j < n; ++j) std::swap(A[(size_t)p * n + j], A[(size_t)k * n + j]);
      std::swap(r[p], r[k]);
    }
    for (int i = k + 1; i < n; ++i) {
      const cplx g = A[(size_t)i * n + k] / A[(size_t)k * n + k];
      if (g == 0.0) continue;
      for (int j = k; j < n; ++j) A[(size_t)i * n + j] -= g * A[(size_t)k * n + j];
      r[i] -= g * r[k];
    }
  }
  f->assign(n, 0.0);
  for (int i = n - 1; i >= 0; --i) {
    cplx t = r[i];
    for (int j = i + 1; j < n; ++j) t -= A[(size_t)i * n + j] * (*f)[j];
    (*f)[i] = t / A[(size_t)i * n + i];
  }
  for (int i = 0; i < n; ++i)
    if (!std::isfinite((*f)[i].real()) || !std::isfinite((*f)[i].imag())) return false;
  return true;
}

// Eigenvalues of a real upper Hessenberg matrix (n x n, row-major, overwritten)
// by the Francis double-shift QR iteration with deflation (Golub & Van Loan,
// Sec. 7.5), transforming only the active diagonal block (eigenvalues only).
// Complex eigenvalues come as exact conjugate pairs (Im > 0 first).  Returns
// false if an eigenvalue has not converged after 60 n double steps.
bool hess_eigvals(std::vector<double> H, int n, std::vector<double> *wr, std::vector<double> *wi) {
  auto h = [&](int i, int j) -> double & { return H[(size_t)i * n + j]; };
  wr->assign(n, 0.0);
  wi->assign(n, 0.0);
  int u = n - 1, iter = 0, total = 0;
  while (u >= 0) {
    int l = u;
    for (; l > 0; --l) {
      double s = std::fabs(h(l - 1, l - 1)) + std::fabs(h(l, l));
      if (s == 0.0) s = 1.0;
      if (std::fabs(h(l, l - 1)) <= 0x1p-53 * s) {
        h(l, l - 1) = 0.0;
        break;
      }
    }
    if (l == u) {  // 1 x 1 block
      (*wr)[u] = h(u, u);
      --u;
      iter = 0;
      continue;
    }
    if (l == u - 1) {  // 2 x 2 block
      const double a = h(u - 1, u - 1), b = h(u - 1, u), c = h(u, u - 1), d = h(u, u);
      const double mid = 0.5 * (a + d), p = 0.5 * (a - d), disc = p * p + b * c;
      if (disc >= 0.0) {
        const double sq = std::sqrt(disc);
        const double r1 = mid + (mid >= 0.0 ? sq : -sq);
        const double r2 = r1 != 0.0 ? (a * d - b * c) / r1 : mid - sq;
        (*wr)[u - 1] = r1;
        (*wr)[u] = r2;
      } else {
        const double sq = std::sqrt(-disc);
        (*wr)[u - 1] = (*wr)[u] = mid;
        (*wi)[u - 1] = sq;
        (*wi)[u] = -sq;
      }
      u -= 2;
      iter = 0;
      continue;
    }
    if (++total > 60 * n) return false;
    ++iter;
    double s, t;  // sum and product of the two shifts
    if (iter % 11 == 10) {  // exceptional shift after a run without deflation
      const double w = std::fabs(h(u, u - 1)) + std::fabs(h(u - 1, u - 2));
      s = 1.5 * w + h(u, u);
      t = s * s / 4.0 + w * w;
    } else {
      s = h(u - 1, u - 1) + h(u, u);
      t = h(u - 1, u - 1) * h(u, u) - h(u - 1, u) * h(u, u - 1);
    }
    // first column of (H - s1 I)(H - s2 I) restricted to the block
    double x = h(l, l) * h(l, l) + h(l, l + 1) * h(l + 1, l) - s * h(l, l) + t;
    double y = h(l + 1, l) * (h(l, l) + h(l + 1, l + 1) - s);
    double z = h(l + 1, l) * h(l + 2, l + 1);
    for (int k = l; k <= u - 1; ++k) {
      const int r = k <= u - 2 ? 3 : 2;  // reflector size
      double v[3] = {x, y, r == 3 ? z : 0.0};
      const double nrm = std::sqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
      if (nrm != 0.0) {
        const double alpha = v[0] >= 0.0 ? -nrm : nrm;
        v[0] -= alpha;
        const double vv = v[0] * v[0] + v[1] * v[1] + v[2] * v[2];
        if (vv != 0.0) {
          const double beta = 2.0 / vv;
          for (int j = std::max(l, k - 1); j <= u; ++j) {  // rows k .. k+r-1 from the left
            double sm = 0.0;
            for (int q = 0; q < r; ++q) sm += v[q] * h(k + q, j);
            sm *= beta;
            for (int q = 0; q < r; ++q) h(k + q, j) -= sm * v[q];
          }
          for (int i = l; i <= std::min(k + 3, u); ++i) {  // columns k .. k+r-1 from the right
            double sm = 0.0;
            for (int q = 0; q < r; ++q) sm += h(i, k + q) * v[q];
            sm *= beta;
            for (int q = 0; q < r; ++q) h(i, k + q) -= sm * v[q];
          }
        }
      }
      if (k + 1 <= u - 1) {
        x = h(k + 1, k);
        y = h(k + 2, k);
        z = k + 3 <= u ? h(k + 3, k) : 0.0;
      }
    }
  }
  return true;
}

// Solve M^T f = e_last for a dense n x n M (row-major) by Gaussian
// elimination with partial pivoting; false if M is singular.
bool solve_transposed_last(const std::vector<double> &M, int n, std::vector<double> *f) {
  std::vector<double> T((size_t)n * n), rhs(n, 0.0);
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) T[(size_t)i * n + j] = M[(size_t)j * n + i];
  rhs[n - 1] = 1.0;
  for (int k = 0; k < n; ++k) {
    int pr = k;
    for (int i = k + 1; i < n; ++i)
      if (std::fabs(T[(size_t)i * n + k]) > std::fabs(T[(size_t)pr * n + k])) pr = i;
    if (T[(size_t)pr * n + k] == 0.0) return false;
    if (pr != k) {
      for (int j = 0; j < n; ++j) std::swap(T[(size_t)k * n + j], T[(size_t)pr * n + j]);
      std::swap(rhs[k], rhs[pr]);
    }
    for (int i = k + 1; i < n; ++i) {
      const double m = T[(size_t)i * n + k] / T[(size_t)k * n + k];
      if (m == 0.0) continue;
      for (int j = k; j < n; ++j) T[(size_t)i * n + j] -= m * T[(size_t)k * n + j];
      rhs[i] -= m * rhs[k];
    }
  }
  f->assign(n, 0.0);
  for (int i = n - 1; i >= 0; --i) {
    double sm = rhs[i];
    for (int j = i + 1; j < n; ++j) sm -= T[(size_t)i * n + j] * (*f)[j];
    (*f)[i] = sm / T[(size_t)i * n + i];
  }
  return true;
}

// Eigenvalues of a symmetric n x n matrix M (row-major, overwritten) by the
// cyclic Jacobi method (Golub & Van Loan, Sec. 8.5), ascending.
std::vector<double> sym_eigvals(std::vector<double> M, int n) {
  auto at = [&](int i, int j) -> double & { return M[(size_t)i * n + j]; };
  for (int sweep = 0; sweep < 100; ++sweep) {
    double off = 0.0, tot = 0.0;
    for (int i = 0; i < n; ++i)
      for (int j = 0; j < n; ++j) {
        tot += at(i, j) * at(i, j);
        if (i != j) off += at(i, j) * at(i, j);
      }
    if (off <= 1e-30 * tot) break;
    for (int p = 0; p < n - 1; ++p)
      for (int q = p + 1; q < n; ++q) {
        const double apq = at(p, q);
        if (apq == 0.0) continue;
        // rotation that zeroes M[p][q]: tan of the angle t solves t^2 + 2 tau t - 1 = 0
        const double tau = (at(q, q) - at(p, p)) / (2.0 * apq);
        const double t = (tau >= 0 ? 1.0 : -1.0) / (std::fabs(tau) + std::sqrt(1.0 + tau * tau));
        const double cs = 1.0 / std::sqrt(1.0 + t * t), sn = t * cs;
        for (int k = 0; k < n; ++k) {  // columns p, q
          const double mkp = at(k, p), mkq = at(k, q);
          at(k, p) = cs * mkp - sn * mkq;
          at(k, q) = sn * mkp + cs * mkq;
        }
        for (int k = 0; k < n; ++k) {  // rows p, q
          const double mpk = at(p, k), mqk = at(q, k);
          at(p, k) = cs * mpk - sn * mqk;
          at(q, k) = sn * mpk + cs * mqk;
        }
      }
  }
  std::vector<double> ev(n);
  for (int i = 0; i < n; ++i) ev[i] = at(i, i);
  std::sort(ev.begin(), ev.end());
  return ev;
}

// Harmonic Ritz values of a symmetric positive definite tridiagonal T
// (diagonal al, off-diagonal be[0..m-2]) with next coefficient beta = h_{m+1,m}:
// the eigenvalues of T + beta^2 T^{-1} e_m e_m^T, i.e. of the symmetric pencil
// (T^2 + beta^2 e_m e_m^T, T).  With T = L L^T (Cholesky, L lower bidiagonal)
// they are the eigenvalues of the symmetric L^{-1} (T^2 + beta^2 e_m e_m^T) L^{-T}.
// Returns false if T is not positive definite.
bool harmonic_ritz(const std::vector<double> &al, const std::vector<double> &be, double beta,
                   std::vector<double> *out) {
  const int m = (int)al.size();
  std::vector<double> ld(m), ls(m > 1 ? m - 1 : 0);  // diagonal and sub-diagonal of L
  for (int i = 0; i < m; ++i) {
    const double piv = al[i] - (i > 0 ? ls[i - 1] * ls[i - 1] : 0.0);
    if (!(piv > 0.0)) return false;
    ld[i] = std::sqrt(piv);
    if (i + 1 < m) ls[i] = be[i] / ld[i];
  }
  // B = T^2 + beta^2 e_m e_m^T (dense, symmetric)
  std::vector<double> T((size_t)m * m, 0.0), B((size_t)m * m, 0.0);
  for (int i = 0; i < m; ++i) {
    T[(size_t)i * m + i] = al[i];
    if (i + 1 < m) T[(size_t)i * m + i + 1] = T[(size_t)(i + 1) * m + i] = be[i];
  }
  for (int i = 0; i < m; ++i)
    for (int j = std::max(0, i - 2); j <= std::min(m - 1, i + 2); ++j) {
      double s = 0.0;
      for (int k = std::max(0, i - 1); k <= std::min(m - 1, i + 1); ++k) s += T[(size_t)i * m + k] * T[(size_t)k * m + j];
      B[(size_t)i * m + j] = s;
    }
  B[(size_t)(m - 1) * m + m - 1] += beta * beta;
  // C = L^{-1} B (forward substitution on each column), then M = C L^{-T}
  // (forward substitution on each row of C, i.e. on the columns of C^T)
  for (int j = 0; j < m; ++j)
    for (int i = 0; i < m; ++i) {
      double v = B[(size_t)i * m + j] - (i > 0 ? ls[i - 1] * B[(size_t)(i - 1) * m + j] : 0.0);
      B[(size_t)i * m + j] = v / ld[i];
    }
  for (int i = 0; i < m; ++i)
    for (int j = 0; j < m; ++j) {
      double v = B[(size_t)i * m + j] - (j > 0 ? ls[j - 1] * B[(size_t)i * m + j - 1] : 0.0);
      B[(size_t)i * m + j] = v / ld[j];
    }
  for (int i = 0; i < m; ++i)  // symmetrize the rounding
    for (int j = i + 1; j < m; ++j) {
      const double s = 0.5 * (B[(size_t)i * m + j] + B[(size_t)j * m + i]);
      B[(size_t)i * m + j] = B[(size_t)j * m + i] = s;
    }
  *out = sym_eigvals(B, m);
  return true;
}

// ---- least-squares polynomial on a discretized contour (Sec. 5.3) ----

// Arnoldi on diag(z_1..z_N) from the vector of ones / sqrt(N) (modified
// Gram-Schmidt): d orthonormal basis polynomials for <p1, p2> = sum_i
// p1(z_i) conj(p2(z_i)); H (d x (d-1), column-major in H[j + k d]) with
// z p_{k} = sum_{j<=k+1} h_{j,k} p_j; alpha_j = <z^{-1/2}, p_j>.  False if
// the points carry fewer than d distinct values (a zero h_{k+1,k}).
bool lsq_poly(const std::vector<cplx> &z, int d, std::vector<cplx> *H, std::vector<cplx> *alpha) {
  const size_t N = z.size();
  std::vector<cplx> P(N * (size_t)d);
  H->assign((size_t)d * (size_t)d, 0.0);
  alpha->assign(d, 0.0);
  for (size_t i = 0; i < N; ++i) P[i] = 1.0 / std::sqrt((double)N);
  std::vector<cplx> w(N);
  for (int k = 1; k < d; ++k) {
    for (size_t i = 0; i < N; ++i) w[i] = z[i] * P[(size_t)(k - 1) * N + i];
    for (int j = 0; j < k; ++j) {
      cplx h = 0.0;
      for (size_t i = 0; i < N; ++i) h += std::conj(P[(size_t)j * N + i]) * w[i];
      (*H)[j + (size_t)(k - 1) * d] = h;
      for (size_t i = 0; i < N; ++i) w[i] -= h * P[(size_t)j * N + i];
    }
    double nr = 0.0;
    for (size_t i = 0; i < N; ++i) nr += std::norm(w[i]);
    nr = std::sqrt(nr);
    if (!(nr > 0.0) || !std::isfinite(nr)) return false;
    (*H)[k + (size_t)(k - 1) * d] = nr;
    for (size_t i = 0; i < N; ++i) P[(size_t)k * N + i] = w[i] / nr;
  }
  for (int j = 0; j < d; ++j) {
    cplx a = 0.0;
    for (size_t i = 0; i < N; ++i) a += std::conj(P[(size_t)j * N + i]) / std::sqrt(z[i]);
    (*alpha)[j] = a;
  }
  return true;
}

// q(z) = sum_j alpha_j p_j(z) by the basis recurrence of lsq_poly.
cplx lsq_eval(const std::vector<cplx> &H, const std::vector<cplx> &alpha, size_t N, cplx z) {
  const int d = (int)alpha.size();
  std::vector<cplx> p(d);
  p[0] = 1.0 / std::sqrt((double)N);
  cplx q = alpha[0] * p[0];
  for (int k = 1; k < d; ++k) {
    cplx w = z * p[k - 1];
    for (int j = 0; j < k; ++j) w -= H[j + (size_t)(k - 1) * d] * p[j];
    p[k] = w / H[k + (size_t)(k - 1) * d];
    q += alpha[k] * p[k];
  }
  return q;
}

// d points of a conjugation-symmetric set in Leja order for interpolation:
// greedy by product distance over the members with Im >= 0, a complex
// choice bringing its conjugate along; when one slot is left a real point is
// taken.  False if the set cannot supply d points that way.
bool leja_select(const std::vector<cplx> &pts, int d, std::vector<cplx> *out) {
  std::vector<cplx> cand;
  for (const cplx &z : pts)
    if (z.imag() >= 0.0) cand.push_back(z);
  out->clear();
  std::vector<double> logp(cand.size(), 0.0);
  std::vector<char> used(cand.size(), 0);
  auto add = [&](const cplx &x) {
    out->push_back(x);
    for (size_t i = 0; i < cand.size(); ++i)
      logp[i] += cand[i] == x ? -INFINITY : std::log(std::abs(cand[i] - x));
  };
  int reals = 0;
  for (const cplx &z : cand) reals += z.imag() == 0.0 ? 1 : 0;
  while ((int)out->size() < d) {
    const int left = d - (int)out->size();
    int best = -1;
    double bs = -INFINITY;
    for (size_t i = 0; i < cand.size(); ++i) {
      if (used[i]) continue;
      // keep the rest fillable: an odd remainder needs a real point left
      if (cand[i].imag() != 0.0) {
        if (left < 2 || ((left - 2) % 2 == 1 && reals < 1)) continue;
      } else if ((left - 1) % 2 == 1 && reals - 1 < 1) {
        continue;
      }
      const double sc = out->empty() ? std::abs(cand[i]) : logp[i];
      if (best < 0 || sc > bs) {
        bs = sc;
        best = (int)i;
      }
    }
    if (best < 0 || (!std::isfinite(bs) && !out->empty())) return false;
    used[best] = 1;
    if (cand[best].imag() == 0.0) --reals;
    add(cand[best]);
    if (cand[best].imag() > 0.0) add(std::conj(cand[best]));
  }
  return true;
}

// The contour of Sec. 5.3 from Ritz values: their convex hull made symmetric
// about the real axis, densely resampled, points with |z| < r_min moved
// radially onto that circle (the part of the hull there becomes the arc),
// then npts points at equal arc length (npts/2 on the upper half from the
// right end on the real axis to the left end, mirrored).  All-real Ritz
// values give npts points evenly spaced on [max(min, r_min), max].
std::vector<cplx> lsq_contour(const std::vector<cplx> &ritz, double r_min, int npts) {
  bool real = true;
  double mn = INFINITY, mx = -INFINITY;
  for (const cplx &z : ritz) {
    real = real && z.imag() == 0.0;
    mn = std::fmin(mn, z.real());
    mx = std::fmax(mx, z.real());
  }
  std::vector<cplx> out;
  if (real) {
    const double lo = std::fmax(mn, r_min);
    for (int i = 0; i < npts; ++i) out.emplace_back(lo + (mx - lo) * (double)i / (npts - 1), 0.0);
    return out;
  }
  // upper hull, right to left (monotone chain over the symmetric set)
  std::vector<std::pair<double, double>> P;
  for (const cplx &z : ritz) {
    P.emplace_back(z.real(), z.imag());
    P.emplace_back(z.real(), -z.imag());
  }
  std::sort(P.begin(), P.end());
  P.erase(std::unique(P.begin(), P.end()), P.end());
  std::vector<std::pair<double, double>> up;
  for (auto it = P.rbegin(); it != P.rend(); ++it) {
    while (up.size() >= 2) {
      const auto &o = up[up.size() - 2], &a = up.back();
      const double cr = (a.first - o.first) * (it->second - o.second) - (a.second - o.second) * (it->first - o.first);
      if (cr <= 0.0)
        up.pop_back();
      else
        break;
    }
    up.push_back(*it);
  }
  std::vector<cplx> chain;
  chain.emplace_back(P.back().first, 0.0);
  for (const auto &p : up)
    if (p.second > 0.0) chain.emplace_back(p.first, p.second);
  chain.emplace_back(P.front().first, 0.0);
  // dense resampling at 40 npts points of equal chain length
  std::vector<double> seg(chain.size() - 1), s(chain.size(), 0.0);
  for (size_t i = 0; i + 1 < chain.size(); ++i) {
    seg[i] = std::abs(chain[i + 1] - chain[i]);
    s[i + 1] = s[i] + seg[i];
  }
  const int nd = 40 * npts;
  std::vector<cplx> dense(nd);
  for (int i = 0; i < nd; ++i) {
    const double t = s.back() * (double)i / (nd - 1);
    size_t k = std::upper_bound(s.begin(), s.end(), t) - s.begin();
    k = k == 0 ? 0 : k - 1;
    if (k >= seg.size()) k = seg.size() - 1;
    while (k + 1 < seg.size() && seg[k] == 0.0) ++k;
    cplx z = seg[k] > 0.0 ? chain[k] + (chain[k + 1] - chain[k]) * ((t - s[k]) / seg[k]) : chain[k];
    if (std::abs(z) < r_min) z *= r_min / std::abs(z);
    dense[i] = z;
  }
  // equal arc length along the modified curve
  std::vector<double> arc(nd, 0.0);
  for (int i = 1; i < nd; ++i) arc[i] = arc[i - 1] + std::abs(dense[i] - dense[i - 1]);
  const int m = npts / 2;
  std::vector<cplx> half(m);
  size_t j = 0;
  for (int i = 0; i < m; ++i) {
    const double t = arc.back() * (double)i / (m - 1);
    while (j + 1 < (size_t)nd - 1 && arc[j + 1] < t) ++j;
    const double w = arc[j + 1] > arc[j] ? (t - arc[j]) / (arc[j + 1] - arc[j]) : 0.0;
    half[i] = dense[j] + (dense[j + 1] - dense[j]) * std::fmin(1.0, std::fmax(0.0, w));
  }
  half[0] = half[0].real();
  half[m - 1] = half[m - 1].real();
  out = half;
  for (int i = 1; i + 1 < m; ++i) out.push_back(std::conj(half[i]));
  return out;
}

// d points of a set in Leja order, no conjugate symmetry (the points of a
// contour for a complex operator): the point of largest modulus, then each
// time the point with the largest product of distances to those taken.
bool leja_select_cx(const std::vector<cplx> &pts, int d, std::vector<cplx> *out) {
  out->clear();
  std::vector<double> logp(pts.size(), 0.0);
  std::vector<char> used(pts.size(), 0);
  while ((int)out->size() < d) {
    int best = -1;
    double bs = -INFINITY;
    for (size_t i = 0; i < pts.size(); ++i) {
      if (used[i]) continue;
      const double sc = out->empty() ? std::abs(pts[i]) : logp[i];
      if (best < 0 || sc > bs) {
        bs = sc;
        best = (int)i;
      }
    }
    if (best < 0 || (!std::isfinite(bs) && !out->empty())) return false;
    used[best] = 1;
    const cplx x = pts[best];
    out->push_back(x);
    for (size_t i = 0; i < pts.size(); ++i) logp[i] += pts[i] == x ? -INFINITY : std::log(std::abs(pts[i] - x));
  }
  return true;
}

// The contour of Sec. 5.3 for a complex operator (no symmetry about the real
// axis): the convex hull of the Ritz values as a closed polygon, densely
// resampled, points with |z| < r_min moved radially onto that circle, then
// npts points at equal arc length around the closed curve.  A single point
// (or collinear values) gives the segment between the extreme ones.
std::vector<cplx> lsq_contour_cx(const std::vector<cplx> &ritz, double r_min, int npts) {
  std::vector<std::pair<double, double>> P;
  for (const cplx &z : ritz) P.emplace_back(z.real(), z.imag());
  std::sort(P.begin(), P.end());
  P.erase(std::unique(P.begin(), P.end()), P.end());
  auto cross = [](const std::pair<double, double> &o, const std::pair<double, double> &a,
                  const std::pair<double, double> &b) {
    return (a.first - o.first) * (b.second - o.second) - (a.second - o.second) * (b.first - o.first);
  };
  // Andrew's monotone chain: lower hull left to right, upper hull right to left
  std::vector<std::pair<double, double>> hull;
  for (const auto &p : P) {
    while (hull.size() >= 2 && cross(hull[hull.size() - 2], hull.back(), p) <= 0.0) hull.pop_back();
    hull.push_back(p);
  }
  const size_t lower = hull.size();
  for (auto it = P.rbegin() + 1; it != P.rend(); ++it) {
    while (hull.size() > lower && cross(hull[hull.size() - 2], hull.back(), *it) <= 0.0) hull.pop_back();
    hull.push_back(*it);
  }
  std::vector<cplx> poly;  // closed: last vertex equals the first
  for (const auto &p : hull) poly.emplace_back(p.first, p.second);
  if (poly.size() < 3) {  // degenerate hull: the segment between the extremes, both ways
    poly.clear();
    poly.emplace_back(P.front().first, P.front().second);
    poly.emplace_back(P.back().first, P.back().second);
    poly.emplace_back(P.front().first, P.front().second);
  }
  std::vector<double> s(poly.size(), 0.0);
  for (size_t i = 0; i + 1 < poly.size(); ++i) s[i + 1] = s[i] + std::abs(poly[i + 1] - poly[i]);
  const int nd = 40 * npts;
  std::vector<cplx> dense(nd);
  for (int i = 0; i < nd; ++i) {
    const double t = s.back() * (double)i / nd;
    size_t k = std::upper_bound(s.begin(), s.end(), t) - s.begin();
    k = k == 0 ? 0 : k - 1;
    if (k + 1 >= poly.size()) k = poly.size() - 2;
    const double len = s[k + 1] - s[k];
    cplx z = len > 0.0 ? poly[k] + (poly[k + 1] - poly[k]) * ((t - s[k]) / len) : poly[k];
    if (std::abs(z) < r_min) z *= r_min / std::abs(z);
    dense[i] = z;
  }
  std::vector<double> arc(nd + 1, 0.0);
  for (int i = 1; i <= nd; ++i) arc[i] = arc[i - 1] + std::abs(dense[i % nd] - dense[i - 1]);
  std::vector<cplx> out(npts);
  size_t j = 0;
  for (int i = 0; i < npts; ++i) {
    const double t = arc.back() * (double)i / npts;
    while (j + 1 < (size_t)nd && arc[j + 1] < t) ++j;
    const double w = arc[j + 1] > arc[j] ? (t - arc[j]) / (arc[j + 1] - arc[j]) : 0.0;
    out[i] = dense[j] + (dense[(j + 1) % nd] - dense[j]) * std::fmin(1.0, std::fmax(0.0, w));
  }
  return out;
}

