// Host FP64 table generation for the SGL transform.
//
// Every table the kernels read is built here, on the host, once per plan:
//  * radial nodes t_i (zeros of L_B^(1/2)) by Sturm-sequence bisection on the
//    Jacobi matrix of the Laguerre recurrence Eq. (laguerre_recursion),
//    refined by Newton steps on the orthonormal recurrence in long double;
//  * the radial functions T_nl(i) = N_nl R_nl(r_i) exp(-t_i/2) by Lemma 3.7
//    (read for the normalized functions N_nl R_nl), started from
//    sqrt(2/Gamma(l+3/2)) r^l exp(-t/2) built multiplicatively in l;
//  * radial weights what_i = (w_i/2) exp(t_i) as the reciprocal Christoffel
//    function 1 / sum_{n<=B} T_n0(i)^2 (Gauss weights of the rule in t = r^2);
//  * the equiangular sphere rule of Thm 3.1 with beta_j = (pi/B) b_j;
//  * fully normalized Legendre functions Lambda_lm(theta_j) = Y_lm e^{-i m phi}
//    (Def 2.1 with the Condon-Shortley phase) by the normalized form of
//    Eq. (legendre_recurrence), with sectoral seeds built multiplicatively in m.
#include <math.h>

#include <algorithm>
#include <string>
#include <vector>

#include "sgl_internal.h"

namespace sgl {

namespace {

const long double kPiL = 3.141592653589793238462643383279502884L;

// Jacobi matrix of the Laguerre weight t^alpha e^{-t}: diagonal 2k + alpha + 1,
// off-diagonal sqrt(k (k + alpha)), k >= 1.
int sturm_count(const std::vector<double>& d, const std::vector<double>& e2, double x) {
  int count = 0;
  double q = d[0] - x;
  if (q < 0) ++count;
  for (size_t k = 1; k < d.size(); ++k) {
    if (q == 0.0) q = 1e-300;
    q = (d[k] - x) - e2[k] / q;
    if (q < 0) ++count;
  }
  return count;
}

// Orthonormal Laguerre recurrence value and derivative at t (degree n).
void orthonormal_laguerre(int n, long double alpha, long double t, long double& p, long double& dp) {
  long double pm1 = 0.0L, dpm1 = 0.0L;
  long double p0 = 1.0L, dp0 = 0.0L;
  long double bk = 0.0L;
  for (int k = 0; k < n; ++k) {
    long double ak = 2.0L * k + alpha + 1.0L;
    long double bk1 = sqrtl((long double)(k + 1) * ((long double)(k + 1) + alpha));
    long double p1 = ((t - ak) * p0 - bk * pm1) / bk1;
    long double dp1 = (p0 + (t - ak) * dp0 - bk * dpm1) / bk1;
    pm1 = p0; dpm1 = dp0;
    p0 = p1; dp0 = dp1;
    bk = bk1;
  }
  p = p0;
  dp = dp0;
}

bool radial_nodes(int B, std::vector<double>& t, std::string& msg) {
  const double alpha = 0.5;
  std::vector<double> d(B), e2(B, 0.0);
  double hi = 0.0;
  for (int k = 0; k < B; ++k) {
    d[k] = 2.0 * k + alpha + 1.0;
    if (k > 0) e2[k] = k * (k + alpha);
  }
  for (int k = 0; k < B; ++k) {
    double r = d[k] + (k > 0 ? sqrt(e2[k]) : 0.0) + (k + 1 < B ? sqrt(e2[k + 1]) : 0.0);
    hi = std::max(hi, r);
  }
  t.assign(B, 0.0);
  for (int i = 0; i < B; ++i) {
    double lo = 0.0, up = hi;
    for (int it = 0; it < 200 && up - lo > 1e-15 * std::max(1.0, up); ++it) {
      double mid = 0.5 * (lo + up);
      if (sturm_count(d, e2, mid) > i) up = mid; else lo = mid;
    }
    long double x = 0.5L * ((long double)lo + (long double)up);
    for (int it = 0; it < 6; ++it) {
      long double p, dp;
      orthonormal_laguerre(B, alpha, x, p, dp);
      if (dp == 0.0L) break;
      long double step = p / dp;
      x -= step;
      if (fabsl(step) <= 1e-19L * fabsl(x)) break;
    }
    if (!(x > 0.0L) || !isfinite((double)x)) {
      msg = "radial node search failed";
      return false;
    }
    t[i] = (double)x;
  }
  for (int i = 1; i < B; ++i) {
    if (!(t[i] > t[i - 1])) {
      msg = "radial nodes not increasing";
      return false;
    }
  }
  return true;
}

}  // namespace

bool build_tables(int B, HostTables& out, std::string& msg) {
  if (!bandlimit_supported(B)) {
    msg = "unsupported bandlimit";
    return false;
  }
  out.B = B;
  if (!radial_nodes(B, out.t, msg)) return false;
  out.r.resize(B);
  for (int i = 0; i < B; ++i) out.r[i] = sqrt(out.t[i]);

  // radial functions, Lemma 3.7 (normalized reading)
  out.T.assign((size_t)B * B * B, 0.0);
  std::vector<double> seed(B);
  for (int i = 0; i < B; ++i)
    seed[i] = (double)(sqrtl(2.0L / (sqrtl(kPiL) / 2.0L)) * expl(-0.5L * (long double)out.t[i]));
  for (int l = 0; l < B; ++l) {
    if (l > 0)
      for (int i = 0; i < B; ++i) seed[i] *= out.r[i] / sqrt(l + 0.5);
    for (int i = 0; i < B; ++i) {
      double prev = 0.0, cur = seed[i];
      const double t = out.t[i];
      out.T[((size_t)l * B + l) * B + i] = cur;  // n = l + 1
      for (int n = l + 1; n < B; ++n) {
        double a = (2.0 * n - l - 0.5 - t) / sqrt((n + 0.5) * (n - l));
        double c = sqrt((n - 0.5) / (n + 0.5) * (double)(n - l - 1) / (double)(n - l));
        double nxt = a * cur - c * prev;
        prev = cur;
        cur = nxt;
        out.T[((size_t)l * B + n) * B + i] = cur;  // degree n + 1
      }
    }
  }

  // radial weights: reciprocal Christoffel function of the l = 0 column
  out.what.resize(B);
  for (int i = 0; i < B; ++i) {
    long double s = 0.0L;
    for (int n = 0; n < B; ++n) {
      long double v = out.T[((size_t)0 * B + n) * B + i];
      s += v * v;
    }
    out.what[i] = (double)(1.0L / s);
    if (!(out.what[i] > 0.0) || !isfinite(out.what[i])) {
      msg = "radial weight not finite";
      return false;
    }
  }

  // sphere rule, Thm 3.1 (order L = B) with the azimuthal factor pi/B
  out.theta.resize(2 * B);
  out.phi.resize(2 * B);
  out.beta.resize(2 * B);
  for (int j = 0; j < 2 * B; ++j) {
    long double th = (2.0L * j + 1.0L) * kPiL / (4.0L * B);
    long double s = 0.0L;
    for (int l = 0; l < B; ++l)
      s += sinl((2.0L * j + 1.0L) * (2.0L * l + 1.0L) * kPiL / (4.0L * B)) / (2.0L * l + 1.0L);
    long double b = sinl(th) * (2.0L / B) * s;
    out.theta[j] = (double)th;
    out.phi[j] = (double)(j * kPiL / B);
    out.beta[j] = (double)(kPiL / B * b);
  }

  // Legendre functions on the half grid j' < B
  out.lam.assign((size_t)B * B * B, 0.0);
  for (int j = 0; j < B; ++j) {
    const long double th = (2.0L * j + 1.0L) * kPiL / (4.0L * B);
    const double x = (double)cosl(th);
    const double sn = (double)sinl(th);
    double sect = 1.0 / sqrt(4.0 * (double)kPiL);  // Lambda_00
    for (int m = 0; m < B; ++m) {
      if (m > 0) sect *= -sqrt((2.0 * m + 1.0) / (2.0 * m)) * sn;
      double pm2 = 0.0, pm1 = sect;
      out.lam[((size_t)m * B + m) * B + j] = sect;
      for (int l = m + 1; l < B; ++l) {
        // Lambda_{l,m} from Lambda_{l-1,m}, Lambda_{l-2,m}
        double a = sqrt((4.0 * l * l - 1.0) / ((double)(l - m) * (l + m)));
        double c = sqrt(((l - 1.0) * (l - 1.0) - (double)m * m) / (4.0 * (l - 1.0) * (l - 1.0) - 1.0));
        double v = a * (x * pm1 - c * pm2);
        pm2 = pm1;
        pm1 = v;
        out.lam[((size_t)m * B + l) * B + j] = v;
      }
    }
  }
  return true;
}

}  // namespace sgl
