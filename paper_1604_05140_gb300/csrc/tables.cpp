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
// On the paper's own grid (SGL_GRID_HALF_RANGE_HERMITE) the radii are the 2B
// nodes r_i of the half-range Gauss-Hermite rule of order 2B (Thm 3.3) and the
// radial quadrature weight is a_i r_i^2 (Eq. zwischenstufe_2), so
// what_i = a_i r_i^2 exp(r_i^2).  The rule comes from the discretized
// Stieltjes procedure in long double: the weight exp(-r^2) on [0, sqrt(4N) + 10]
// is replaced by composite 20-point Gauss-Legendre panels of width 1/32 in
// u = sqrt(r) (its mass beyond is below exp(-1000)), the monic recurrence coefficients of the
// orthogonal polynomials follow from discrete inner products, the nodes are the
// eigenvalues of the Jacobi matrix (Sturm bisection, then Newton steps on the
// recurrence) and the weights the reciprocal Christoffel function of the
// orthonormal polynomials.
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

// Gauss-Legendre nodes and weights of order q on [-1, 1] (Newton on the
// Legendre recurrence).
void gauss_legendre(int q, std::vector<long double>& x, std::vector<long double>& w) {
  x.resize(q);
  w.resize(q);
  for (int i = 0; i < q; ++i) {
    long double z = cosl(kPiL * (i + 0.75L) / (q + 0.5L));
    long double dp = 1.0L;
    for (int it = 0; it < 100; ++it) {
      long double p0 = 1.0L, p1 = z;
      for (int k = 2; k <= q; ++k) {
        const long double p2 = ((2.0L * k - 1.0L) * z * p1 - (k - 1.0L) * p0) / k;
        p0 = p1;
        p1 = p2;
      }
      dp = q * (z * p1 - p0) / (z * z - 1.0L);
      const long double step = p1 / dp;
      z -= step;
      if (fabsl(step) < 1e-30L) break;
    }
    x[i] = z;
    w[i] = 2.0L / ((1.0L - z * z) * dp * dp);
  }
}

// Half-range Gauss-Hermite rule of order N (Thm 3.3): nodes r_i and weights
// a_i, by the discretized Stieltjes procedure (see the file header).
bool half_range_hermite(int N, std::vector<long double>& r, std::vector<long double>& a, std::string& msg) {
  // discretize in u = sqrt(r): int p(r) e^{-r^2} dr = int p(u^2) e^{-u^4} 2u du;
  // the zeros of the orthogonal polynomials, which crowd towards r = 0, are
  // nearly evenly spaced in u (0.017 .. 0.045 apart at N = 256)
  std::vector<long double> gx, gw;
  gauss_legendre(20, gx, gw);
  const long double umax = sqrtl(sqrtl(4.0L * N) + 10.0L), h = 1.0L / 32.0L;
  const int panels = (int)ceill(umax / h);
  std::vector<long double> xs, ws;
  for (int p = 0; p < panels; ++p)
    for (int q = 0; q < 20; ++q) {
      const long double u = h * (p + 0.5L * (gx[q] + 1.0L));
      xs.push_back(u * u);
      ws.push_back(0.5L * h * gw[q] * 2.0L * u * expl(-u * u * u * u));
    }
  const size_t M = xs.size();
  std::vector<long double> al(N), be(N), pm(M, 0.0L), p(M, 1.0L), pn(M);
  long double nprev = 1.0L;
  for (int k = 0; k < N; ++k) {
    long double nk = 0.0L, xk = 0.0L;
    for (size_t s = 0; s < M; ++s) {
      const long double v = ws[s] * p[s] * p[s];
      nk += v;
      xk += v * xs[s];
    }
    al[k] = xk / nk;
    be[k] = k == 0 ? nk : nk / nprev;
    nprev = nk;
    for (size_t s = 0; s < M; ++s) pn[s] = (xs[s] - al[k]) * p[s] - (k > 0 ? be[k] : 0.0L) * pm[s];
    pm.swap(p);
    p.swap(pn);
  }
  // nodes: eigenvalues of the Jacobi matrix, Sturm bisection then Newton
  std::vector<double> d(N), e2(N, 0.0);
  double hi = 0.0;
  for (int k = 0; k < N; ++k) {
    d[k] = (double)al[k];
    if (k > 0) e2[k] = (double)be[k];
  }
  for (int k = 0; k < N; ++k)
    hi = std::max(hi, d[k] + (k > 0 ? sqrt(e2[k]) : 0.0) + (k + 1 < N ? sqrt(e2[k + 1]) : 0.0));
  r.assign(N, 0.0L);
  a.assign(N, 0.0L);
  for (int i = 0; i < N; ++i) {
    double lo = 0.0, up = hi;
    for (int it = 0; it < 200 && up - lo > 1e-15 * std::max(1.0, up); ++it) {
      const double mid = 0.5 * (lo + up);
      if (sturm_count(d, e2, mid) > i) up = mid; else lo = mid;
    }
    long double x = 0.5L * ((long double)lo + (long double)up);
    for (int it = 0; it < 8; ++it) {  // Newton on the monic p_N
      long double q0 = 0.0L, q1 = 1.0L, dq0 = 0.0L, dq1 = 0.0L;
      for (int k = 0; k < N; ++k) {
        const long double bk = k > 0 ? be[k] : 0.0L;
        const long double q2 = (x - al[k]) * q1 - bk * q0;
        const long double dq2 = q1 + (x - al[k]) * dq1 - bk * dq0;
        q0 = q1;
        q1 = q2;
        dq0 = dq1;
        dq1 = dq2;
      }
      if (dq1 == 0.0L) break;
      const long double step = q1 / dq1;
      x -= step;
      if (fabsl(step) <= 1e-19L * fabsl(x)) break;
    }
    // Christoffel function of the orthonormal polynomials
    long double o0 = 0.0L, o1 = 1.0L / sqrtl(be[0]), sum = o1 * o1;
    for (int k = 0; k + 1 < N; ++k) {
      const long double o2 = ((x - al[k]) * o1 - (k > 0 ? sqrtl(be[k]) : 0.0L) * o0) / sqrtl(be[k + 1]);
      o0 = o1;
      o1 = o2;
      sum += o1 * o1;
    }
    r[i] = x;
    a[i] = 1.0L / sum;
    if (!(x > 0.0L) || !(a[i] > 0.0L) || !isfinite((double)x) || (i > 0 && !(r[i] > r[i - 1]))) {
      msg = "half-range Gauss-Hermite rule failed";
      return false;
    }
  }
  return true;
}

}  // namespace

bool build_tables(int B, int grid, HostTables& out, std::string& msg) {
  if (!bandlimit_supported(B)) {
    msg = "unsupported bandlimit";
    return false;
  }
  out.B = B;
  const bool hermite = grid == SGL_GRID_HALF_RANGE_HERMITE;
  const int R = hermite ? 2 * B : B;
  out.R = R;
  std::vector<long double> hr, ha;  // half-range Gauss-Hermite nodes and weights
  if (hermite) {
    if (!half_range_hermite(R, hr, ha, msg)) return false;
    out.t.resize(R);
    for (int i = 0; i < R; ++i) out.t[i] = (double)(hr[i] * hr[i]);
  } else if (!radial_nodes(B, out.t, msg)) {
    return false;
  }
  out.r.resize(R);
  for (int i = 0; i < R; ++i) out.r[i] = hermite ? (double)hr[i] : sqrt(out.t[i]);

  // radial functions, Lemma 3.7 (normalized reading), at the R radii
  out.T.assign((size_t)B * B * R, 0.0);
  std::vector<double> seed(R);
  for (int i = 0; i < R; ++i)
    seed[i] = (double)(sqrtl(2.0L / (sqrtl(kPiL) / 2.0L)) * expl(-0.5L * (long double)out.t[i]));
  for (int l = 0; l < B; ++l) {
    if (l > 0)
      for (int i = 0; i < R; ++i) seed[i] *= out.r[i] / sqrt(l + 0.5);
    for (int i = 0; i < R; ++i) {
      double prev = 0.0, cur = seed[i];
      const double t = out.t[i];
      out.T[((size_t)l * B + l) * R + i] = cur;  // n = l + 1
      for (int n = l + 1; n < B; ++n) {
        double a = (2.0 * n - l - 0.5 - t) / sqrt((n + 0.5) * (n - l));
        double c = sqrt((n - 0.5) / (n + 0.5) * (double)(n - l - 1) / (double)(n - l));
        double nxt = a * cur - c * prev;
        prev = cur;
        cur = nxt;
        out.T[((size_t)l * B + n) * R + i] = cur;  // degree n + 1
      }
    }
  }

  // radial weights: on the Laguerre grid the reciprocal Christoffel function
  // of the l = 0 column; on the paper's grid a_i r_i^2 exp(r_i^2)
  out.what.resize(R);
  for (int i = 0; i < R; ++i) {
    if (hermite) {
      out.what[i] = (double)(ha[i] * hr[i] * hr[i] * expl(hr[i] * hr[i]));
    } else {
      long double s = 0.0L;
      for (int n = 0; n < B; ++n) {
        long double v = out.T[((size_t)0 * B + n) * R + i];
        s += v * v;
      }
      out.what[i] = (double)(1.0L / s);
    }
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

  // cosine coefficients for the seminaive Legendre transform (Eq. dct_trick):
  // on the half grid j' < B, Q = Lambda_lm / w_m expands in cos(2k' theta)
  // (even l - m, a DCT-II of length B inverts it) or cos((2k'+1) theta) (odd
  // l - m, a DCT-IV); only k' up to half the degree (l, or l - 1 for odd m)
  // can be non-zero, and the rest is set to zero
  out.lcos.assign((size_t)B * B * B, 0.0);
  std::vector<double> q(B), cs2((size_t)B * B), cs4((size_t)B * B), snt(B);
  for (int j = 0; j < B; ++j) snt[j] = (double)sinl((2.0L * j + 1.0L) * kPiL / (4.0L * B));
  for (int k = 0; k < B; ++k)
    for (int j = 0; j < B; ++j) {
      cs2[(size_t)k * B + j] = (double)cosl((long double)k * (2.0L * j + 1.0L) * kPiL / (2.0L * B));
      cs4[(size_t)k * B + j] = (double)cosl((2.0L * k + 1.0L) * (2.0L * j + 1.0L) * kPiL / (4.0L * B));
    }
  for (int m = 0; m < B; ++m)
    for (int l = m; l < B; ++l) {
      const bool odd_p = (l - m) & 1;
      const int deg = (m & 1) ? l - 1 : l;
      const int kmax = odd_p ? (deg - 1) / 2 : deg / 2;
      for (int j = 0; j < B; ++j) q[j] = out.lam[((size_t)m * B + l) * B + j] / ((m & 1) ? snt[j] : 1.0);
      for (int k = 0; k <= kmax && k < B; ++k) {
        const double* cs = (odd_p ? cs4.data() : cs2.data()) + (size_t)k * B;
        long double acc = 0.0L;
        for (int j = 0; j < B; ++j) acc += (long double)q[j] * cs[j];
        double v = (double)(acc * 2.0L / B);
        if (!odd_p && k == 0) v *= 0.5;
        out.lcos[((size_t)m * B + l) * B + k] = v;
      }
    }
  return true;
}

}  // namespace sgl
