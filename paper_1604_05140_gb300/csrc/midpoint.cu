// Midpoint-rule SGL coefficients on a Cartesian grid (sgl_midpoint).
//
// The paper's Discussion describes the current practice this transform is
// meant to replace: sample f on a regular Cartesian grid and approximate each
// coefficient by the midpoint rule.  The inner product it approximates is
// Eq. (inner_product), <f, H_nlm> = int f conj(H_nlm) exp(-|x|^2) dx, so
//   fhat_nlm ~= sum_k f(x_k) conj(H_nlm(x_k)) exp(-|x_k|^2) dV,
// x_k the midpoints of the M^3 cells of [-L, L]^3, dV = (2L/M)^3.  No
// sampling theorem makes this exact; it is built for the accuracy / cost
// comparison with the SGL transform.
//
// Per block: a slice of the grid points, a group of coefficients and up to
// kFn functions.  Threads first build, for a batch of kPts points, the
// normalized Legendre functions Lambda_lm(cos theta) (Def 2.1, normalized
// Eq. legendre_recurrence), the radial functions T_nl(r) = N_nl R_nl(r)
// exp(-r^2/2) (Lemma 3.7, normalized reading), e^{-i m phi} and the weighted
// samples of the block's functions in shared memory; then each thread
// accumulates a fixed set of coefficients of every one of those functions over
// the points (the basis value of a (point, coefficient) pair is formed once and
// used for all kFn functions), and finally adds its partial sums to the output
// (one atomic add per coefficient, function and block).
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include <string>

#include "sgl_internal.h"

namespace sgl {

void set_global_error(const std::string& msg);  // api.cu: message of sgl_last_error(NULL)

namespace {

constexpr int kPts = 16;          // points per shared-memory batch
constexpr int kThreads = 256;
constexpr int kPer = 2;           // coefficients per thread
constexpr int kFn = 8;            // functions per block (grid y: groups of kFn)
constexpr int kCoefBlock = kPer * kThreads;  // coefficients per block (grid z)

sgl_status midpoint_fail(sgl_status st, const std::string& msg) {
  set_global_error(msg);
  return st;
}

template <typename real>
struct MidArgs {
  const real* f;       // [batch][M^3] complex (re, im)
  real* out;           // [batch][Omega] complex, accumulated
  int B, M, batch;
  int64_t omega;
  int64_t pts_per_block;
  double L;
};

template <typename real>
__global__ void __launch_bounds__(kThreads, 2) midpoint_kernel(MidArgs<real> a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int B = a.B;
  const int nlm = B * (B + 1) / 2;  // entries of one triangular table
  real* lam = reinterpret_cast<real*>(smem_raw);      // [kPts][m][l >= m]: index m*B - m(m-1)/2 + (l - m)
  real* rad = lam + kPts * nlm;                       // [kPts][l][n-1 >= l]: index l*B - l(l-1)/2 + (n-1-l)
  real* eph = rad + kPts * nlm;                       // [kPts][m < B][2]: e^{-i m phi}
  real* fw = eph + kPts * 2 * B;                      // [kPts][kFn][2]: f_j(x_k) exp(-|x_k|^2 / 2) dV
  // recurrence coefficients, once per block (no square roots or divisions in
  // the per-point loops): Legendre a, c at [m][l]; radial 1/s, (2n-l-1/2)/s
  // and c at [l][n-1]; sectoral and radial seed factors per m and per l
  real* la = fw + 2 * kPts * kFn;
  real* lc = la + nlm;
  real* rs = lc + nlm;
  real* r0 = rs + nlm;
  real* rc = r0 + nlm;
  real* sf = rc + nlm;    // [m]: -sqrt((2m+1)/(2m)), m >= 1
  real* rf = sf + B;      // [l]: 1/sqrt(l + 1/2), l >= 1
  for (int w = threadIdx.x; w < nlm; w += blockDim.x) {
    int m = 0;
    while ((m + 1) * B - (m + 1) * m / 2 <= w) ++m;  // row m of the [m][l >= m] triangle
    const int l = m + (w - (m * B - m * (m - 1) / 2));
    la[w] = l > m ? sqrt((4 * (real)l * l - 1) / ((real)(l - m) * (l + m))) : 0;
    lc[w] = l > m + 1 ? sqrt(((l - 1) * (real)(l - 1) - (real)m * m) / (4 * (real)(l - 1) * (l - 1) - 1)) : 0;
    // the same triangle read as [l][n-1 >= l]: row l = m, n - 1 = l_index
    const int ll = m, n = l;  // degree n + 1 of T, recurrence from n
    if (n > ll) {
      const real inv = 1 / sqrt((n + (real)0.5) * (n - ll));
      rs[w] = inv;
      r0[w] = (2 * (real)n - ll - (real)0.5) * inv;
      rc[w] = sqrt((n - (real)0.5) / (n + (real)0.5) * (real)(n - ll - 1) / (real)(n - ll));
    } else {
      rs[w] = r0[w] = rc[w] = 0;
    }
  }
  for (int w = threadIdx.x; w < B; w += blockDim.x) {
    sf[w] = w > 0 ? -sqrt((2 * w + 1) / (real)(2 * w)) : 0;
    rf[w] = w > 0 ? 1 / sqrt(w + (real)0.5) : 0;
  }
  const int b0 = blockIdx.y * kFn;  // first function of the block
  const int nfb = a.batch - b0 < kFn ? a.batch - b0 : kFn;
  const int64_t M3 = (int64_t)a.M * a.M * a.M;
  const int64_t p0 = (int64_t)blockIdx.x * a.pts_per_block;
  const int64_t p1 = p0 + a.pts_per_block < M3 ? p0 + a.pts_per_block : M3;
  const double h = 2.0 * a.L / a.M;
  const real dV = (real)(h * h * h);
  const real kPi = (real)3.14159265358979323846;
  // coefficients of this thread: omega = blockIdx.z * kCoefBlock + threadIdx.x + q * kThreads,
  // with their (n, l, m) decoded once: table offsets, |m|, sign and sign of m
  real acc_re[kPer][kFn], acc_im[kPer][kFn];
  int li[kPer], ri[kPer], amq[kPer], neg[kPer];
  real sgnq[kPer];
#pragma unroll
  for (int q = 0; q < kPer; ++q) {
#pragma unroll
    for (int j = 0; j < kFn; ++j) acc_re[q][j] = acc_im[q][j] = 0;
    const int64_t om = (int64_t)blockIdx.z * kCoefBlock + threadIdx.x + (int64_t)q * kThreads;
    li[q] = -1;
    if (om >= a.omega) continue;
    // (n, l, m) of omega = n(n-1)(2n-1)/6 + l(l+1) + m
    int n = 1;
    while ((int64_t)(n + 1) * n * (2 * n + 1) / 6 <= om) ++n;
    const int e = (int)(om - (int64_t)n * (n - 1) * (2 * n - 1) / 6);
    int l = (int)sqrtf((float)e);
    while (l * l > e) --l;
    while ((l + 1) * (l + 1) <= e) ++l;
    const int m = e - l * (l + 1), am = m < 0 ? -m : m;
    sgnq[q] = (m < 0 && (am & 1)) ? (real)-1 : (real)1;  // Lambda_{l,-m} = (-1)^m Lambda_lm
    li[q] = am * B - am * (am - 1) / 2 + (l - am);
    ri[q] = l * B - l * (l - 1) / 2 + (n - 1 - l);
    amq[q] = am;
    neg[q] = m < 0;
  }

  for (int64_t pb = p0; pb < p1; pb += kPts) {
    const int np = (int)(p1 - pb < kPts ? p1 - pb : kPts);
    __syncthreads();
    // per point: coordinates, weight, e^{-i m phi}; per (point, m): Legendre
    // column; per (point, l): radial column
    for (int w = threadIdx.x; w < kPts * B; w += blockDim.x) {
      const int k = w / B, m = w - k * B;
      if (k >= np) continue;
      const int64_t p = pb + k;
      const int ix = (int)(p / ((int64_t)a.M * a.M)), iy = (int)((p / a.M) % a.M), iz = (int)(p % a.M);
      const real x = (real)(-a.L + (ix + 0.5) * h), y = (real)(-a.L + (iy + 0.5) * h), z = (real)(-a.L + (iz + 0.5) * h);
      const real rho2 = x * x + y * y, t = rho2 + z * z, r = sqrt(t);
      const real rho = sqrt(rho2);
      const real ct = r > 0 ? z / r : (real)1, st = r > 0 ? rho / r : (real)0;
      // e^{-i m phi} as the m-th power of (x - i y) / rho (phi = 0 on the z axis)
      {
        const real c1 = rho > 0 ? x / rho : (real)1, s1 = rho > 0 ? -y / rho : (real)0;
        real c = 1, sn = 0;
        for (int mm = 0; mm < m; ++mm) {
          const real cn = c * c1 - sn * s1;
          sn = c * s1 + sn * c1;
          c = cn;
        }
        eph[(k * B + m) * 2] = c;
        eph[(k * B + m) * 2 + 1] = sn;
      }
      // weight exp(-|x|^2) dV, of which T_nl carries exp(-|x|^2 / 2): work
      // item (k, m) weights the samples of functions j = m, m + B, .. (zero
      // past the batch)
      const real e2 = exp(-t / 2);
      for (int j = m; j < kFn; j += B) {
        real fr = 0, fi = 0;
        if (j < nfb) {
          const int64_t fo = ((int64_t)(b0 + j) * M3 + p) * 2;
          fr = a.f[fo] * e2 * dV;
          fi = a.f[fo + 1] * e2 * dV;
        }
        fw[(k * kFn + j) * 2] = fr;
        fw[(k * kFn + j) * 2 + 1] = fi;
      }
      const int tri = m * B - m * (m - 1) / 2;  // row m (or l = m) of a triangle
      // Lambda_lm(theta), l = m .. B-1: sectoral seed, then the recurrence in l
      real sect = (real)(1.0 / sqrt(4.0 * 3.14159265358979323846));
      for (int mm = 1; mm <= m; ++mm) sect *= sf[mm] * st;
      real* lm = lam + k * nlm + tri;
      real pm2 = 0, pm1 = sect;
      lm[0] = sect;
      for (int l = m + 1; l < B; ++l) {
        const real v = la[tri + l - m] * (ct * pm1 - lc[tri + l - m] * pm2);
        pm2 = pm1;
        pm1 = v;
        lm[l - m] = v;
      }
      // T_nl(r), n = l+1 .. B, for l = m (one column per thread)
      {
        const int l = m;
        real seed = sqrt((real)2 / (sqrt(kPi) / 2)) * e2;
        for (int ll = 1; ll <= l; ++ll) seed *= r * rf[ll];
        real* rl = rad + k * nlm + tri;
        real prev = 0, cur = seed;
        rl[0] = cur;
        for (int n = l + 1; n < B; ++n) {
          const int w = tri + n - l;
          const real nxt = (r0[w] - t * rs[w]) * cur - rc[w] * prev;
          prev = cur;
          cur = nxt;
          rl[n - l] = cur;
        }
      }
    }
    __syncthreads();
    // accumulate: coefficient omega(n, l, m) of function j += f_j w
    // conj(T_nl Lambda_l|m| s_m e^{i m phi}); the sign s_m is applied to the
    // sums at the end
    for (int k = 0; k < np; ++k) {
      real fr[kFn], fi[kFn];
#pragma unroll
      for (int j = 0; j < kFn; ++j) {
        fr[j] = fw[(k * kFn + j) * 2];
        fi[j] = fw[(k * kFn + j) * 2 + 1];
      }
#pragma unroll
      for (int q = 0; q < kPer; ++q) {
        if (li[q] < 0) continue;
        const real amp = lam[k * nlm + li[q]] * rad[k * nlm + ri[q]];
        // e^{-i m phi}: the table for m >= 0, its conjugate for m < 0
        const real ec = eph[(k * B + amq[q]) * 2];
        const real es = neg[q] ? -eph[(k * B + amq[q]) * 2 + 1] : eph[(k * B + amq[q]) * 2 + 1];
        const real hr = amp * ec, hi = amp * es;
        // four multiply-adds per function (written out: acc += (a - b) would
        // round a - b first and cost a third instruction)
#pragma unroll
        for (int j = 0; j < kFn; ++j) {
          acc_re[q][j] = fma(fr[j], hr, acc_re[q][j]);
          acc_re[q][j] = fma(-fi[j], hi, acc_re[q][j]);
          acc_im[q][j] = fma(fr[j], hi, acc_im[q][j]);
          acc_im[q][j] = fma(fi[j], hr, acc_im[q][j]);
        }
      }
    }
  }
#pragma unroll
  for (int q = 0; q < kPer; ++q) {
    if (li[q] < 0) continue;
    const int64_t om = (int64_t)blockIdx.z * kCoefBlock + threadIdx.x + (int64_t)q * kThreads;
#pragma unroll
    for (int j = 0; j < kFn; ++j) {
      if (j >= nfb) break;
      atomicAdd(&a.out[((int64_t)(b0 + j) * a.omega + om) * 2], sgnq[q] * acc_re[q][j]);
      atomicAdd(&a.out[((int64_t)(b0 + j) * a.omega + om) * 2 + 1], sgnq[q] * acc_im[q][j]);
    }
  }
}

template <typename real>
cudaError_t launch_midpoint(int B, int M, double L, int batch, const void* f, void* coeffs, cudaStream_t s) {
  MidArgs<real> a;
  a.f = (const real*)f;
  a.out = (real*)coeffs;
  a.B = B;
  a.M = M;
  a.batch = batch;
  a.omega = coeff_count(B);
  a.L = L;
  const int64_t M3 = (int64_t)M * M * M;
  const int64_t groups = (a.omega + kCoefBlock - 1) / kCoefBlock;
  // about four blocks per SM over the function and coefficient groups, at
  // least kPts points each
  const int64_t fgroups = (batch + kFn - 1) / kFn;
  int64_t blocks = (4 * 152 + fgroups * groups - 1) / (fgroups * groups);
  if (blocks < 1) blocks = 1;
  a.pts_per_block = (M3 + blocks - 1) / blocks;
  if (a.pts_per_block < kPts) a.pts_per_block = kPts;
  const int64_t nbx = (M3 + a.pts_per_block - 1) / a.pts_per_block;
  const size_t nlm = (size_t)B * (B + 1) / 2;
  const size_t smem = sizeof(real) * (2 * kPts * nlm + (size_t)kPts * 2 * B + 2 * kPts * kFn + 5 * nlm + 2 * (size_t)B);
  cudaError_t e = cudaMemsetAsync(coeffs, 0, (size_t)batch * a.omega * 2 * sizeof(real), s);
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(midpoint_kernel<real>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  midpoint_kernel<real><<<dim3((unsigned)nbx, (unsigned)fgroups, (unsigned)groups), kThreads, smem, s>>>(a);
  return cudaGetLastError();
}

}  // namespace

}  // namespace sgl

extern "C" sgl_status sgl_midpoint(int B, int M, double L, int batch, int prec, const void* f, void* coeffs,
                                   sgl_stream_t stream) {
  using namespace sgl;
  if (B < 1 || B > 32) return midpoint_fail(SGL_ERR_UNSUPPORTED, "sgl_midpoint accepts bandlimits 1..32");
  if (M < 1 || M > 1024 || batch < 1 || batch > 65535 || !(L > 0.0))
    return midpoint_fail(SGL_ERR_ARG, "sgl_midpoint: M in 1..1024, batch in 1..65535, L > 0");
  if (prec != SGL_FP64 && prec != SGL_FP32) return midpoint_fail(SGL_ERR_ARG, "sgl_midpoint: SGL_FP64 or SGL_FP32");
  if (!f || !coeffs) return midpoint_fail(SGL_ERR_ARG, "null data pointer");
  const size_t cb = prec == SGL_FP64 ? 16 : 8;
  cudaPointerAttributes at;
  for (const void* p : {f, (const void*)coeffs}) {
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess || at.type != cudaMemoryTypeDevice) {
      cudaGetLastError();
      return midpoint_fail(SGL_ERR_ARG, "sgl_midpoint takes device pointers");
    }
    if ((uintptr_t)p % cb) return midpoint_fail(SGL_ERR_ARG, "data pointers must be aligned to the complex element size");
  }
  const cudaError_t e = prec == SGL_FP64
                            ? launch_midpoint<double>(B, M, L, batch, f, coeffs, (cudaStream_t)stream)
                            : launch_midpoint<float>(B, M, L, batch, f, coeffs, (cudaStream_t)stream);
  if (e != cudaSuccess) return midpoint_fail(SGL_ERR_CUDA, std::string("sgl_midpoint launch: ") + cudaGetErrorString(e));
  return SGL_OK;
}
