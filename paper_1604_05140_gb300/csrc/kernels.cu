// CUDA kernels of the SGL transform for sm_103a: the phi-FFT of every ring
// and the Legendre / radial contractions on the CUDA cores (FP64 and FP32).
//
// Forward (Algorithm 3):
//   fft_fwd   G[i][j][m] = sum_k ftil[i][j][k] e^{-i m phi_k}     (Eq. SFFT_rearranged, inner sum)
//             written as E = G_j + G_{2B-1-j}, O = G_j - G_{2B-1-j}, j < B,
//             using Lambda_lm(pi - theta) = (-1)^{l+m} Lambda_lm(theta)
//   gemm<LEG_F> S[l][m][i] = sum_j' beta_j' Lambda_lm(theta_j') {E|O}[m][j'][i]  (Eq. DLT)
//   gemm<RAD_F> fhat[n,l,m] = sum_i what_i T_nl(i) S[l][m][i]                  (Eq. DRT_matrix)
// Inverse (Algorithm 4): gemm<RAD_I> (iDRT, R_l^T), gemm<LEG_I> (Legendre
// synthesis, Eq. iSFFT_rearranged inner sum), fft_inv (inverse phi-FFT).
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>

#include "sgl_internal.h"

namespace sgl {

// ---------------------------------------------------------------------------
// complex helpers
// ---------------------------------------------------------------------------
template <typename real>
// aligned as a whole value, so that loads and stores move (re, im) at once
struct alignas(2 * sizeof(real)) cx {
  real x, y;
};

template <typename real>
__device__ __forceinline__ cx<real> cadd(cx<real> a, cx<real> b) { return {a.x + b.x, a.y + b.y}; }
template <typename real>
__device__ __forceinline__ cx<real> csub(cx<real> a, cx<real> b) { return {a.x - b.x, a.y - b.y}; }
template <typename real>
__device__ __forceinline__ cx<real> cmul(cx<real> a, cx<real> b) {
  return {a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x};
}

// twiddle e^{-2 pi i k/N} (INV: conjugate) from a table of N entries
template <typename real, bool INV>
__device__ __forceinline__ cx<real> tw(const real* __restrict__ wre, const real* __restrict__ wim, int k) {
  return {wre[k], INV ? -wim[k] : wim[k]};
}

// In-register radix-2 DIT FFT of compile-time size N (power of two <= 16);
// input and output in natural order.  Twiddle of size-len stage index q:
// W_N_total^{q * (N_total/len)} = table[q * wstep * (N/len)].
template <typename real, int N, bool INV>
__device__ __forceinline__ void fft_reg(cx<real>* v, const real* wre, const real* wim, int wstep) {
  if constexpr (N > 1) {
    constexpr int LOG = (N == 2) ? 1 : (N == 4) ? 2 : (N == 8) ? 3 : 4;
#pragma unroll
    for (int i = 0; i < N; ++i) {
      int j = 0;
#pragma unroll
      for (int b = 0; b < LOG; ++b) j |= ((i >> b) & 1) << (LOG - 1 - b);
      if (i < j) {
        cx<real> t = v[i];
        v[i] = v[j];
        v[j] = t;
      }
    }
#pragma unroll
    for (int len = 2; len <= N; len <<= 1) {
      const int half = len >> 1;
#pragma unroll
      for (int start = 0; start < N; start += len) {
#pragma unroll
        for (int q = 0; q < half; ++q) {
          cx<real> w = tw<real, INV>(wre, wim, q * (N / len) * wstep);
          cx<real> a = v[start + q];
          cx<real> b = cmul(v[start + q + half], w);
          v[start + q] = cadd(a, b);
          v[start + q + half] = csub(a, b);
        }
      }
    }
  }
}

// Direct DFT of runtime size n <= 16 (any n), input u, output v.
template <typename real, bool INV>
__device__ __forceinline__ void dft_reg(const cx<real>* u, cx<real>* v, int n, const real* wre,
                                        const real* wim, int wstep) {
#pragma unroll
  for (int k = 0; k < 16; ++k) {
    if (k < n) {
      cx<real> acc = {0, 0};
#pragma unroll
      for (int q = 0; q < 16; ++q) {
        if (q < n) {
          int idx = (q * k) % n;
          cx<real> w = tw<real, INV>(wre, wim, idx * wstep);
          cx<real> p = cmul(u[q], w);
          acc = cadd(acc, p);
        }
      }
      v[k] = acc;
    }
  }
}

// ---------------------------------------------------------------------------
// phi-FFT kernels
// ---------------------------------------------------------------------------
// Shared memory per CTA: R = 2*JP rings, each stored as separate real and
// imaginary planes of n1 rows x (n2+1) columns (padded), ring pitch odd.
struct FftArgs {
  const SegDesc* segs;
  const int64_t* fn_samp;
  const int4* ctas;      // (seg, shell, j0, 0)
  const void* tab;       // misc tables in the real type
  const void* in;
  void* out;
  void* w1;
  int JP;                // ring pairs per CTA
  int mode;              // fwd: 0 none, 1 *exp(-t/2), 2 *exp(+t/2);
                         // inv: 0 none, 1 *exp(+t/2), 2 *what*beta, 3 *what*beta*exp(-t/2)
  int64_t pair_limit;    // real functions in pairs: reals in the sample array; 0 complex samples
  unsigned* amax;        // forward, FP16x3 plans: per-function largest |E/O| (else null)
  int64_t pair_gap;      // real functions in pairs: reals from the pair's first function to its second
};

__host__ __device__ inline int ring_pitch(int n1, int n2) {
  int p = n1 * (n2 + 1);
  return (p % 2 == 0) ? p + 1 : p;
}

template <typename real, int N1, int N2C, bool INV>
__device__ __forceinline__ void fft_rings(real* sre, real* sim, const real* wre, const real* wim, int R, int n2,
                                          int N, int pitch) {
  const int n1 = N1;
  const int n2p = n2 + 1;
  // step A: N1-point DFT over n1 for every (ring, n2), then twiddle W_N^{n2 k1}
  for (int w = threadIdx.x; w < R * n2; w += blockDim.x) {
    const int r = w / n2, c2 = w - r * n2;
    real* pr = sre + r * pitch + c2;
    real* pi = sim + r * pitch + c2;
    cx<real> v[N1];
#pragma unroll
    for (int a = 0; a < N1; ++a) v[a] = {pr[a * n2p], pi[a * n2p]};
    fft_reg<real, N1, INV>(v, wre, wim, N / N1);
#pragma unroll
    for (int a = 1; a < N1; ++a) v[a] = cmul(v[a], tw<real, INV>(wre, wim, c2 * a));
#pragma unroll
    for (int a = 0; a < N1; ++a) {
      pr[a * n2p] = v[a].x;
      pi[a * n2p] = v[a].y;
    }
  }
  __syncthreads();
  // step B: n2-point DFT over n2 for every (ring, k1)
  for (int w = threadIdx.x; w < R * n1; w += blockDim.x) {
    const int r = w / n1, k1 = w - r * n1;
    real* pr = sre + r * pitch + k1 * n2p;
    real* pi = sim + r * pitch + k1 * n2p;
    if constexpr (N2C > 0) {
      cx<real> v[N2C];
#pragma unroll
      for (int a = 0; a < N2C; ++a) v[a] = {pr[a], pi[a]};
      fft_reg<real, N2C, INV>(v, wre, wim, N / N2C);
#pragma unroll
      for (int a = 0; a < N2C; ++a) {
        pr[a] = v[a].x;
        pi[a] = v[a].y;
      }
    } else {
      cx<real> u[16], v[16];
#pragma unroll
      for (int a = 0; a < 16; ++a)
        if (a < n2) u[a] = {pr[a], pi[a]};
      dft_reg<real, INV>(u, v, n2, wre, wim, N / n2);
#pragma unroll
      for (int a = 0; a < 16; ++a)
        if (a < n2) {
          pr[a] = v[a].x;
          pi[a] = v[a].y;
        }
    }
  }
  __syncthreads();
}

// Forward: rings j0+q and 2B-1-(j0+q) of shell (b, i) -> E/O spectra.
template <typename real, int N1, int N2C>
__global__ void __launch_bounds__(256) fft_fwd_kernel(FftArgs a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int4 cta = a.ctas[blockIdx.x];
  const SegDesc sg = a.segs[cta.x];
  const int B = sg.B, N = 2 * B, NB = sg.NB, NR = sg.R;  // NR radii
  const int n2 = sg.n2;
  const int shell = cta.y, j0 = cta.z;
  const int b = shell / NR, i = shell - b * NR;
  const int JP = min(a.JP, B - j0);
  const int R = 2 * JP;
  const int pitch = ring_pitch(N1, n2);
  real* wre = reinterpret_cast<real*>(smem_raw);
  real* wim = wre + N;
  real* sre = wim + N;
  real* sim = sre + 2 * a.JP * pitch;
  const real* misc = reinterpret_cast<const real*>(a.tab) + sg.tab_misc;
  for (int k = threadIdx.x; k < N; k += blockDim.x) {
    wre[k] = misc[3 * NR + 2 * B + 2 * k];
    wim[k] = misc[3 * NR + 2 * B + 2 * k + 1];
  }
  real scale = 1;
  if (a.mode == 1) scale = misc[NR + i];
  if (a.mode == 2) scale = misc[2 * NR + i];
  const cx<real>* in = reinterpret_cast<const cx<real>*>(a.in) + a.fn_samp[sg.fn0 + b] + (int64_t)i * N * N;
  // real functions in pairs: the pair's first function starts at twice the
  // complex offset (in reals), the second one function (pair_gap reals) later
  const real* inA = reinterpret_cast<const real*>(a.in) + 2 * a.fn_samp[sg.fn0 + b] + (int64_t)i * N * N;
  const bool hasB = 2 * a.fn_samp[sg.fn0 + b] + a.pair_gap < a.pair_limit;
  for (int e = threadIdx.x; e < R * N; e += blockDim.x) {
    const int r = e / N, k = e - r * N;
    const int q = r >> 1;
    const int j = (r & 1) ? (N - 1 - (j0 + q)) : (j0 + q);
    cx<real> v;
    if (a.pair_limit) {
      const int64_t o = (int64_t)j * N + k;
      v = {inA[o], hasB ? inA[a.pair_gap + o] : (real)0};
    } else {
      v = in[(int64_t)j * N + k];
    }
    const int c1 = k / n2, c2 = k - c1 * n2;
    sre[r * pitch + c1 * (n2 + 1) + c2] = v.x * scale;
    sim[r * pitch + c1 * (n2 + 1) + c2] = v.y * scale;
  }
  __syncthreads();
  fft_rings<real, N1, N2C, false>(sre, sim, wre, wim, R, n2, N, pitch);
  // E/O spectra for m in (-B, B): spectral index k = m mod N at slot (k % n1, k / n1)
  real* w1 = reinterpret_cast<real*>(a.w1) + sg.w1_off;
  const int total = (2 * B - 1) * 4 * JP;
  float mx = 0.f;
  for (int e = threadIdx.x; e < total; e += blockDim.x) {
    const int q = e % JP;
    const int rest = e / JP;
    const int c = rest & 1, p = (rest >> 1) & 1, m_idx = rest >> 2;
    const int m = m_idx - (B - 1);
    const int k = m >= 0 ? m : N + m;
    const int slot = (k % N1) * (n2 + 1) + k / N1;
    const real* plane = c ? sim : sre;
    const real g0 = plane[(2 * q) * pitch + slot];
    const real g1 = plane[(2 * q + 1) * pitch + slot];
    const real v = p ? (g0 - g1) : (g0 + g1);
    w1[(((((int64_t)m_idx * 2 + p) * NB + b) * 2 + c) * NR + i) * B + j0 + q] = v;
    mx = fmaxf(mx, fabsf((float)v));
  }
  if (a.amax) cta_amax(mx, a.amax + sg.fn0 + b);
}

// Inverse: G[m][b][c][i][j] (layout 0) or G[m][b][j][i][c] (layout 1) of
// the CTA's rings -> samples.
template <typename real, int N1, int N2C>
__global__ void __launch_bounds__(256) fft_inv_kernel(FftArgs a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int4 cta = a.ctas[blockIdx.x];
  const SegDesc sg = a.segs[cta.x];
  const int B = sg.B, N = 2 * B, NB = sg.NB, NR = sg.R;  // NR radii
  const int n2 = sg.n2;
  // cta.w selects the spectra layout (see fft16_inv_kernel): 0 -> one shell
  // i = cta.y % NR and ring pairs j0 = cta.z ...; 1 -> shells i0 = cta.y % NR ...
  // and one ring pair jp = cta.z
  const int lay = cta.w;
  const int b = cta.y / NR, i_or_i0 = cta.y - b * NR, j0 = cta.z;
  const int JP = min(a.JP, lay ? NR - i_or_i0 : B - j0);
  const int R = 2 * JP;
  const int pitch = ring_pitch(N1, n2);
  real* wre = reinterpret_cast<real*>(smem_raw);
  real* wim = wre + N;
  real* sre = wim + N;
  real* sim = sre + 2 * a.JP * pitch;
  const real* misc = reinterpret_cast<const real*>(a.tab) + sg.tab_misc;
  for (int k = threadIdx.x; k < N; k += blockDim.x) {
    wre[k] = misc[3 * NR + 2 * B + 2 * k];
    wim[k] = misc[3 * NR + 2 * B + 2 * k + 1];
  }
  // ring r (layout 0): r < JP -> j = j0 + r; r >= JP -> j = N - j0 - 2*JP + r (mirror run)
  // ring r (layout 1): shell i0 + (r mod JP), j = jp (r < JP) or N - 1 - jp
  auto ring_i = [&](int r) { return lay ? i_or_i0 + (r < JP ? r : r - JP) : i_or_i0; };
  auto ring_j = [&](int r) { return lay ? (r < JP ? j0 : N - 1 - j0) : (r < JP ? j0 + r : N - j0 - 2 * JP + r); };
  const real* g = reinterpret_cast<const real*>(a.w1) + sg.w1_off;
  // Nyquist bin (k = B) is zero
  for (int e = threadIdx.x; e < 2 * R; e += blockDim.x) {
    const int r = e >> 1;
    const int slot = (B / n2) * (n2 + 1) + (B % n2);
    ((e & 1) ? sim : sre)[r * pitch + slot] = 0;
  }
  const int total = (2 * B - 1) * 2 * R;
  for (int e = threadIdx.x; e < total; e += blockDim.x) {
    const int r = e % R;
    const int rest = e / R;
    const int c = rest & 1, m_idx = rest >> 1;
    const int m = m_idx - (B - 1);
    const int k = m >= 0 ? m : N + m;
    const int i = ring_i(r), j = ring_j(r);
    // layout 0: [m_idx][b][c][i][j]; layout 1: [m_idx][b][j][i][c]
    const real v = lay ? g[(((int64_t)m_idx * NB + b) * N + j) * (2 * NR) + 2 * i + c]
                       : g[(((int64_t)m_idx * NB + b) * 2 + c) * NR * N + (int64_t)i * N + j];
    const int c1 = k / n2, c2 = k - c1 * n2;
    (c ? sim : sre)[r * pitch + c1 * (n2 + 1) + c2] = v;
  }
  __syncthreads();
  fft_rings<real, N1, N2C, true>(sre, sim, wre, wim, R, n2, N, pitch);
  cx<real>* out = reinterpret_cast<cx<real>*>(a.out) + a.fn_samp[sg.fn0 + b];
  for (int e = threadIdx.x; e < R * N; e += blockDim.x) {
    const int r = e / N, k = e - r * N;
    const int i = ring_i(r), j = ring_j(r);
    const int slot = (k % N1) * (n2 + 1) + k / N1;
    real s = 1;
    if (a.mode == 1) s = misc[2 * NR + i];
    if (a.mode == 2) s = misc[i];
    if (a.mode == 3) s = misc[i] * misc[NR + i];
    if (a.mode >= 2) s *= misc[3 * NR + j];
    cx<real> v = {sre[r * pitch + slot] * s, sim[r * pitch + slot] * s};
    const int64_t o = ((int64_t)i * N + j) * N + k;
    if (a.pair_limit) {  // real and imaginary parts to the pair's two functions
      real* outA = reinterpret_cast<real*>(a.out) + 2 * a.fn_samp[sg.fn0 + b];
      outA[o] = v.x;
      if (2 * a.fn_samp[sg.fn0 + b] + a.pair_gap < a.pair_limit) outA[a.pair_gap + o] = v.y;
    } else {
      out[o] = v;
    }
  }
}

// ---------------------------------------------------------------------------
// SIMT GEMM stages (FP64 / FP32 on the CUDA cores)
// ---------------------------------------------------------------------------
enum Prob { LEG_F = 0, RAD_F = 1, RAD_I = 2, LEG_I = 3 };

struct GemmArgs {
  const SegDesc* segs;
  const int64_t* fn_coef;
  const int64_t* si_rows;
  const int4* tiles;
  const void* tab;
  const void* x;     // stage input (W1, W2 or coefficients)
  void* y;           // stage output
  int weighted;      // forward stages: use the weighted tables
  int seminaive;     // forward Legendre stage: x holds DCTs, table of cosine coefficients
};

constexpr int TM = 64, TN = 64, TK = 16;

__device__ __forceinline__ int64_t omega_idx(int n, int l, int m) {
  return (int64_t)n * (n - 1) * (2 * n - 1) / 6 + (int64_t)l * (l + 1) + m;
}
__device__ __forceinline__ int64_t leg_rows_before_d(int B, int m, int p) {
  int64_t rows = (int64_t)m * B - (int64_t)m * (m - 1) / 2;
  if (p == 1) rows += (m >= B) ? 0 : (B - 1 - m) / 2 + 1;
  return rows;
}
__device__ __forceinline__ int n_par_d(int B, int m, int p) {
  int first = m + p;
  return first >= B ? 0 : (B - 1 - first) / 2 + 1;
}

struct GroupCtx {
  int B, NB, R, rows, N, K, KP, KPpad;
  int xs, as;  // row strides of X (forward stages) and of the table A
  int g;       // group id within the stage
  int m, am, p, l, m_idx;
  int64_t xbase, xbase2, abase, abase2;
};

template <int PROB>
__device__ __forceinline__ void group_setup(const GemmArgs& a, const SegDesc& sg, int g, GroupCtx& c) {
  c.B = sg.B;
  c.NB = sg.NB;
  c.R = sg.R;
  c.g = g;
  const int B = sg.B, NB = sg.NB, R = sg.R;  // R radii
  if (PROB == LEG_F) {
    c.m_idx = g >> 1;
    c.p = g & 1;
    c.m = c.m_idx - (B - 1);
    c.am = c.m < 0 ? -c.m : c.m;
    c.rows = NB * 2 * R;
    c.N = n_par_d(B, c.am, c.p);
    c.K = B;
    c.xs = c.as = B;
    c.xbase = sg.w1_off + ((int64_t)c.m_idx * 2 + c.p) * NB * 2 * R * B;
    c.abase = (a.seminaive ? sg.tab_leg_s : a.weighted ? sg.tab_leg_f : sg.tab_leg_i) +
              leg_rows_before_d(B, c.am, c.p) * B;
  } else if (PROB == RAD_F) {
    c.l = g;
    c.rows = NB * (2 * c.l + 1) * 2;
    c.N = B - c.l;
    c.K = R;
    c.xs = c.as = R;
    c.xbase = sg.w2_off + (int64_t)NB * 2 * R * c.l * c.l;
    c.abase = (a.weighted ? sg.tab_rad_f : sg.tab_rad_i) + ((int64_t)c.l * B - (int64_t)c.l * (c.l - 1) / 2) * R;
  } else if (PROB == RAD_I) {
    c.l = g;
    c.rows = NB * (2 * c.l + 1) * 2;
    c.N = R;
    c.K = B - c.l;
    c.as = R;
    c.abase = sg.tab_rad_i + ((int64_t)c.l * B - (int64_t)c.l * (c.l - 1) / 2) * R;
  } else {  // LEG_I
    c.m_idx = g;
    c.m = g - (B - 1);
    c.am = c.m < 0 ? -c.m : c.m;
    c.rows = NB * 2 * R;
    c.N = B;
    c.as = B;
    c.KP = n_par_d(B, c.am, 0);
    c.KPpad = (c.KP + TK - 1) / TK * TK;
    c.K = c.KPpad + n_par_d(B, c.am, 1);
    const int64_t* sr = a.si_rows + sg.si_rows;
    c.xbase = sg.w2_off + sr[2 * c.m_idx] * (int64_t)NB * 2 * R;
    c.xbase2 = sg.w2_off + sr[2 * c.m_idx + 1] * (int64_t)NB * 2 * R;
    c.abase = sg.tab_leg_i + leg_rows_before_d(B, c.am, 0) * B;
    c.abase2 = sg.tab_leg_i + leg_rows_before_d(B, c.am, 1) * B;
  }
}

template <int PROB, typename real>
__device__ __forceinline__ real load_x(const GemmArgs& a, const SegDesc& sg, const GroupCtx& c, int row, int k) {
  const real* X = reinterpret_cast<const real*>(a.x);
  if (row >= c.rows || k >= c.K) return 0;
  if (PROB == LEG_F || PROB == RAD_F) {
    return X[c.xbase + (int64_t)row * c.xs + k];
  } else if (PROB == RAD_I) {
    const int per_b = (2 * c.l + 1) * 2;
    const int b = row / per_b;
    const int rem = row - b * per_b;
    const int mm = rem >> 1, cc = rem & 1;
    const int64_t off = a.fn_coef[sg.fn0 + b] + omega_idx(c.l + 1 + k, c.l, mm - c.l);
    return X[2 * off + cc];
  } else {
    const int64_t NB2R = (int64_t)c.NB * 2 * c.R;  // one l' row of S_i
    if (k < c.KPpad) {
      if (k >= c.KP) return 0;
      return X[c.xbase + k * NB2R + row];
    }
    return X[c.xbase2 + (k - c.KPpad) * NB2R + row];
  }
}

template <int PROB, typename real>
__device__ __forceinline__ real load_a(const GemmArgs& a, const GroupCtx& c, int col, int k) {
  const real* A = reinterpret_cast<const real*>(a.tab);
  if (col >= c.N || k >= c.K) return 0;
  if (PROB == LEG_F || PROB == RAD_F) {
    return A[c.abase + (int64_t)col * c.as + k];
  } else if (PROB == RAD_I) {
    return A[c.abase + (int64_t)k * c.as + col];
  } else {
    if (k < c.KPpad) {
      if (k >= c.KP) return 0;
      return A[c.abase + (int64_t)k * c.as + col];
    }
    return A[c.abase2 + (int64_t)(k - c.KPpad) * c.as + col];
  }
}

template <int PROB, typename real>
__device__ __forceinline__ void store_y(const GemmArgs& a, const SegDesc& sg, const GroupCtx& c, int row, int col,
                                        real v, real v2) {
  if (row >= c.rows || col >= c.N) return;
  real* Y = reinterpret_cast<real*>(a.y);
  const int B = c.B, NB = c.NB, R = c.R;
  if (PROB == LEG_F) {
    const int b = row / (2 * R);
    const int cc = (row / R) & 1;
    const int i = row % R;
    const int l = c.am + c.p + 2 * col;
    const real s = (c.m < 0 && (c.am & 1)) ? real(-1) : real(1);
    Y[sg.w2_off + (int64_t)NB * 2 * R * l * l + (((int64_t)b * (2 * l + 1) + (c.m + l)) * 2 + cc) * R + i] = s * v;
  } else if (PROB == RAD_F) {
    const int per_b = (2 * c.l + 1) * 2;
    const int b = row / per_b;
    const int rem = row - b * per_b;
    const int mm = rem >> 1, cc = rem & 1;
    const int64_t off = a.fn_coef[sg.fn0 + b] + omega_idx(c.l + 1 + col, c.l, mm - c.l);
    Y[2 * off + cc] = v;
  } else if (PROB == RAD_I) {
    const int per_b = (2 * c.l + 1) * 2;
    const int b = row / per_b;
    const int rem = row - b * per_b;
    const int mm = rem >> 1, cc = rem & 1;
    const int m = mm - c.l;
    const int am = m < 0 ? -m : m;
    const int p = (c.l - am) & 1;
    const int lp = (c.l - am - p) >> 1;
    const int m_idx = m + B - 1;
    const int64_t srow = a.si_rows[sg.si_rows + 2 * m_idx + p] + lp;
    Y[sg.w2_off + srow * NB * 2 * R + ((int64_t)b * 2 + cc) * R + col] = v;
  } else {
    const real s = (c.m < 0 && (c.am & 1)) ? real(-1) : real(1);
    const int64_t base = sg.w1_off + (int64_t)c.m_idx * NB * 2 * R * 2 * B + (int64_t)row * 2 * B;
    Y[base + col] = s * (v + v2);
    Y[base + 2 * B - 1 - col] = s * (v - v2);
  }
}

// Tiles of TMv x TNv outputs (64 x 64, 128 x 32, 256 x 16 with 256 threads;
// 64 x 48 with 192), each thread 4 x 4 of them; the columns of a group left
// after its whole 64-column blocks (N <= 48, 32 or 16 of them) use the
// narrower shapes, so that padding columns do not cost multiply-adds.
template <int PROB, typename real, int TMv, int TNv>
__global__ void __launch_bounds__(TMv * TNv / 16) gemm_simt_kernel(GemmArgs a) {
  constexpr int NT = TMv * TNv / 16;  // threads
  static_assert(TMv % 4 == 0 && TNv % 4 == 0 && NT % 32 == 0 && NT <= 256, "4 x 4 outputs per thread");
  constexpr int CX = TNv / 4, RX = TMv / 4;  // threads along columns and rows
  __shared__ real Xs[TK][TMv + 1];
  __shared__ real As[TK][TNv + 1];
  const int4 t = a.tiles[blockIdx.x];
  const SegDesc sg = a.segs[t.x];
  GroupCtx c;
  group_setup<PROB>(a, sg, t.y, c);
  const int row0 = t.z, col0 = t.w;
  const int tx = threadIdx.x % CX, ty = threadIdx.x / CX;
  real acc[4][4], acc2[4][4];
#pragma unroll
  for (int r = 0; r < 4; ++r)
#pragma unroll
    for (int q = 0; q < 4; ++q) acc[r][q] = acc2[r][q] = 0;
  // seminaive forward Legendre: the tile's highest degree l bounds the DCT
  // indices k' it needs (k' <= deg / 2, the table is zero beyond)
  int kend = c.K;
  if (PROB == LEG_F && a.seminaive) {
    const int cmax = min(col0 + TNv, c.N) - 1;
    const int l = c.am + c.p + 2 * cmax;
    const int deg = (c.am & 1) ? l - 1 : l;
    kend = min(c.K, (c.p ? (deg - 1) / 2 : deg / 2) + 1);
  }
  for (int k0 = 0; k0 < kend; k0 += TK) {
    // X tile: TM rows x TK (k fastest across threads for coalesced row reads)
    for (int e = threadIdx.x; e < TMv * TK; e += NT) {
      const int rr = e / TK, kk = e % TK;
      Xs[kk][rr] = load_x<PROB, real>(a, sg, c, row0 + rr, k0 + kk);
    }
    for (int e = threadIdx.x; e < TNv * TK; e += NT) {
      int cc, kk;
      if (PROB == RAD_I || PROB == LEG_I) {  // tables stored [k][col]: col fastest
        kk = e / TNv;
        cc = e % TNv;
      } else {
        cc = e / TK;
        kk = e % TK;
      }
      As[kk][cc] = load_a<PROB, real>(a, c, col0 + cc, k0 + kk);
    }
    __syncthreads();
    const bool second = (PROB == LEG_I) && (k0 >= c.KPpad);
#pragma unroll
    for (int kk = 0; kk < TK; ++kk) {
      real xv[4], av[4];
#pragma unroll
      for (int r = 0; r < 4; ++r) xv[r] = Xs[kk][ty + RX * r];
#pragma unroll
      for (int q = 0; q < 4; ++q) av[q] = As[kk][tx + CX * q];
      if (second) {
#pragma unroll
        for (int r = 0; r < 4; ++r)
#pragma unroll
          for (int q = 0; q < 4; ++q) acc2[r][q] = fma(xv[r], av[q], acc2[r][q]);
      } else {
#pragma unroll
        for (int r = 0; r < 4; ++r)
#pragma unroll
          for (int q = 0; q < 4; ++q) acc[r][q] = fma(xv[r], av[q], acc[r][q]);
      }
    }
    __syncthreads();
  }
#pragma unroll
  for (int r = 0; r < 4; ++r)
#pragma unroll
    for (int q = 0; q < 4; ++q)
      store_y<PROB, real>(a, sg, c, row0 + ty + RX * r, col0 + tx + CX * q, acc[r][q], acc2[r][q]);
}

// ---------------------------------------------------------------------------
// seminaive Legendre transform: DCTs of the forward spectra
// ---------------------------------------------------------------------------
// Eq. (dct_trick) with the theta-parity fold: an E vector (symmetric part)
// pairs with cos(2k' theta), an O vector with cos((2k'+1) theta), so the DCT
// of the weighted data u_j' = beta_j' w_m(theta_j') x_j' over the half grid
// is a DCT-II (E) or a DCT-IV (O) of length B:
//   E: D_k' = sum_j' u_j' cos(k'(2j'+1) pi / 2B) = Re(e^{-i pi k'/2B} Y_k') / 2,
//      Y the FFT of length 2B of (u_0 .. u_{B-1}, u_{B-1} .. u_0);
//   O: D_k' = sum_j' u_j' cos((2k'+1)(2j'+1) pi / 4B) = Re(e^{-i pi (2k'+1)/4B} Z_k'),
//      Z the FFT of length 2B of (u_j' e^{-i pi j'/2B}, then B zeros).
// w_m = sin(theta) for odd |m| (the cosine-coefficient table holds
// Lambda_lm / w_m), 1 otherwise; beta only for weighted transforms.  In place
// on the spectra, vectors [m_idx][p][b][c][i] of B reals each; the FFT is the
// phi-FFT's shared-memory one.

struct DctArgs {
  const SegDesc* segs;
  const int4* ctas;  // (segment, first vector, vectors, 0)
  const void* tab;
  void* w1;
  int weighted;
};

template <typename real, int N1, int N2C>
__global__ void __launch_bounds__(256) dct_kernel(DctArgs a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int4 cta = a.ctas[blockIdx.x];
  const SegDesc sg = a.segs[cta.x];
  const int B = sg.B, N = 2 * B, NB = sg.NB, NR = sg.R;
  const int n2 = sg.n2;
  const int NV = cta.z;
  const int pitch = ring_pitch(N1, n2);
  real* wre = reinterpret_cast<real*>(smem_raw);
  real* wim = wre + N;
  real* sre = wim + N;
  real* sim = sre + kDctVec * pitch;
  const real* tab = reinterpret_cast<const real*>(a.tab);
  const real* misc = tab + sg.tab_misc;
  const real* dc = tab + sg.tab_dct;  // [cos pi k/2B | sin | cos pi(2k+1)/4B | sin | sin theta]
  for (int k = threadIdx.x; k < N; k += blockDim.x) {
    wre[k] = misc[3 * NR + 2 * B + 2 * k];
    wim[k] = misc[3 * NR + 2 * B + 2 * k + 1];
  }
  real* w1 = reinterpret_cast<real*>(a.w1) + sg.w1_off;
  const int64_t per_m = (int64_t)2 * NB * 2 * NR;  // vectors per m_idx
  for (int e = threadIdx.x; e < NV * B; e += blockDim.x) {
    const int r = e / B, j = e - r * B;
    const int64_t vec = cta.y + r;
    const int m_idx = (int)(vec / per_m);
    const int p = (int)((vec / (per_m / 2)) & 1);
    const int am = m_idx - (B - 1) < 0 ? (B - 1) - m_idx : m_idx - (B - 1);
    real u = w1[vec * B + j];
    if (a.weighted) u *= misc[3 * NR + j];
    if (am & 1) u *= dc[4 * B + j];
    real* pr = sre + r * pitch;
    real* pi = sim + r * pitch;
    auto slot = [&](int k) { const int c1 = k / n2; return c1 * (n2 + 1) + (k - c1 * n2); };
    if (p == 0) {
      pr[slot(j)] = u;
      pi[slot(j)] = 0;
      pr[slot(N - 1 - j)] = u;
      pi[slot(N - 1 - j)] = 0;
    } else {
      pr[slot(j)] = u * dc[j];
      pi[slot(j)] = -u * dc[B + j];
      pr[slot(B + j)] = 0;
      pi[slot(B + j)] = 0;
    }
  }
  __syncthreads();
  fft_rings<real, N1, N2C, false>(sre, sim, wre, wim, NV, n2, N, pitch);
  for (int e = threadIdx.x; e < NV * B; e += blockDim.x) {
    const int r = e / B, k = e - r * B;
    const int64_t vec = cta.y + r;
    const int p = (int)((vec / (per_m / 2)) & 1);
    const int sl = (k % N1) * (n2 + 1) + k / N1;
    const real yr = sre[r * pitch + sl], yi = sim[r * pitch + sl];
    w1[vec * B + k] = p == 0 ? (real)0.5 * (dc[k] * yr + dc[B + k] * yi) : dc[2 * B + k] * yr + dc[3 * B + k] * yi;
  }
}

template <typename real>
static cudaError_t launch_dct_t(const DctArgs& a, int n1, int n2, int first, int nctas, size_t smem, cudaStream_t s) {
  void (*fn)(DctArgs) = nullptr;
#define SGL_PICK(N1, N2C) fn = dct_kernel<real, N1, N2C>;
  if (n1 == 16 && n2 == 16) { SGL_PICK(16, 16) }
  else if (n1 == 16 && n2 == 8) { SGL_PICK(16, 8) }
  else if (n1 == 16) { SGL_PICK(16, 0) }
  else if (n1 == 8) { SGL_PICK(8, 0) }
  else if (n1 == 4) { SGL_PICK(4, 0) }
  else if (n1 == 2) { SGL_PICK(2, 0) }
  else { SGL_PICK(1, 0) }
#undef SGL_PICK
  cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  DctArgs b = a;
  b.ctas = a.ctas + first;
  fn<<<nctas, 256, smem, s>>>(b);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------
template <typename real>
size_t fft_smem_bytes(int n1, int n2, int B, int JP) {
  return sizeof(real) * (2 * 2 * B + 2 * 2 * (size_t)JP * ring_pitch(n1, n2));
}

int fft_pairs_per_cta(int prec, int B) {
  int jp = (prec == SGL_FP64) ? 8 : 16;
  return jp < B ? jp : B;
}

template <typename real, bool INV>
static cudaError_t launch_fft_t(const Plan& P, const FftArgs& a, int n1, int n2, int nctas, size_t smem,
                                cudaStream_t s) {
  void (*fn)(FftArgs) = nullptr;
#define SGL_PICK(N1, N2C)                                                                   \
  fn = INV ? (void (*)(FftArgs))fft_inv_kernel<real, N1, N2C> : (void (*)(FftArgs))fft_fwd_kernel<real, N1, N2C>;
  if (n1 == 16 && n2 == 16) { SGL_PICK(16, 16) }
  else if (n1 == 16 && n2 == 8) { SGL_PICK(16, 8) }
  else if (n1 == 16) { SGL_PICK(16, 0) }
  else if (n1 == 8) { SGL_PICK(8, 0) }
  else if (n1 == 4) { SGL_PICK(4, 0) }
  else if (n1 == 2) { SGL_PICK(2, 0) }
  else { SGL_PICK(1, 0) }
#undef SGL_PICK
  cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  fn<<<nctas, 256, smem, s>>>(a);
  return cudaGetLastError();
}

template <typename real, int TMv, int TNv>
static void launch_gemm_shape(int prob, const GemmArgs& a, int ntiles, cudaStream_t s) {
  constexpr int NT = TMv * TNv / 16;
  switch (prob) {
    case LEG_F: gemm_simt_kernel<LEG_F, real, TMv, TNv><<<ntiles, NT, 0, s>>>(a); break;
    case RAD_F: gemm_simt_kernel<RAD_F, real, TMv, TNv><<<ntiles, NT, 0, s>>>(a); break;
    case RAD_I: gemm_simt_kernel<RAD_I, real, TMv, TNv><<<ntiles, NT, 0, s>>>(a); break;
    default: gemm_simt_kernel<LEG_I, real, TMv, TNv><<<ntiles, NT, 0, s>>>(a); break;
  }
}

// shape w of GemmSched: 0 -> 64 x 64, 1 -> 128 x 32, 2 -> 256 x 16, 3 -> 64 x 48
template <typename real>
static cudaError_t launch_gemm_t(int prob, const GemmArgs& a, int w, int ntiles, cudaStream_t s) {
  if (ntiles == 0) return cudaSuccess;
  if (w == 0) launch_gemm_shape<real, 64, 64>(prob, a, ntiles, s);
  else if (w == 1) launch_gemm_shape<real, 128, 32>(prob, a, ntiles, s);
  else if (w == 2) launch_gemm_shape<real, 256, 16>(prob, a, ntiles, s);
  else launch_gemm_shape<real, 64, 48>(prob, a, ntiles, s);
  return cudaGetLastError();
}

// The FFT launches use one kernel instantiation per (n1, n2) class, so plans
// whose segments differ in those factors launch one FFT kernel per segment
// (the CTA list is sorted by segment; each launch gets its slice).
struct FftSlice {
  int first, count, n1, n2, B;
};

// Consecutive segments that run the same kernel instantiation with the same
// ring pairs per CTA share one launch (each CTA reads its segment); B of a
// slice is its largest bandlimit, which sizes the shared memory.
static void fft_slices(const Plan& P, std::vector<FftSlice>& out, bool inv) {
  out.clear();
  int first = 0, last_cls = -1, last_jp = -1;
  for (size_t s = 0; s < P.segs.size(); ++s) {
    const SegDesc& sg = P.segs[s];
    const int JP = fft_jp(P, sg.B, inv);
    const int per_shell = (sg.B + JP - 1) / JP;  // ring-pair groups per shell
    const int count = sg.NB * sg.R * per_shell;   // R shells per function (R = B on the tensor-core path)
    // kernel class: the register FFT of 2B = 16 * n2 where it applies (one
    // instantiation per n2), else the general kernel of factor n1 with a
    // run-time n2
    const int cls = fft16_handles(P.prec == SGL_FP64, P.real_pairs, sg.n1, sg.n2) ? 100 + sg.n2 : sg.n1;
    if (!out.empty() && cls == last_cls && JP == last_jp) {
      FftSlice& f = out.back();
      f.count += count;
      f.B = std::max(f.B, sg.B);
    } else {
      out.push_back({first, count, sg.n1, sg.n2, sg.B});
    }
    first += count;
    last_cls = cls;
    last_jp = JP;
  }
}

// Whether the slices of one direction run as one launch of the multi-size
// register FFT (fft16.cu): the plan's choice (autotuned), several slices,
// every one a register-FFT size of FP32 complex samples, one ring-pair count.
static bool fft_merged(const Plan& P, const std::vector<FftSlice>& sl, bool inv) {
  if (!P.fft_merge || sl.size() < 2 || P.prec == SGL_FP64 || P.real_pairs) return false;
  const int jp = fft_jp(P, sl[0].B, inv);
  for (const FftSlice& f : sl)
    if (!fft16_handles(false, false, f.n1, f.n2) || fft_jp(P, f.B, inv) != jp) return false;
  return true;
}

int fft_launches(const Plan& P, bool inv) {
  std::vector<FftSlice> sl;
  fft_slices(P, sl, inv);
  return fft_merged(P, sl, inv) ? 1 : (int)sl.size();
}

template <typename real>
static cudaError_t run_fft(Plan& P, bool inv, const void* in, void* out, int mode, cudaStream_t s) {
  StageTimer timer(P, inv ? ST_FFT_I : ST_FFT_F, s);
  std::vector<FftSlice> sl;
  fft_slices(P, sl, inv);
  if (fft_merged(P, sl, inv)) {
    int count = 0, max_n2 = 0;
    for (const FftSlice& f : sl) {
      count += f.count;
      max_n2 = std::max(max_n2, f.n2);
    }
    Fft16Args a16 = {P.d_segs, P.d_fn_samp, inv ? P.d_fft_inv : P.d_fft_fwd, P.d_tab, in, out, P.d_w1,
                     fft_jp(P, sl[0].B, inv), mode, 0, (!inv && P.d_amax) ? P.d_amax + AMAX_EO * P.nfn : nullptr, 0};
    cudaError_t e = cudaSuccess;
    fft16_launch_multi(inv, a16, max_n2, count, s, &e);
    if (e != cudaSuccess) return e;
    timer.finish();
    return cudaSuccess;
  }
  for (const FftSlice& f : sl) {
    FftArgs a;
    a.segs = P.d_segs;
    a.fn_samp = P.d_fn_samp;
    a.ctas = (inv ? P.d_fft_inv : P.d_fft_fwd) + f.first;
    a.tab = P.d_tab;
    a.in = in;
    a.out = out;
    a.w1 = P.d_w1;
    a.JP = fft_jp(P, f.B, inv);
    a.mode = mode;
    a.pair_limit = P.real_pairs ? P.n_samples : 0;
    a.pair_gap = P.real_pairs ? sample_count(P.fn_B[0], n_radial(P.fn_B[0], P.grid)) : 0;
    a.amax = (!inv && P.d_amax) ? P.d_amax + AMAX_EO * P.nfn : nullptr;
    {
      Fft16Args a16 = {a.segs, a.fn_samp, a.ctas, a.tab, a.in, a.out, a.w1, a.JP, a.mode, a.pair_limit, a.amax, a.pair_gap};
      cudaError_t e16 = cudaSuccess;
      if (fft16_launch<real>(inv, a16, f.n1, f.n2, f.count, s, &e16)) {
        if (e16 != cudaSuccess) return e16;
        continue;
      }
    }
    size_t smem = fft_smem_bytes<real>(f.n1, f.n2, f.B, a.JP);
    cudaError_t e = inv ? launch_fft_t<real, true>(P, a, f.n1, f.n2, f.count, smem, s)
                        : launch_fft_t<real, false>(P, a, f.n1, f.n2, f.count, smem, s);
    if (e != cudaSuccess) return e;
  }
  timer.finish();
  return cudaSuccess;
}

// TF32x3 tensor-core stages (tc_gemm.cu)
cudaError_t run_tc_stage(Plan& P, int prob, const void* x, void* y, int weighted, cudaStream_t s);

template <typename real>
static cudaError_t run_gemm(Plan& P, int prob, const GemmSched& sch, const void* x, void* y, int weighted,
                            cudaStream_t s, bool seminaive = false) {
  GemmArgs a;
  a.seminaive = seminaive ? 1 : 0;
  a.segs = P.d_segs;
  a.fn_coef = P.d_fn_coef;
  a.si_rows = P.d_si_rows;
  a.tab = P.d_tab;
  a.x = x;
  a.y = y;
  a.weighted = weighted;
  cudaError_t e = cudaSuccess;
  for (int w = 0; w < kGemmShapes && e == cudaSuccess; ++w) {
    a.tiles = sch.d_tiles[w];
    e = launch_gemm_t<real>(prob, a, w, sch.ntiles[w], s);
  }
  return e;
}

// DCT launches of the seminaive forward Legendre stage, one per segment
template <typename real>
static cudaError_t run_dct(Plan& P, bool weights, cudaStream_t s) {
  DctArgs a;
  a.segs = P.d_segs;
  a.ctas = P.d_dct_ctas;
  a.tab = P.d_tab;
  a.w1 = P.d_w1;
  a.weighted = weights ? 1 : 0;
  int first = 0;
  for (size_t k = 0; k < P.segs.size(); ++k) {
    const SegDesc& sg = P.segs[k];
    const int64_t nvec = (int64_t)(2 * sg.B - 1) * 2 * sg.NB * 2 * sg.R;
    const int nctas = (int)((nvec + kDctVec - 1) / kDctVec);
    const size_t smem = sizeof(real) * (4 * (size_t)sg.B + 2 * (size_t)kDctVec * ring_pitch(sg.n1, sg.n2));
    const cudaError_t e = launch_dct_t<real>(a, sg.n1, sg.n2, first, nctas, smem, s);
    if (e != cudaSuccess) return e;
    first += nctas;
  }
  return cudaSuccess;
}

// FP16x3 plans: the largest |coefficient| (real and imaginary parts) of
// every function, folded into amax[f] (segment order; cleared beforehand).
// blockIdx.x: slices of one function's coefficients, blockIdx.y: functions
// (strided beyond gridDim.y).
__global__ void __launch_bounds__(256) coef_amax_kernel(const cx<float>* coef, const SegDesc* segs, int nseg,
                                                        const int64_t* fn_coef, int nfn, unsigned* amax) {
  for (int f = blockIdx.y; f < nfn; f += gridDim.y) {
    int B = 0;
    for (int s = 0; s < nseg; ++s)
      if (f >= segs[s].fn0 && f < segs[s].fn0 + segs[s].NB) B = segs[s].B;
    const int64_t n = (int64_t)B * (B + 1) * (2 * B + 1) / 6;
    const cx<float>* c = coef + fn_coef[f];
    float mx = 0.f;
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x) {
      const cx<float> v = c[k];
      mx = fmaxf(mx, fmaxf(fabsf(v.x), fabsf(v.y)));
    }
    cta_amax(mx, amax + f);
  }
}

// FP16x3 data scales of a call: clear the slot, and for the inverse measure
// the coefficients (the forward phi-FFT measures its own output).
static cudaError_t fp16_scales(Plan& P, bool inv, const void* coeffs, cudaStream_t s) {
  if (!P.d_amax) return cudaSuccess;
  unsigned* slot = P.d_amax + (inv ? AMAX_COEF : AMAX_EO) * P.nfn;
  cudaError_t e = cudaMemsetAsync(slot, 0, (size_t)P.nfn * sizeof(unsigned), s);
  if (e != cudaSuccess || !inv) return e;
  const int64_t om = coeff_count(P.maxB);
  const dim3 grid((unsigned)std::max<int64_t>(1, std::min<int64_t>(64, (om + 4095) / 4096)),
                  (unsigned)std::min(P.nfn, 65535));
  coef_amax_kernel<<<grid, 256, 0, s>>>((const cx<float>*)coeffs, P.d_segs, (int)P.segs.size(), P.d_fn_coef,
                                        P.nfn, slot);
  return cudaGetLastError();
}

template <typename real>
static cudaError_t forward_t(Plan& P, const void* samples, void* coeffs, cudaStream_t s, bool weights) {
  int mode = 0;
  if (P.samples == SGL_SAMPLES_PHYSICAL) mode = weights ? 1 : 2;
  cudaError_t e = fp16_scales(P, false, nullptr, s);
  if (e != cudaSuccess) return e;
  e = run_fft<real>(P, false, samples, nullptr, mode, s);
  if (e != cudaSuccess) return e;
  if (tc_precision(P.prec)) {
    e = run_tc_stage(P, LEG_F, P.d_w1, P.d_w2, weights, s);
    if (e != cudaSuccess) return e;
    return run_tc_stage(P, RAD_F, P.d_w2, coeffs, weights, s);
  }
  {
    StageTimer timer(P, ST_LEG_F, s);
    if (P.seminaive) e = run_dct<real>(P, weights, s);
    if (e == cudaSuccess) e = run_gemm<real>(P, LEG_F, P.leg_fwd, P.d_w1, P.d_w2, weights, s, P.seminaive);
    timer.finish();
  }
  if (e != cudaSuccess) return e;
  StageTimer timer(P, ST_RAD_F, s);
  e = run_gemm<real>(P, RAD_F, P.rad_fwd, P.d_w2, coeffs, weights, s);
  timer.finish();
  return e;
}

template <typename real>
static cudaError_t inverse_t(Plan& P, const void* coeffs, void* samples, cudaStream_t s, bool weights) {
  cudaError_t e;
  if (tc_precision(P.prec)) {
    e = fp16_scales(P, true, coeffs, s);
    if (e != cudaSuccess) return e;
    e = run_tc_stage(P, RAD_I, coeffs, P.d_w2, 0, s);
    if (e != cudaSuccess) return e;
    e = run_tc_stage(P, LEG_I, P.d_w2, P.d_w1, 0, s);
  } else {
    {
      StageTimer timer(P, ST_RAD_I, s);
      e = run_gemm<real>(P, RAD_I, P.rad_inv, coeffs, P.d_w2, 0, s);
      timer.finish();
    }
    if (e != cudaSuccess) return e;
    StageTimer timer(P, ST_LEG_I, s);
    e = run_gemm<real>(P, LEG_I, P.leg_inv, P.d_w2, P.d_w1, 0, s);
    timer.finish();
  }
  if (e != cudaSuccess) return e;
  int mode = 0;
  if (weights) mode = (P.samples == SGL_SAMPLES_PHYSICAL) ? 3 : 2;
  else if (P.samples == SGL_SAMPLES_PHYSICAL) mode = 1;
  return run_fft<real>(P, true, nullptr, samples, mode, s);
}

// ---------------------------------------------------------------------------
// real functions in pairs
// ---------------------------------------------------------------------------
// A real f has fhat_{n,l,-m} = (-1)^m conj(fhat_{n,l,m}) (Def 2.1:
// Y_l^{-m} = (-1)^m conj(Y_l^m), and the radial part is real).  Write
// S(F)_m = (-1)^m conj(F_{-m}); S is conjugate-linear and fixes the
// coefficients of every real function.  Pair q carries real functions 2q and
// 2q + 1 as one complex function g = f_2q + i f_2q+1, whose coefficients are
// C = F_2q + i F_2q+1, so S(C) = F_2q - i F_2q+1 and
//   F_2q = (C + S(C)) / 2,   F_2q+1 = (C - S(C)) / (2i).
// Shell n of pair q (its n^2 coefficients are contiguous from
// omega(n, 0, 0), element e = l(l+1) + m) per block; each thread computes its
// elements from themselves and their mirrors m -> -m.

// l and m of element e = l(l+1) + m of a shell
__device__ __forceinline__ void lm_of(int e, int& l, int& m) {
  l = (int)sqrtf((float)e);
  while (l * l > e) --l;
  while ((l + 1) * (l + 1) <= e) ++l;
  m = e - l * (l + 1);
}

template <typename real>
__global__ void __launch_bounds__(256) real_split_kernel(const cx<real>* C, cx<real>* out, int64_t Om, int npairs,
                                                         int nreal) {
  const int n = blockIdx.x + 1;
  const int64_t s0 = (int64_t)n * (n - 1) * (2 * n - 1) / 6;
  for (int q = blockIdx.y; q < npairs; q += gridDim.y) {
    const cx<real>* c = C + (int64_t)q * Om + s0;
    cx<real>* o1 = out + (int64_t)(2 * q) * Om + s0;
    const bool has2 = 2 * q + 1 < nreal;
    for (int e = threadIdx.x; e < n * n; e += blockDim.x) {
      int l, m;
      lm_of(e, l, m);
      const real sg = (m & 1) ? (real)-1 : (real)1;
      const cx<real> cp = c[e], cm = c[l * (l + 1) - m];
      const cx<real> d = {sg * cm.x, -sg * cm.y};  // S(C)_m
      o1[e] = {(cp.x + d.x) * (real)0.5, (cp.y + d.y) * (real)0.5};
      if (has2) o1[Om + e] = {(cp.y - d.y) * (real)0.5, -(cp.x - d.x) * (real)0.5};  // (C - S(C)) / 2i
    }
  }
}

// Inverse direction: pair q's complex coefficients from the user's
// coefficients a_2q, a_2q+1, each replaced by its symmetric part
// (a + S(a)) / 2 (the coefficients of the real part of its inverse), so that
// the real and imaginary parts of the complex inverse are Re inverse(a_2q)
// and Re inverse(a_2q+1).
template <typename real>
__global__ void __launch_bounds__(256) real_combine_kernel(const cx<real>* in, cx<real>* C, int64_t Om, int npairs,
                                                           int nreal) {
  const int n = blockIdx.x + 1;
  const int64_t s0 = (int64_t)n * (n - 1) * (2 * n - 1) / 6;
  for (int q = blockIdx.y; q < npairs; q += gridDim.y) {
    const cx<real>* a1 = in + (int64_t)(2 * q) * Om + s0;
    const bool has2 = 2 * q + 1 < nreal;
    cx<real>* c = C + (int64_t)q * Om + s0;
    for (int e = threadIdx.x; e < n * n; e += blockDim.x) {
      int l, m;
      lm_of(e, l, m);
      const int em = l * (l + 1) - m;
      const real sg = (m & 1) ? (real)-1 : (real)1;
      cx<real> g1 = a1[e], g2 = {0, 0};
      {
        const cx<real> t = a1[em];
        g1 = {(g1.x + sg * t.x) * (real)0.5, (g1.y - sg * t.y) * (real)0.5};
      }
      if (has2) {
        const cx<real> u = a1[Om + e], t = a1[Om + em];
        g2 = {(u.x + sg * t.x) * (real)0.5, (u.y - sg * t.y) * (real)0.5};
      }
      c[e] = {g1.x - g2.y, g1.y + g2.x};  // g1 + i g2
    }
  }
}

template <typename real>
static cudaError_t run_real_pairs(Plan& P, bool split, const void* src, void* dst, cudaStream_t s) {
  const int B = P.fn_B[0];
  const int npairs = (P.nreal + 1) / 2;
  const dim3 grid((unsigned)B, (unsigned)std::min(npairs, 65535));
  if (split)
    real_split_kernel<real><<<grid, 256, 0, s>>>((const cx<real>*)src, (cx<real>*)dst, coeff_count(B), npairs, P.nreal);
  else
    real_combine_kernel<real><<<grid, 256, 0, s>>>((const cx<real>*)src, (cx<real>*)dst, coeff_count(B), npairs,
                                                   P.nreal);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// radial halves (tensor-core plans on the paper's grid)
// ---------------------------------------------------------------------------
// Function f runs as the functions 2f and 2f + 1 of B radii each (its first
// and second half of the 2B-node radial rule).  The radial sums of
// Eq. DRT_matrix over the 2B nodes are the sums of the two halves' partial
// sums (forward, and the adjoint of the inverse); both halves synthesize from
// the same coefficients (inverse, and the adjoint of the forward).
template <typename real>
__global__ void halves_sum_kernel(const cx<real>* __restrict__ vc, cx<real>* __restrict__ out, int64_t omega,
                                  int nuser) {
  const int64_t n = omega * nuser;
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x) {
    const int64_t f = k / omega, w = k - f * omega;
    const cx<real> a = vc[2 * f * omega + w], b = vc[(2 * f + 1) * omega + w];
    out[k] = {a.x + b.x, a.y + b.y};
  }
}

template <typename real>
__global__ void halves_copy_kernel(const cx<real>* __restrict__ in, cx<real>* __restrict__ vc, int64_t omega,
                                   int nuser) {
  const int64_t n = omega * nuser;
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x) {
    const int64_t f = k / omega, w = k - f * omega;
    const cx<real> v = in[k];
    vc[2 * f * omega + w] = v;
    vc[(2 * f + 1) * omega + w] = v;
  }
}

static cudaError_t run_halves(const Plan& P, bool sum, const void* src, void* dst, cudaStream_t s) {
  const int64_t omega = coeff_count(P.fn_B[0]);
  const int64_t n = omega * P.nuser;
  const unsigned blocks = (unsigned)std::min<int64_t>((n + 255) / 256, 4 * 152);
  if (sum)  // tensor-core precisions compute in FP32
    halves_sum_kernel<float><<<blocks, 256, 0, s>>>((const cx<float>*)src, (cx<float>*)dst, omega, P.nuser);
  else
    halves_copy_kernel<float><<<blocks, 256, 0, s>>>((const cx<float>*)src, (cx<float>*)dst, omega, P.nuser);
  return cudaGetLastError();
}

cudaError_t run_forward(Plan& P, const void* samples, void* coeffs, cudaStream_t s, bool weights) {
  if (P.radial_halves) {  // the halves' partial sums, then (real functions) the pairs' split
    void* pc = P.real_pairs ? P.d_pcoef : coeffs;
    cudaError_t e = forward_t<float>(P, samples, P.d_ccoef, s, weights);
    if (e == cudaSuccess) e = run_halves(P, true, P.d_ccoef, pc, s);
    if (e == cudaSuccess && P.real_pairs) e = run_real_pairs<float>(P, true, pc, coeffs, s);
    return e;
  }
  if (P.real_pairs) {
    const bool d = P.prec == SGL_FP64;
    cudaError_t e = d ? forward_t<double>(P, samples, P.d_ccoef, s, weights)
                      : forward_t<float>(P, samples, P.d_ccoef, s, weights);
    if (e != cudaSuccess) return e;
    return d ? run_real_pairs<double>(P, true, P.d_ccoef, coeffs, s)
             : run_real_pairs<float>(P, true, P.d_ccoef, coeffs, s);
  }
  if (P.prec == SGL_FP64) return forward_t<double>(P, samples, coeffs, s, weights);
  return forward_t<float>(P, samples, coeffs, s, weights);
}

cudaError_t run_inverse(Plan& P, const void* coeffs, void* samples, cudaStream_t s, bool weights) {
  if (P.radial_halves) {  // (real functions) the pairs' coefficients, then both halves of each
    const void* pc = coeffs;
    cudaError_t e = cudaSuccess;
    if (P.real_pairs) {
      e = run_real_pairs<float>(P, false, coeffs, P.d_pcoef, s);
      pc = P.d_pcoef;
    }
    if (e == cudaSuccess) e = run_halves(P, false, pc, P.d_ccoef, s);
    return e != cudaSuccess ? e : inverse_t<float>(P, P.d_ccoef, samples, s, weights);
  }
  if (P.real_pairs) {
    const bool d = P.prec == SGL_FP64;
    cudaError_t e = d ? run_real_pairs<double>(P, false, coeffs, P.d_ccoef, s)
                      : run_real_pairs<float>(P, false, coeffs, P.d_ccoef, s);
    if (e != cudaSuccess) return e;
    return d ? inverse_t<double>(P, P.d_ccoef, samples, s, weights)
             : inverse_t<float>(P, P.d_ccoef, samples, s, weights);
  }
  if (P.prec == SGL_FP64) return inverse_t<double>(P, coeffs, samples, s, weights);
  return inverse_t<float>(P, coeffs, samples, s, weights);
}

// Host-side helpers used by the plan builder
size_t fft_smem_for(int prec, int n1, int n2, int B) {
  int JP = fft_pairs_per_cta(prec, B);
  return prec == SGL_FP64 ? fft_smem_bytes<double>(n1, n2, B, JP) : fft_smem_bytes<float>(n1, n2, B, JP);
}

void gemm_tile_dims(int& tm, int& tn, int& tk) {
  tm = TM;
  tn = TN;
  tk = TK;
}

}  // namespace sgl
