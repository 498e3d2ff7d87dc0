// phi-FFT kernels for ring lengths 2B = 16 * N2 with 2 <= N2 <= 16 (every
// bandlimit B = 8 * N2 from 16 to 128), the four-step form of the inner sum
// of Eq. (SFFT_rearranged):
//   X[k1 + 16 k2] = sum_{n2} W_N^{n2 k1} W_{N2}^{n2 k2} sum_{n1} x[N2 n1 + n2] W_16^{n1 k1}.
//
// Data path: HBM -> registers (16 independent loads per thread) -> 16-point
// FFT -> one swizzled shared-memory transpose -> N2-point DFT (radix 2 for
// powers of two, mixed radix otherwise) -> HBM.
// A CTA owns one shell (b, i) and JP ring pairs (theta_j, theta_{2B-1-j});
// the forward kernel emits E = G_j + G_mirror and O = G_j - G_mirror directly
// from registers, the inverse kernel gathers its spectra from the Legendre
// synthesis output.  The general kernels in kernels.cu cover every other 2B.
#include <cuda_runtime.h>
#include <stdint.h>

#include "sgl_internal.h"

namespace sgl {

namespace {

template <typename real>
// aligned as a whole value, so that loads and stores move (re, im) at once
struct alignas(2 * sizeof(real)) c2 {
  real x, y;
};

template <typename real>
__device__ __forceinline__ c2<real> operator+(c2<real> a, c2<real> b) { return {a.x + b.x, a.y + b.y}; }
template <typename real>
__device__ __forceinline__ c2<real> operator-(c2<real> a, c2<real> b) { return {a.x - b.x, a.y - b.y}; }
template <typename real>
__device__ __forceinline__ c2<real> cmul(c2<real> a, c2<real> b) {
  return {a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x};
}

// cos(2 pi k / 16), k < 16
constexpr double kCos16[16] = {
    1.0, 0.92387953251128675613, 0.70710678118654752440, 0.38268343236508977173,
    0.0, -0.38268343236508977173, -0.70710678118654752440, -0.92387953251128675613,
    -1.0, -0.92387953251128675613, -0.70710678118654752440, -0.38268343236508977173,
    0.0, 0.38268343236508977173, 0.70710678118654752440, 0.92387953251128675613};

// v * e^{-2 pi i K / N} (INV: e^{+...}) for compile-time K, N (N | 16 * something)
template <typename real, int K, int N, bool INV>
__device__ __forceinline__ c2<real> rot(c2<real> v) {
  constexpr int k = ((K % N) + N) % N;
  if constexpr (k == 0) {
    return v;
  } else if constexpr (4 * k == N) {  // -i (forward), +i (inverse)
    return INV ? c2<real>{-v.y, v.x} : c2<real>{v.y, -v.x};
  } else if constexpr (2 * k == N) {
    return {-v.x, -v.y};
  } else if constexpr (4 * k == 3 * N) {  // +i forward
    return INV ? c2<real>{v.y, -v.x} : c2<real>{-v.y, v.x};
  } else {
    // angle 2 pi k / N = 2 pi (16 k / N) / 16 when N divides 16 k
    static_assert((16 * k) % N == 0, "twiddle not on the 16-point circle");
    constexpr int q = 16 * k / N;
    constexpr double cd = kCos16[q];
    constexpr double sd = kCos16[(q + 12) % 16];  // sin(x) = cos(x - pi/2)
    const real c = (real)cd;
    const real s = (real)sd;
    const real sn = INV ? s : -s;
    return {v.x * c - v.y * sn, v.x * sn + v.y * c};
  }
}

template <int N, int I>
struct BitRev {
  static constexpr int LOG = N == 2 ? 1 : N == 4 ? 2 : N == 8 ? 3 : 4;
  static constexpr int value() {
    int j = 0;
    for (int b = 0; b < LOG; ++b) j |= ((I >> b) & 1) << (LOG - 1 - b);
    return j;
  }
};

template <typename real, int N, bool INV, int LEN, int START, int Q>
__device__ __forceinline__ void bfly(c2<real>* v) {
  c2<real> a = v[START + Q];
  c2<real> b = rot<real, Q * (N / LEN), N, INV>(v[START + Q + LEN / 2]);
  v[START + Q] = a + b;
  v[START + Q + LEN / 2] = a - b;
}

template <typename real, int N, bool INV, int LEN, int START, int Q>
__device__ __forceinline__ void stage_q(c2<real>* v) {
  if constexpr (Q < LEN / 2) {
    bfly<real, N, INV, LEN, START, Q>(v);
    stage_q<real, N, INV, LEN, START, Q + 1>(v);
  }
}

template <typename real, int N, bool INV, int LEN, int START>
__device__ __forceinline__ void stage_s(c2<real>* v) {
  if constexpr (START < N) {
    stage_q<real, N, INV, LEN, START, 0>(v);
    stage_s<real, N, INV, LEN, START + LEN>(v);
  }
}

template <typename real, int N, bool INV, int LEN>
__device__ __forceinline__ void stages(c2<real>* v) {
  if constexpr (LEN <= N) {
    stage_s<real, N, INV, LEN, 0>(v);
    stages<real, N, INV, LEN * 2>(v);
  }
}

template <typename real, int N, int I>
__device__ __forceinline__ void bitrev_perm(c2<real>* v) {
  if constexpr (I < N) {
    constexpr int J = BitRev<N, I>::value();
    if constexpr (I < J) {
      c2<real> t = v[I];
      v[I] = v[J];
      v[J] = t;
    }
    bitrev_perm<real, N, I + 1>(v);
  }
}

// In-register N-point DFT (N = 8 or 16), natural order in and out.
template <typename real, int N, bool INV>
__device__ __forceinline__ void fft_n(c2<real>* v) {
  bitrev_perm<real, N, 0>(v);
  stages<real, N, INV, 2>(v);
}

constexpr bool is_pow2(int n) { return (n & (n - 1)) == 0; }
// smallest prime factor of n >= 2
constexpr int smallest_factor(int n) {
  for (int p = 2; p * p <= n; ++p)
    if (n % p == 0) return p;
  return n;
}

// P-point DFT of x in natural order, in place, P = 2 or an odd prime, with
// w[j] = W_NT^j (P divides NT).  Odd P: the sums s_j = x_j + x_{P-j} and
// differences d_j = x_j - x_{P-j} (j = 1 .. (P-1)/2) give
//   X_0 = x_0 + sum_j s_j,
//   X_k, X_{P-k} = A_k -/+ i B_k,  A_k = x_0 + sum_j s_j cos(2 pi jk/P),
//                                  B_k = sum_j d_j sin(2 pi jk/P)
// (forward; the inverse swaps the signs), real-by-complex products only:
// (P-1)^2 real multiply-adds against 4 (P-1)^2 for the plain sum.
template <typename real, int P, int NT, bool INV>
__device__ __forceinline__ void dft_prime(c2<real>* x, const c2<real>* w) {
  if constexpr (P == 2) {
    const c2<real> a = x[0], b = x[1];
    x[0] = a + b;
    x[1] = a - b;
  } else {
    constexpr int H = (P - 1) / 2, WSP = NT / P;
    c2<real> sm[H], df[H];
    c2<real> x0 = x[0], tot = x[0];
#pragma unroll
    for (int j = 1; j <= H; ++j) {
      sm[j - 1] = x[j] + x[P - j];
      df[j - 1] = x[j] - x[P - j];
      tot = tot + sm[j - 1];
    }
    x[0] = tot;
#pragma unroll
    for (int k = 1; k <= H; ++k) {
      c2<real> A = x0, Bv = {(real)0, (real)0};
#pragma unroll
      for (int j = 1; j <= H; ++j) {
        const c2<real> t = w[((j * k) % P) * WSP];  // cos - i sin of 2 pi jk / P
        A = {A.x + sm[j - 1].x * t.x, A.y + sm[j - 1].y * t.x};
        Bv = {Bv.x - df[j - 1].x * t.y, Bv.y - df[j - 1].y * t.y};
      }
      // -i Bv = (Bv.y, -Bv.x)
      const c2<real> mib = {Bv.y, -Bv.x};
      x[k] = INV ? A - mib : A + mib;
      x[P - k] = INV ? A + mib : A - mib;
    }
  }
}

// N-point DFT (INV: the inverse, unscaled) of v in natural order, in place,
// 2 <= N <= 16.  Powers of two: the radix-2 FFT above.  Other sizes: mixed
// radix, decimation in time over the smallest prime factor P: P subsequences
// of stride P, each transformed recursively (Q = N / P points), then for each
// q < Q the twiddled values W_N^{rq} sub_r[q] go through one P-point DFT,
// which gives the outputs q + Q s; prime sizes by dft_prime.  w[j] = W_NT^j,
// j < NT, is the root table of the size NT this transform belongs to (N
// divides NT); every index into it is a compile-time constant once the loops
// are unrolled, so w stays in registers.
template <typename real, int N, int NT, bool INV>
__device__ __forceinline__ void dft_any(c2<real>* v, const c2<real>* w) {
  if constexpr (is_pow2(N)) {
    fft_n<real, N, INV>(v);
  } else {
    constexpr int P = smallest_factor(N), Q = N / P, WS = NT / N;
    if constexpr (Q == 1) {
      dft_prime<real, N, NT, INV>(v, w);
    } else {
      c2<real> sub[P][Q];
#pragma unroll
      for (int r = 0; r < P; ++r) {
#pragma unroll
        for (int n = 0; n < Q; ++n) sub[r][n] = v[n * P + r];
        dft_any<real, Q, NT, INV>(sub[r], w);
      }
#pragma unroll
      for (int q = 0; q < Q; ++q) {
        c2<real> t[P];
        t[0] = sub[0][q];
#pragma unroll
        for (int r = 1; r < P; ++r) {
          const int e = (r * q) % N;
          if (e == 0) {
            t[r] = sub[r][q];
          } else {
            c2<real> tw = w[e * WS];
            if (INV) tw.y = -tw.y;
            t[r] = cmul(sub[r][q], tw);
          }
        }
        dft_prime<real, P, NT, INV>(t, w);
#pragma unroll
        for (int s = 0; s < P; ++s) v[q + Q * s] = t[s];
      }
    }
  }
}

// Shared-memory position (complex units) of row `row` (< 16), column `col`
// (< N2) of ring r, laid out so that both access patterns of the transpose —
// consecutive (ring, column) items at one row, and the 16 ring pairs at one
// (row, column) — spread over the banks.  Powers of two: rows of N2 columns,
// swizzled by row and ring pair (XOR).  Other N2: columns of 16 rows padded to
// 17 (ring stride 17 N2), the rows rotated by the ring pair: consecutive items
// then step by one bank, and ring pair q lands q (2 N2 + 1) banks further, an
// odd multiple, so the 16 pairs hit 16 different banks (no remainder by N2).
template <int N2>
__device__ __forceinline__ int spos(int r, int row, int col) {
  if constexpr (is_pow2(N2)) return r * (16 * N2) + row * N2 + ((col ^ row ^ (r >> 1)) & (N2 - 1));
  else return r * (17 * N2) + col * 17 + ((row + (r >> 1)) & 15);
}

// Complex elements of one ring in the transpose buffer.
template <int N2>
constexpr int ring_elems() {
  return is_pow2(N2) ? 16 * N2 : 17 * N2;
}

}  // namespace

// Forward: samples -> E/O spectra.  blockDim = 16 * JP.  PAIRS: real
// functions in pairs, the first at twice the complex offset (in reals) as the
// real part, the one pair_gap reals later as the imaginary part (zero past
// pair_limit).
template <typename real, int N2, bool PAIRS>
__device__ __forceinline__ void fft16_fwd_body(const Fft16Args& a) {
  constexpr int N = 16 * N2;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  c2<real>* tw = reinterpret_cast<c2<real>*>(smem_raw);      // [k1 < 16][c < N2]: W_N^{c k1}
  c2<real>* buf = tw + N;                                    // 2*JP rings of ring_elems<N2>()
  c2<real>* w2s = buf + 2 * a.JP * ring_elems<N2>();         // W_N2^j, j < N2
  const int4 cta = a.ctas[blockIdx.x];
  const SegDesc sg = a.segs[cta.x];
  const int B = sg.B, NB = sg.NB, NR = sg.R;  // NR radii
  const int shell = cta.y, j0 = cta.z;
  const int b = shell / NR, i = shell - b * NR;
  const int JPmax = a.JP;
  const int JP = min(JPmax, B - j0);
  const int R = 2 * JP;
  const real* misc = reinterpret_cast<const real*>(a.tab) + sg.tab_misc;
  // twiddles indexed [k1][c], so that the threads of a warp (consecutive c)
  // read consecutive words
  for (int k = threadIdx.x; k < N; k += blockDim.x) {
    const int e = (k % N2) * (k / N2);  // < N
    tw[k] = {misc[3 * NR + 2 * B + 2 * e], misc[3 * NR + 2 * B + 2 * e + 1]};
  }
  for (int k = threadIdx.x; k < N2; k += blockDim.x)  // W_N2^k = W_N^{16 k}
    w2s[k] = {misc[3 * NR + 2 * B + 32 * k], misc[3 * NR + 2 * B + 32 * k + 1]};
  real scale = 1;
  if (a.mode == 1) scale = misc[NR + i];
  if (a.mode == 2) scale = misc[2 * NR + i];
  const c2<real>* in = reinterpret_cast<const c2<real>*>(a.in) + a.fn_samp[sg.fn0 + b] + (int64_t)i * N * N;
  const real* inA = reinterpret_cast<const real*>(a.in) + 2 * a.fn_samp[sg.fn0 + b] + (int64_t)i * N * N;
  const bool hasB = PAIRS && 2 * a.fn_samp[sg.fn0 + b] + a.pair_gap < a.pair_limit;
  __syncthreads();

  // step A: items (r, n2), n2 fastest; 16-point DFT over n1, twiddle, store
  constexpr int PER = (N2 + 7) / 8;  // (2*JP rings x N2 columns) / (16*JP threads), rounded up
  c2<real> v[PER][16];
  int rr[PER], cc[PER];
#pragma unroll
  for (int u = 0; u < PER; ++u) {
    const int item = threadIdx.x + u * blockDim.x;
    rr[u] = item / N2;
    cc[u] = item % N2;
    if (rr[u] < R) {
      const int q = rr[u] >> 1;
      const int j = (rr[u] & 1) ? (N - 1 - (j0 + q)) : (j0 + q);
      if constexpr (PAIRS) {
        const real* ringA = inA + (int64_t)j * N + cc[u];
#pragma unroll
        for (int n1 = 0; n1 < 16; ++n1) v[u][n1] = {ringA[n1 * N2], hasB ? ringA[a.pair_gap + n1 * N2] : (real)0};
      } else {
        const c2<real>* ring = in + (int64_t)j * N + cc[u];
#pragma unroll
        for (int n1 = 0; n1 < 16; ++n1) v[u][n1] = ring[n1 * N2];
      }
    }
  }
#pragma unroll
  for (int u = 0; u < PER; ++u) {
    if (rr[u] < R) {
#pragma unroll
      for (int n1 = 0; n1 < 16; ++n1) v[u][n1] = {v[u][n1].x * scale, v[u][n1].y * scale};
      fft_n<real, 16, false>(v[u]);
#pragma unroll
      for (int k1 = 1; k1 < 16; ++k1) v[u][k1] = cmul(v[u][k1], tw[k1 * N2 + cc[u]]);
#pragma unroll
      for (int k1 = 0; k1 < 16; ++k1) buf[spos<N2>(rr[u], k1, cc[u])] = v[u][k1];
    }
  }
  __syncthreads();

  // step B: items (q, k1), q fastest; N2-point DFT over n2 of both rings of
  // the pair, then E/O straight to global memory
  const int q = threadIdx.x % JPmax;
  const int k1 = threadIdx.x / JPmax;
  float mx = 0.f;  // largest |E/O| of this thread (FP16x3 data scale)
  if (q < JP && k1 < 16) {
    c2<real> x0[N2], x1[N2], w2[N2];
#pragma unroll
    for (int n2 = 0; n2 < N2; ++n2) {
      x0[n2] = buf[spos<N2>(2 * q, k1, n2)];
      x1[n2] = buf[spos<N2>(2 * q + 1, k1, n2)];
      if constexpr (!is_pow2(N2)) w2[n2] = w2s[n2];
    }
    dft_any<real, N2, N2, false>(x0, w2);
    dft_any<real, N2, N2, false>(x1, w2);
    real* w1 = reinterpret_cast<real*>(a.w1) + sg.w1_off;
    const int64_t sp = (int64_t)NB * 2 * NR * B;              // stride of p
    const int64_t sm = 2 * sp;                                // stride of m_idx
    const int64_t base = (((int64_t)b * 2) * NR + i) * B + j0 + q;  // c = 0, p = 0, m_idx = 0
    const int64_t sc = (int64_t)NR * B;                       // stride of c
#pragma unroll
    for (int k2 = 0; k2 < N2; ++k2) {
      const int k = k1 + 16 * k2;
      if (k == B) continue;  // Nyquist: not a coefficient
      const int m = k < B ? k : k - N;
      const int64_t o = base + (int64_t)(m + B - 1) * sm;
      const c2<real> e = x0[k2] + x1[k2];
      const c2<real> d = x0[k2] - x1[k2];
      w1[o] = e.x;
      w1[o + sc] = e.y;
      w1[o + sp] = d.x;
      w1[o + sp + sc] = d.y;
      if (a.amax) mx = fmaxf(mx, fmaxf(fmaxf(fabsf((float)e.x), fabsf((float)e.y)),
                                         fmaxf(fabsf((float)d.x), fabsf((float)d.y))));
    }
  }
  if (a.amax) cta_amax(mx, a.amax + sg.fn0 + b);
}

// Inverse: G spectra -> samples.  blockDim = 16 * JP.  PAIRS: real and
// imaginary parts to the pair's two real functions (as in the forward kernel).
template <typename real, int N2, bool PAIRS>
__device__ __forceinline__ void fft16_inv_body(const Fft16Args& a) {
  constexpr int N = 16 * N2;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  c2<real>* tw = reinterpret_cast<c2<real>*>(smem_raw);    // W_N^k, k < N
  c2<real>* buf = tw + N;
  const int4 cta = a.ctas[blockIdx.x];
  const SegDesc sg = a.segs[cta.x];
  const int B = sg.B, NB = sg.NB, NR = sg.R;  // NR radii
  // cta.w = 0: spectra stored [m][b][c][i][j]; the CTA owns shell i and ring
  //            pairs j0 .. j0+JP-1 (cta.y = b*NR + i, cta.z = j0);
  // cta.w = 1: spectra stored [m][b][j][i][c] (complex pairs); the CTA owns
  //            shells i0 .. i0+JP-1 and the single ring pair jp (cta.y = b*NR + i0, cta.z = jp)
  const int lay = cta.w;
  const int b = cta.y / NR, i_or_i0 = cta.y - b * NR, j_or_jp = cta.z;
  const int JPmax = a.JP;
  const int JP = min(JPmax, lay ? NR - i_or_i0 : B - j_or_jp);
  const int R = 2 * JP;
  const real* misc = reinterpret_cast<const real*>(a.tab) + sg.tab_misc;
  for (int k = threadIdx.x; k < N; k += blockDim.x)
    tw[k] = {misc[3 * NR + 2 * B + 2 * k], misc[3 * NR + 2 * B + 2 * k + 1]};
  __syncthreads();

  // step 1: items (q, k1); gather X[k1 + 16 k2] of both rings, inverse
  // N2-point DFT over k2, twiddle W_N^{-n2 k1}, store row k1
  const int q = threadIdx.x % JPmax;
  const int k1 = threadIdx.x / JPmax;
  if (q < JP && k1 < 16) {
    const real* g = reinterpret_cast<const real*>(a.w1) + sg.w1_off;
    const int iq = lay ? i_or_i0 + q : i_or_i0;
    const int jA = lay ? j_or_jp : j_or_jp + q;
    const int jB = N - 1 - jA;
    c2<real> x0[N2], x1[N2];
    if (lay) {
      // complex element (m_idx, j, i) of function b: m_idx*sm + b*N*NR + j*NR + i
      const c2<real>* gc = reinterpret_cast<const c2<real>*>(g);
      const int64_t sm = (int64_t)NB * N * NR;
      const int64_t base = (int64_t)b * N * NR + iq;
      const int64_t oA = base + (int64_t)jA * NR, oB = base + (int64_t)jB * NR;
#pragma unroll
      for (int k2 = 0; k2 < N2; ++k2) {
        const int k = k1 + 16 * k2;
        if (k == B) {
          x0[k2] = {0, 0};
          x1[k2] = {0, 0};
        } else {
          const int m = k < B ? k : k - N;
          const int64_t o = (int64_t)(m + B - 1) * sm;
          x0[k2] = gc[o + oA];
          x1[k2] = gc[o + oB];
        }
      }
    } else {
      // element (m_idx, c, j) of ring (b, iq): m_idx*sm + c*sc + base + j
      const int64_t sm = (int64_t)NB * 2 * NR * N;
      const int64_t sc = (int64_t)NR * N;
      const int64_t base = (((int64_t)b * 2) * NR + iq) * N;
      const int64_t oA = base + jA, oB = base + jB;
#pragma unroll
      for (int k2 = 0; k2 < N2; ++k2) {
        const int k = k1 + 16 * k2;
        if (k == B) {
          x0[k2] = {0, 0};
          x1[k2] = {0, 0};
        } else {
          const int m = k < B ? k : k - N;
          const int64_t o = (int64_t)(m + B - 1) * sm;
          x0[k2] = {g[o + oA], g[o + sc + oA]};
          x1[k2] = {g[o + oB], g[o + sc + oB]};
        }
      }
    }
    c2<real> w2[N2];  // W_N2^j = W_N^{16 j}
    if constexpr (!is_pow2(N2)) {
#pragma unroll
      for (int j = 0; j < N2; ++j) w2[j] = tw[16 * j];
    }
    dft_any<real, N2, N2, true>(x0, w2);
    dft_any<real, N2, N2, true>(x1, w2);
#pragma unroll
    for (int n2 = 0; n2 < N2; ++n2) {
      c2<real> w = tw[n2 * k1];
      w.y = -w.y;
      buf[spos<N2>(2 * q, k1, n2)] = cmul(x0[n2], w);
      buf[spos<N2>(2 * q + 1, k1, n2)] = cmul(x1[n2], w);
    }
  }
  __syncthreads();

  // step 2: items (r, n2), n2 fastest; inverse 16-point DFT over k1 -> x[N2 n1 + n2]
  c2<real>* out = reinterpret_cast<c2<real>*>(a.out) + a.fn_samp[sg.fn0 + b];
  for (int item = threadIdx.x; item < R * N2; item += blockDim.x) {
    const int r = item / N2, n2 = item % N2;
    c2<real> v[16];
#pragma unroll
    for (int kk = 0; kk < 16; ++kk) v[kk] = buf[spos<N2>(r, kk, n2)];
    fft_n<real, 16, true>(v);
    const int qq = r >> 1;
    const int i = lay ? i_or_i0 + qq : i_or_i0;
    const int jq = lay ? j_or_jp : j_or_jp + qq;
    const int j = (r & 1) ? (N - 1 - jq) : jq;
    real s = 1;
    if (a.mode == 1) s = misc[2 * NR + i];
    if (a.mode == 2) s = misc[i];
    if (a.mode == 3) s = misc[i] * misc[NR + i];
    if (a.mode >= 2) s *= misc[3 * NR + j];
    if constexpr (PAIRS) {
      const int64_t f0 = 2 * a.fn_samp[sg.fn0 + b];
      real* ringA = reinterpret_cast<real*>(a.out) + f0 + ((int64_t)i * N + j) * N + n2;
#pragma unroll
      for (int n1 = 0; n1 < 16; ++n1) ringA[n1 * N2] = v[n1].x * s;
      if (f0 + a.pair_gap < a.pair_limit) {
#pragma unroll
        for (int n1 = 0; n1 < 16; ++n1) ringA[a.pair_gap + n1 * N2] = v[n1].y * s;
      }
    } else {
      c2<real>* ring = out + ((int64_t)i * N + j) * N + n2;
#pragma unroll
      for (int n1 = 0; n1 < 16; ++n1) ring[n1 * N2] = {v[n1].x * s, v[n1].y * s};
    }
  }
}

template <typename real, int N2, bool PAIRS>
__global__ void __launch_bounds__(256) fft16_fwd_kernel(Fft16Args a) {
  fft16_fwd_body<real, N2, PAIRS>(a);
}

template <typename real, int N2, bool PAIRS>
__global__ void __launch_bounds__(256) fft16_inv_kernel(Fft16Args a) {
  fft16_inv_body<real, N2, PAIRS>(a);
}

// One launch over segments of several register-FFT sizes (FP32 complex
// samples): each CTA runs the body of its own segment's N2.  Its register
// count is the largest of the bodies'.
#define SGL_FFT16_CASES(BODY)                                                                  \
  switch (a.segs[a.ctas[blockIdx.x].x].n2) {                                                    \
    case 2: BODY<float, 2, false>(a); break;                                                    \
    case 3: BODY<float, 3, false>(a); break;                                                    \
    case 4: BODY<float, 4, false>(a); break;                                                    \
    case 5: BODY<float, 5, false>(a); break;                                                    \
    case 6: BODY<float, 6, false>(a); break;                                                    \
    case 7: BODY<float, 7, false>(a); break;                                                    \
    case 8: BODY<float, 8, false>(a); break;                                                    \
    case 9: BODY<float, 9, false>(a); break;                                                    \
    case 10: BODY<float, 10, false>(a); break;                                                  \
    case 11: BODY<float, 11, false>(a); break;                                                  \
    case 12: BODY<float, 12, false>(a); break;                                                  \
    case 13: BODY<float, 13, false>(a); break;                                                  \
    case 14: BODY<float, 14, false>(a); break;                                                  \
    case 15: BODY<float, 15, false>(a); break;                                                  \
    case 16: BODY<float, 16, false>(a); break;                                                  \
    default: break;                                                                             \
  }

__global__ void __launch_bounds__(256) fft16_fwd_multi_kernel(Fft16Args a) { SGL_FFT16_CASES(fft16_fwd_body) }
__global__ void __launch_bounds__(256) fft16_inv_multi_kernel(Fft16Args a) { SGL_FFT16_CASES(fft16_inv_body) }
#undef SGL_FFT16_CASES

// One launch of the multi-size kernel over nctas CTAs whose segments' sizes
// are at most 16 * max_n2.
bool fft16_launch_multi(bool inv, const Fft16Args& a, int max_n2, int nctas, cudaStream_t s, cudaError_t* err) {
  if (max_n2 < 2 || max_n2 > 16 || a.pair_limit) return false;
  void (*fn)(Fft16Args) = inv ? fft16_inv_multi_kernel : fft16_fwd_multi_kernel;
  const int N = 16 * max_n2;
  // transpose rings of at most 17 max_n2 elements (padded layout of the sizes that are not powers of two)
  const size_t smem = sizeof(c2<float>) * ((size_t)N + (size_t)2 * a.JP * 17 * max_n2 + (size_t)max_n2);
  cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e == cudaSuccess) {
    fn<<<nctas, 16 * a.JP, smem, s>>>(a);
    e = cudaGetLastError();
  }
  *err = e;
  return true;
}

// Launch helper: returns false when (n1, n2) is not handled here.  Every
// 2B = 16 * N2 with 2 <= N2 <= 16 for FP32 complex samples; N2 in {8, 16} for
// FP64 and for real functions in pairs.
template <typename real, int N2>
static void (*pick_fft16(bool inv, bool pairs))(Fft16Args) {
  if constexpr (N2 == 8 || N2 == 16) {
    if (pairs) return inv ? fft16_inv_kernel<real, N2, true> : fft16_fwd_kernel<real, N2, true>;
  }
  if (pairs) return nullptr;
  return inv ? fft16_inv_kernel<real, N2, false> : fft16_fwd_kernel<real, N2, false>;
}

template <typename real>
bool fft16_launch(bool inv, const Fft16Args& a, int n1, int n2, int nctas, cudaStream_t s, cudaError_t* err) {
  if (n1 != 16 || n2 < 2 || n2 > 16) return false;
  const bool pairs = a.pair_limit != 0;
  void (*fn)(Fft16Args) = nullptr;
  if (n2 == 16) fn = pick_fft16<real, 16>(inv, pairs);
  else if (n2 == 8) fn = pick_fft16<real, 8>(inv, pairs);
  else if constexpr (sizeof(real) == 4) {
    switch (n2) {
      case 2: fn = pick_fft16<real, 2>(inv, pairs); break;
      case 3: fn = pick_fft16<real, 3>(inv, pairs); break;
      case 4: fn = pick_fft16<real, 4>(inv, pairs); break;
      case 5: fn = pick_fft16<real, 5>(inv, pairs); break;
      case 6: fn = pick_fft16<real, 6>(inv, pairs); break;
      case 7: fn = pick_fft16<real, 7>(inv, pairs); break;
      case 9: fn = pick_fft16<real, 9>(inv, pairs); break;
      case 10: fn = pick_fft16<real, 10>(inv, pairs); break;
      case 11: fn = pick_fft16<real, 11>(inv, pairs); break;
      case 12: fn = pick_fft16<real, 12>(inv, pairs); break;
      case 13: fn = pick_fft16<real, 13>(inv, pairs); break;
      case 14: fn = pick_fft16<real, 14>(inv, pairs); break;
      case 15: fn = pick_fft16<real, 15>(inv, pairs); break;
      default: break;
    }
  }
  if (!fn) return false;
  const int N = 16 * n2;
  const bool p2 = (n2 & (n2 - 1)) == 0;
  const size_t smem = sizeof(c2<real>) * ((size_t)N + (size_t)2 * a.JP * (p2 ? 16 : 17) * n2 + (size_t)n2);
  cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e == cudaSuccess) {
    fn<<<nctas, 16 * a.JP, smem, s>>>(a);
    e = cudaGetLastError();
  }
  *err = e;
  return true;
}

// Whether fft16_launch takes rings of 2B = n1 * n2 (the plan groups FFT
// launches by kernel instantiation).
bool fft16_handles(bool fp64, bool pairs, int n1, int n2) {
  if (n1 != 16 || n2 < 2 || n2 > 16) return false;
  if (fp64 || pairs) return n2 == 8 || n2 == 16;
  return true;
}

template bool fft16_launch<float>(bool, const Fft16Args&, int, int, int, cudaStream_t, cudaError_t*);
template bool fft16_launch<double>(bool, const Fft16Args&, int, int, int, cudaStream_t, cudaError_t*);

}  // namespace sgl
