// TF32x3 tensor-core inverse stages (tcgen05, TMEM, TMA) of the SGL transform.
//
// Inverse radial stage (iDRT, R_l^T of Sect. 3.3.2), one GEMM per degree l:
//   S[i][col] = sum_{n'} T_{l+1+n',l}(i) fhat[col][n'],  col = (b, m, c)
//   A operand: the table, M = 128 rows i, streamed per K chunk by bulk copy;
//   B operand: coefficients gathered by the split warps (N = 128 columns).
//   Output rows i are contiguous in the Legendre stage's input layout.
// Inverse Legendre stage (the inner sum of Eq. iSFFT_rearranged), one tile
// per (m, 128 rows (b, c, i)) with both theta-parities:
//   P[row][j'] = sum_{l' even} S[row][l'] Lambda(theta_j'),  Q likewise for odd,
//   G_j' = P + Q,  G_{2B-1-j'} = P - Q   (Lambda(pi - theta) = (-1)^{l+m} Lambda(theta)).
//   A operand: S rows, loaded l'-major by TMA into a staging ring and
//   transposed to K-major hi/lo by the split warps; B operand: the table.
// Same role layout as the forward kernels (tc_ptx.cuh): producer warp, TMEM
// owner and MMA issuer warp, split warps, epilogue warps; bounded waits.
#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include <vector>

#include "sgl_internal.h"
#include "tc_ptx.cuh"

namespace sgl {

using namespace tcx;

namespace {
constexpr int kThreadsInv = kRoleThreads;
constexpr int kChunk = 128 * 128;   // 128 rows x 32 floats
constexpr int kStagesLegI = 2;    // operand ring of the Legendre synthesis
constexpr int kStagingLegI = 4;   // TMA staging ring of the Legendre synthesis
constexpr int kStagesRadI = 3;

// 128-byte swizzled K-major position of (row, 16-byte chunk q) in a tile
__device__ __forceinline__ int sw_pos(int row, int q) { return row * 128 + ((q ^ (row & 7)) << 4); }

// Split 4*NQ consecutive K values v of one row into TF32 hi/lo and store them
// at 16-byte chunks q0 .. q0+NQ-1 of the row (hi only when !with_lo).
template <int NQ>
__device__ __forceinline__ void split_store(unsigned char* hi, unsigned char* lo, int row, const float* v, int q0,
                                            bool with_lo = true) {
#pragma unroll
  for (int qq = 0; qq < NQ; ++qq) {
    const int q = q0 + qq;
    float4 h, l;
    h.x = tf32_rna(v[4 * qq +0]);
    h.y = tf32_rna(v[4 * qq +1]);
    h.z = tf32_rna(v[4 * qq +2]);
    h.w = tf32_rna(v[4 * qq +3]);
    l.x = tf32_rna(v[4 * qq +0] - h.x);
    l.y = tf32_rna(v[4 * qq +1] - h.y);
    l.z = tf32_rna(v[4 * qq +2] - h.z);
    l.w = tf32_rna(v[4 * qq +3] - h.w);
    *(float4*)(hi + sw_pos(row, q)) = h;
    if (with_lo) *(float4*)(lo + sw_pos(row, q)) = l;
  }
}

// BF16 form: 4*NQ consecutive K values of one row (NQ even) as BF16 hi/lo
// pairs, at 16-byte chunks q0/2 .. q0/2 + NQ/2 - 1 of 64-byte rows.
template <int NQ>
__device__ __forceinline__ void split_store_bf(unsigned char* hi, unsigned char* lo, int row, const float* v,
                                               int q0) {
#pragma unroll
  for (int j = 0; j < NQ / 2; ++j) {
    uint32_t hw[4], lw[4];
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      const uint32_t a = bf16_split(v[8 * j + 2 * e]), b = bf16_split(v[8 * j + 2 * e + 1]);
      hw[e] = (a & 0xFFFFu) | (b << 16);
      lw[e] = (a >> 16) | (b & 0xFFFF0000u);
    }
    const int off = sw64_off(row, q0 / 2 + j);
    *(uint4*)(hi + off) = make_uint4(hw[0], hw[1], hw[2], hw[3]);
    *(uint4*)(lo + off) = make_uint4(lw[0], lw[1], lw[2], lw[3]);
  }
}
}  // namespace

// ===========================================================================
// inverse Legendre
// ===========================================================================
// Accumulators: the tensor cores round partial sums toward zero, so each
// result keeps a main accumulator (hi*hi) and a correction accumulator
// (hi*lo + lo*hi), added with round-to-nearest in the epilogue.  With P and Q
// that is four accumulators per tile, so the j' range is cut in halves of 64
// columns to let two tiles' accumulators fit tensor memory.  Tiles run in the
// order (m, j'-half, rows): only the current half of the table is resident,
// which leaves shared memory for a 4-deep staging ring; each row block is
// read once per half.
struct LegIArgs {
  const int2* tiles;          // (m_idx, row0 | j'-half), ordered by (m_idx, half, row0)
  const int* cta_first;       // tile slice of each CTA (gridDim.x + 1 offsets)
  int ntiles;
  const unsigned char* tabimg;
  const int64_t* am_off;      // image offset per (|m|, half)
  const int* am_kc;           // KC_P | KC_Q << 8 per |m|
  const int64_t* si_rows;     // S row offset per (m_idx, p)
  float* g;                   // output, layout [m_idx][b][c][j < 2B][i]
  int* err;
  int B, NB, npad, kcmax;
  int nprod;                  // TF32 products per K step: 3 or 1 (hi*hi)
};

// BF: BF16 hi/lo operands (kind::f16, 64-byte rows, K = 16 per MMA).
template <bool BF>
__global__ void __launch_bounds__(kThreadsInv, 1) tc_leg_inv_kernel(const __grid_constant__ CUtensorMap smap,
                                                                    LegIArgs a) {
  constexpr int ROWB = BF ? 64 : 128;  // bytes of one operand row of a 32-value K chunk
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char* base = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  const int B = a.B, NB = a.NB, npad = a.npad;
  const int nh = npad > 64 ? 64 : npad;                    // rows (j') of one table half
  const int chunk_tab = nh * ROWB;                         // one table chunk (hi or lo)
  unsigned char* tab = base;                               // [P hi][P lo][Q hi][Q lo] of one half
  unsigned char* stg = tab + (size_t)a.kcmax * 2 * chunk_tab;   // staging ring: 32 l' x 128 rows each
  unsigned char* xs = stg + kStagingLegI * kChunk;         // operand ring: (hi, lo)
  uint64_t* bars = (uint64_t*)(xs + kStagesLegI * 2 * kChunk);
  uint64_t* stgf = bars;                        // [T] staging landed
  uint64_t* stge = stgf + kStagingLegI;         // [T] staging read
  uint64_t* split = stge + kStagingLegI;        // [S] hi/lo ready
  uint64_t* empty = split + kStagesLegI;        // [S] MMAs done
  uint64_t* accf = empty + kStagesLegI;         // [2]
  uint64_t* acce = accf + 2;                    // [2]
  uint64_t* tabf = acce + 2;
  uint64_t* tabe = tabf + 1;
  uint32_t* tmem_slot = (uint32_t*)(tabe + 1);
  volatile int* abort_flag = (volatile int*)(tmem_slot + 1);
  // per-group metadata and the tile slice, copied once to shared memory
  int64_t* s_si = (int64_t*)(bars + 64);          // [(2B-1)*2] S row offsets
  int64_t* s_off = s_si + 2 * (2 * B - 1);         // [2B] table image offsets per (|m|, half)
  int* s_kc = (int*)(s_off + 2 * B);               // [B] KC_P | KC_Q << 8
  int2* s_tiles = (int2*)(((uintptr_t)(s_kc + B) + 7) & ~(uintptr_t)7);
  for (int k = threadIdx.x; k < 2 * (2 * B - 1); k += blockDim.x) s_si[k] = a.si_rows[k];
  for (int k = threadIdx.x; k < 2 * B; k += blockDim.x) s_off[k] = a.am_off[k];
  for (int k = threadIdx.x; k < B; k += blockDim.x) s_kc[k] = a.am_kc[k];

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  uint32_t tmem_cols = 32;
  while (tmem_cols < (uint32_t)(8 * nh)) tmem_cols <<= 1;  // 2 buffers x {P, Q} x {main, corr}
  if (threadIdx.x == 0) {
    for (int s = 0; s < kStagingLegI; ++s) {
      mbar_init(stgf + s, 1);
      mbar_init(stge + s, kSplitThreads);
    }
    for (int s = 0; s < kStagesLegI; ++s) {
      mbar_init(split + s, kSplitThreads);
      mbar_init(empty + s, 2);  // the issuing warp's MMAs done, and the other issuer past the stage
    }
    for (int k = 0; k < 2; ++k) {
      mbar_init(accf + k, 2);  // both MMA issuers
      mbar_init(acce + k, kEpiThreads);
    }
    mbar_init(tabf, 1);
    mbar_init(tabe, 2);
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) tmem_alloc(tmem_slot, tmem_cols);
  const int g_begin = a.cta_first[blockIdx.x];
  const int nt = a.cta_first[blockIdx.x + 1] - g_begin;
  for (int k = threadIdx.x; k < nt; k += blockDim.x) s_tiles[k] = a.tiles[g_begin + k];
  tc_before();
  __syncthreads();
  tc_after();
  const uint32_t tmem = *tmem_slot;
  // the resident table changes with (m_idx, half)
  auto table_key = [&](int2 tl) { return 2 * tl.x + (tl.y & 1); };
  auto abs_m = [&](int m_idx) { return m_idx >= B - 1 ? m_idx - (B - 1) : (B - 1) - m_idx; };

  if (warp == 0) {
    if (lane == 0) {
      int cur = -1, ngrp = 0;
      uint32_t c = 0;
      for (int t = 0; t < nt && !*abort_flag; ++t) {
        const int2 tl = s_tiles[t];
        const int m_idx = tl.x, jh = tl.y & 1;
        const int am = abs_m(m_idx);
        const int kcp = s_kc[am] & 0xff, kcq = s_kc[am] >> 8;
        if (table_key(tl) != cur) {
          if (ngrp > 0 && !mbar_wait(tabe, (ngrp - 1) & 1, abort_flag)) break;
          const uint32_t bytes = (uint32_t)((kcp + kcq) * 2 * chunk_tab);
          mbar_arrive_tx(tabf, bytes);
          bulk_load(tab, a.tabimg + s_off[2 * am + jh], bytes, tabf);
          cur = table_key(tl);
          ++ngrp;
        }
        bool ok = true;
        for (int p = 0; p < 2 && ok; ++p) {
          const int kcn = p ? kcq : kcp;
          const int64_t r0 = s_si[2 * m_idx + p];
          for (int kc = 0; kc < kcn; ++kc, ++c) {
            const int s = c % kStagingLegI;
            if (!mbar_wait(stge + s, ((c / kStagingLegI) & 1) ^ 1, abort_flag)) { ok = false; break; }
            mbar_arrive_tx(stgf + s, kChunk);
            tma_load_2d(stg + s * kChunk, &smap, stgf + s, tl.y & ~1, (int)(r0 + kc * 32));
          }
        }
        if (!ok) break;
      }
    }
  } else if (warp == 1 || warp == kMma2Warp) {
    // MMA issuer `me` takes the chunks of parity p = me (P or Q accumulators)
    if (lane == 0) {
      const int p = warp == 1 ? 0 : 1;
      int cur = -1, ngrp = 0;
      uint32_t c = 0, tcount = 0;
      // the table image stacks nh hi rows over nh lo rows per K chunk: one
      // MMA of width 2 nh gives [X_hi T_hi | X_hi T_lo], a second of width nh
      // adds X_lo T_hi to the correction
      const uint32_t idesc2 = BF ? idesc_bf16(2 * nh) : idesc_tf32(2 * nh);
      const uint32_t idesc1 = BF ? idesc_bf16(nh) : idesc_tf32(nh);
      const uint64_t xdesc0 = BF ? sw64_desc(smem_u32(xs)) : sw128_desc(smem_u32(xs));
      const uint64_t tdesc0 = BF ? sw64_desc(smem_u32(tab)) : sw128_desc(smem_u32(tab));
      for (int t = 0; t < nt && !*abort_flag; ++t, ++tcount) {
        const int2 tl = s_tiles[t];
        const int am = abs_m(tl.x);
        const int kcp = s_kc[am] & 0xff, kcq = s_kc[am] >> 8;
        if (table_key(tl) != cur) {
          if (!mbar_wait(tabf, ngrp & 1, abort_flag)) break;
          cur = table_key(tl);
          ++ngrp;
        }
        const int acc = tcount & 1;
        if (!mbar_wait(acce + acc, ((tcount >> 1) & 1) ^ 1, abort_flag)) break;
        tc_after();
        bool ok = true;
        // accumulators of this buffer: [P main][P corr][Q main][Q corr], nh columns each
        const uint32_t d = tmem + (uint32_t)((4 * acc + 2 * p) * nh);
        const uint64_t tp = tdesc0 + (uint64_t)(((p ? kcp : 0) * 2 * chunk_tab) >> 4);
        // Every chunk of the tile is waited for, so that the ring's phases are
        // followed in order; only the chunks of parity p are issued here.  A
        // stage is refilled only after both issuers are past it (the other
        // issuer's plain arrival on `empty`), so neither can fall a whole ring
        // behind and mistake an older phase of the same parity for the next.
        for (int ch = 0; ch < kcp + kcq; ++ch, ++c) {
          const int s = c % kStagesLegI;
          if (!mbar_wait(split + s, (c / kStagesLegI) & 1, abort_flag)) { ok = false; break; }
          if ((ch >= kcp) != (p == 1)) {
            mbar_arrive(empty + s);
            continue;
          }
          const int kc = p ? ch - kcp : ch;
          tc_after();
          const uint64_t xh = xdesc0 + (uint64_t)((s * 2 * kChunk) >> 4);
          const uint64_t xl = xh + (uint64_t)(kChunk >> 4);
          const uint64_t th = tp + (uint64_t)((kc * 2 * chunk_tab) >> 4);
          if (BF) {  // two K steps of 16
#pragma unroll
            for (int kk = 0; kk < 2; ++kk) {
              const uint32_t first = (kc > 0 || kk > 0) ? 1u : 0u;
              mma_bf16(d, xh + 2 * kk, th + 2 * kk, idesc2, first);
              mma_bf16(d + (uint32_t)nh, xl + 2 * kk, th + 2 * kk, idesc1, 1u);
            }
          } else {
#pragma unroll
            for (int kk = 0; kk < 4; ++kk) {
              const uint32_t first = (kc > 0 || kk > 0) ? 1u : 0u;
              if (a.nprod == 3) {
                mma_tf32(d, xh + 2 * kk, th + 2 * kk, idesc2, first);
                mma_tf32(d + (uint32_t)nh, xl + 2 * kk, th + 2 * kk, idesc1, 1u);
              } else {
                mma_tf32(d, xh + 2 * kk, th + 2 * kk, idesc1, first);
              }
            }
          }
          mma_commit(empty + s);
        }
        if (!ok) break;
        mma_commit(accf + acc);
        if (t + 1 >= nt || table_key(s_tiles[t + 1]) != cur) mma_commit(tabe);
      }
    }
  } else if (warp < kFirstEpiWarp) {
    // staging [32 l'][128 rows] -> K-major hi/lo rows; thread (r, h) converts
    // the 16 values l' = 16h .. 16h+15 of row r
    const int tid = threadIdx.x - 32 * kFirstSplitWarp;
    const int r = tid & 127, h = tid >> 7;
    uint32_t c = 0;
    for (int t = 0; t < nt; ++t) {
      const int am = abs_m(s_tiles[t].x);
      const int kcp = s_kc[am] & 0xff, kcq = s_kc[am] >> 8;
      bool ok = true;
      for (int ch = 0; ch < kcp + kcq; ++ch, ++c) {
        const int st = c % kStagingLegI;
        if (!mbar_wait(stgf + st, (c / kStagingLegI) & 1, abort_flag)) { ok = false; break; }
        float v[16];
        const float* sp = (const float*)(stg + st * kChunk) + 16 * h * 128;
#pragma unroll
        for (int k = 0; k < 16; ++k) v[k] = sp[k * 128 + r];
        mbar_arrive(stge + st);
        const int s = c % kStagesLegI;
        if (!mbar_wait(empty + s, ((c / kStagesLegI) & 1) ^ 1, abort_flag)) { ok = false; break; }
        if (BF) split_store_bf<4>(xs + s * 2 * kChunk, xs + s * 2 * kChunk + kChunk, r, v, 4 * h);
        else split_store<4>(xs + s * 2 * kChunk, xs + s * 2 * kChunk + kChunk, r, v, 4 * h, a.nprod == 3);
        fence_proxy_async();
        mbar_arrive(split + s);
      }
      if (!ok) break;
    }
  } else {
    const int quarter = warp & 3;
    const int ehalf = (warp - kFirstEpiWarp) >> 2;  // alternate 16-column blocks
    const int r_in = quarter * 32 + lane;
    uint32_t tcount = 0;
    for (int t = 0; t < nt; ++t, ++tcount) {
      const int2 tl = s_tiles[t];
      const int acc = tcount & 1;
      if (!mbar_wait(accf + acc, (tcount >> 1) & 1, abort_flag)) break;
      tc_after();
      const int m_idx = tl.x;
      const int m = m_idx - (B - 1);
      const int am = m < 0 ? -m : m;
      const int kcp = s_kc[am] & 0xff, kcq = s_kc[am] >> 8;
      const float sgn = (m < 0 && (am & 1)) ? -1.f : 1.f;
      const int jh = tl.y & 1;
      const int ncols = jh ? npad - 64 : nh;
      const int grow = (tl.y & ~1) + r_in;
      const bool valid = grow < NB * 2 * B;
      const int b = grow / (2 * B), cc = (grow / B) & 1, i = grow % B;
      float* out = a.g + (((int64_t)m_idx * NB + b) * 2 + cc) * (2 * B) * B + i;
      const uint32_t lanes = (uint32_t)(quarter * 32) << 16;
      const uint32_t dP = tmem + (uint32_t)(4 * acc * nh) + lanes;
      const uint32_t dQ = dP + (uint32_t)(2 * nh);
      for (int c0 = 16 * ehalf; c0 < ncols; c0 += 32) {
        float P[16], Q[16];
        if (a.nprod == 1) {
          tmem_ld16x2(dP + (uint32_t)c0, dQ + (uint32_t)c0, P, Q);
        } else {
          if (kcp) tmem_ld16_sum(dP + (uint32_t)c0, dP + (uint32_t)(nh + c0), P);
          if (kcq) tmem_ld16_sum(dQ + (uint32_t)c0, dQ + (uint32_t)(nh + c0), Q);
        }
        if (!kcp)
#pragma unroll
          for (int k = 0; k < 16; ++k) P[k] = 0.f;
        if (!kcq)
#pragma unroll
          for (int k = 0; k < 16; ++k) Q[k] = 0.f;
        if (valid) {
#pragma unroll
          for (int k = 0; k < 16; ++k) {
            const int j = jh * 64 + c0 + k;
            if (j < B) {
              out[(int64_t)j * B] = sgn * (P[k] + Q[k]);
              out[(int64_t)(2 * B - 1 - j) * B] = sgn * (P[k] - Q[k]);
            }
          }
        }
      }
      tc_before();
      mbar_arrive(acce + acc);
    }
  }
  __syncthreads();
  if (*abort_flag) {
    if (threadIdx.x == 0) atomicExch(a.err, 1);
    const uint64_t t0 = gtimer();
    while (gtimer() - t0 < 20000000ull) {
    }
  }
  tc_after();
  if (warp == 1) tmem_dealloc(tmem, tmem_cols);
}

// ===========================================================================
// inverse radial
// ===========================================================================
// Tiles of degrees with more than 64 terms (B - l > 64) are 64 columns wide
// and keep two main/correction pairs (even and odd K steps, one per MMA
// issuer), so that no accumulator takes more than 8 truncating additions of
// hi*hi products; the other tiles are 128 columns wide, one pair per half of
// 64 columns and issuer.  Either way a tile uses 256 TMEM columns, two tiles
// in flight.
struct RadIArgs {
  const int2* tiles;          // (l, col0 | narrow), grouped by l
  const int* cta_first;       // tile slice of each CTA (gridDim.x + 1 offsets)
  int ntiles;
  const unsigned char* tabimg;
  const int64_t* l_off;       // image offset per l (KC_l chunk pairs of 32 KB)
  const int64_t* si_rows;     // S row offset per (m_idx, p)
  const float* coef;          // complex interleaved coefficients
  const int64_t* fn_coef;     // coefficient offset per function of the segment
  float* s;                   // output S, layout [m_idx][p][l'][b][c][i]
  int* err;
  int B, NB;
  int nprod;                  // TF32 products per K step: 3 or 1 (hi*hi)
};

// Coefficients of one K chunk (32 degrees n) of one tile column, gathered by
// split thread tid: 16 (wide tile) or 8 (narrow tile) consecutive degrees.
__device__ __forceinline__ void rad_gather(const RadIArgs& a, int2 tl, int kc, int tid, float* v) {
  const int B = a.B, l = tl.x;
  const bool nar = tl.y & 1;
  const int col_in = nar ? (tid & 63) : (tid & 127);
  const int h = nar ? (tid >> 6) : (tid >> 7);
  const int nv = nar ? 8 : 16;
  const int per_b = (2 * l + 1) * 2;
  const int col = (tl.y & ~1) + col_in;
  const bool valid = col < a.NB * per_b;
  const int b = valid ? col / per_b : 0;
  const int rem = col - b * per_b;
  const int m = (rem >> 1) - l, cc = rem & 1;
  const float* cf = a.coef + 2 * a.fn_coef[b] + cc;
  const int np0 = kc * 32 + h * nv;        // degree n = l + 1 + n'
  int n = l + 1 + np0;
  int64_t off = omega_of(n, l, m);          // omega(n + 1) - omega(n) = n^2
#pragma unroll
  for (int k = 0; k < 16; ++k) {
    if (k < nv) {
      v[k] = (valid && np0 + k < B - l) ? cf[2 * off] : 0.f;
      off += (int64_t)n * n;
      ++n;
    }
  }
}

template <bool BF>
__global__ void __launch_bounds__(kThreadsInv, 1) tc_rad_inv_kernel(RadIArgs a) {
  constexpr int ROWB = BF ? 64 : 128;  // bytes of one operand row of a 32-value K chunk
  constexpr int TCH = 128 * ROWB;      // one table chunk (hi or lo): 128 rows i
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char* base = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  const int B = a.B, NB = a.NB;
  // stage s: [table hi][table lo][data], 16 KB each part (BF16: the table
  // parts use their first 8 KB; data halves of 64 columns are 64 hi rows over
  // 64 lo rows, 16 KB (TF32) or 8 KB (BF16) each)
  unsigned char* st = base;
  uint64_t* bars = (uint64_t*)(st + kStagesRadI * 4 * kChunk);
  uint64_t* tfull = bars;                   // [S] table chunk landed
  uint64_t* split = tfull + kStagesRadI;    // [S] data ready (split threads)
  uint64_t* empty = split + kStagesRadI;    // [S] MMAs done
  uint64_t* accf = empty + kStagesRadI;     // [2]
  uint64_t* acce = accf + 2;                // [2] (epilogue threads)
  uint32_t* tmem_slot = (uint32_t*)(acce + 2);
  volatile int* abort_flag = (volatile int*)(tmem_slot + 1);
  int64_t* s_si = (int64_t*)(bars + 64);          // [(2B-1)*2] S row offsets
  int64_t* s_loff = s_si + 2 * (2 * B - 1);        // [B] table image offsets
  int2* s_tiles = (int2*)(s_loff + B);
  for (int k = threadIdx.x; k < 2 * (2 * B - 1); k += blockDim.x) s_si[k] = a.si_rows[k];
  for (int k = threadIdx.x; k < B; k += blockDim.x) s_loff[k] = a.l_off[k];

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const uint32_t tmem_cols = 512;  // 2 buffers x 256 columns
  if (threadIdx.x == 0) {
    for (int s = 0; s < kStagesRadI; ++s) {
      mbar_init(tfull + s, 1);
      mbar_init(split + s, kSplitThreads);
      mbar_init(empty + s, 2);  // both MMA issuers
    }
    for (int k = 0; k < 2; ++k) {
      mbar_init(accf + k, 2);
      mbar_init(acce + k, kEpiThreads);
    }
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) tmem_alloc(tmem_slot, tmem_cols);
  const int g_begin = a.cta_first[blockIdx.x];
  const int nt = a.cta_first[blockIdx.x + 1] - g_begin;
  for (int k = threadIdx.x; k < nt; k += blockDim.x) s_tiles[k] = a.tiles[g_begin + k];
  tc_before();
  __syncthreads();
  tc_after();
  const uint32_t tmem = *tmem_slot;

  if (warp == 0) {
    if (lane == 0) {
      uint32_t c = 0;
      for (int t = 0; t < nt && !*abort_flag; ++t) {
        const int l = s_tiles[t].x;
        const int kcn = (B - l + 31) / 32;
        bool ok = true;
        for (int kc = 0; kc < kcn; ++kc, ++c) {
          const int s = c % kStagesRadI;
          if (!mbar_wait(empty + s, ((c / kStagesRadI) & 1) ^ 1, abort_flag)) { ok = false; break; }
          // hi and lo chunk of the image, contiguous; the lo part lands at +kChunk
          mbar_arrive_tx(tfull + s, 2 * TCH);
          bulk_load(st + s * 4 * kChunk, a.tabimg + s_loff[l] + (int64_t)kc * 2 * TCH, TCH, tfull + s);
          bulk_load(st + s * 4 * kChunk + kChunk, a.tabimg + s_loff[l] + (int64_t)kc * 2 * TCH + TCH, TCH, tfull + s);
        }
        if (!ok) break;
      }
    }
  } else if (warp == 1 || warp == kMma2Warp) {
    // MMA issuer `me`: narrow tiles, the K steps of parity me into
    // [main_me | corr_me]; wide tiles, the columns 64 me .. 64 me + 63
    if (lane == 0) {
      const int me = warp == 1 ? 0 : 1;
      uint32_t c = 0, tcount = 0;
      const uint64_t sdesc0 = BF ? sw64_desc(smem_u32(st)) : sw128_desc(smem_u32(st));
      // B operand of each half: 64 hi rows over 64 lo rows.  One MMA of width
      // 128 gives [T_hi X_hi | T_hi X_lo], a second of width 64 adds T_lo X_hi.
      const uint32_t idesc2 = BF ? idesc_bf16(128) : idesc_tf32(128);
      const uint32_t idesc1 = BF ? idesc_bf16(64) : idesc_tf32(64);
      for (int t = 0; t < nt && !*abort_flag; ++t, ++tcount) {
        const int2 tl = s_tiles[t];
        const int l = tl.x;
        const bool nar = tl.y & 1;
        const int kcn = (B - l + 31) / 32;
        const int acc = tcount & 1;
        if (!mbar_wait(acce + acc, ((tcount >> 1) & 1) ^ 1, abort_flag)) break;
        tc_after();
        // buffer: [main0 | corr0 | main1 | corr1], 64 columns each
        const uint32_t dm = tmem + (uint32_t)(acc * 256 + me * 128);
        const uint32_t dc = dm + 64u;
        bool ok = true;
        for (int kc = 0; kc < kcn; ++kc, ++c) {
          const int s = c % kStagesRadI;
          const uint32_t ph = (c / kStagesRadI) & 1;
          if (!mbar_wait(tfull + s, ph, abort_flag) || !mbar_wait(split + s, ph, abort_flag)) {
            ok = false;
            break;
          }
          tc_after();
          const uint64_t ah = sdesc0 + (uint64_t)((s * 4 * kChunk) >> 4);
          const uint64_t al = ah + (uint64_t)(kChunk >> 4);
          const uint64_t bh = al + (uint64_t)(kChunk >> 4) + (nar ? 0u : (uint64_t)(me * (128 * ROWB >> 4)));
          if (BF) {  // two K steps of 16: narrow, one per issuer; wide, both
            if (nar) {
              mma_bf16(dm, ah + 2 * me, bh + 2 * me, idesc2, kc > 0 ? 1u : 0u);
              mma_bf16(dc, al + 2 * me, bh + 2 * me, idesc1, 1u);
            } else {
#pragma unroll
              for (int kk = 0; kk < 2; ++kk) {
                mma_bf16(dm, ah + 2 * kk, bh + 2 * kk, idesc2, (kc > 0 || kk > 0) ? 1u : 0u);
                mma_bf16(dc, al + 2 * kk, bh + 2 * kk, idesc1, 1u);
              }
            }
          } else if (a.nprod == 1) {  // hi*hi only: the B operand's hi rows, main accumulator
            if (nar) {
              mma_tf32(dm, ah + 2 * me, bh + 2 * me, idesc1, kc > 0 ? 1u : 0u);
              mma_tf32(dm, ah + 2 * me + 4, bh + 2 * me + 4, idesc1, 1u);
            } else {
#pragma unroll
              for (int kk = 0; kk < 4; ++kk)
                mma_tf32(dm, ah + 2 * kk, bh + 2 * kk, idesc1, (kc > 0 || kk > 0) ? 1u : 0u);
            }
          } else if (nar) {
            const uint32_t first = kc > 0 ? 1u : 0u;
            mma_tf32(dm, ah + 2 * me, bh + 2 * me, idesc2, first);
            mma_tf32(dc, al + 2 * me, bh + 2 * me, idesc1, 1u);
            mma_tf32(dm, ah + 2 * me + 4, bh + 2 * me + 4, idesc2, 1u);
            mma_tf32(dc, al + 2 * me + 4, bh + 2 * me + 4, idesc1, 1u);
          } else {
#pragma unroll
            for (int kk = 0; kk < 4; ++kk) {
              const uint32_t first = (kc > 0 || kk > 0) ? 1u : 0u;
              mma_tf32(dm, ah + 2 * kk, bh + 2 * kk, idesc2, first);
              mma_tf32(dc, al + 2 * kk, bh + 2 * kk, idesc1, 1u);
            }
          }
          mma_commit(empty + s);
        }
        if (!ok) break;
        mma_commit(accf + acc);
      }
    }
  } else if (warp < kFirstEpiWarp) {
    // gather: thread (column, h) loads 16 (wide) or 8 (narrow) consecutive
    // degrees of its column per chunk; the next chunk's loads are issued
    // before the current chunk is split and stored
    const int tid = threadIdx.x - 32 * kFirstSplitWarp;
    float v[16], vn[16];
    int t = 0, kc = 0;
    if (nt > 0) rad_gather(a, s_tiles[0], 0, tid, v);
    for (uint32_t c = 0; t < nt; ++c) {
      const int2 tl = s_tiles[t];
      const bool nar = tl.y & 1;
      int tn = t, kcn_next = kc + 1;
      if (kcn_next == (B - tl.x + 31) / 32) {
        tn = t + 1;
        kcn_next = 0;
      }
      if (tn < nt) rad_gather(a, s_tiles[tn], kcn_next, tid, vn);
      const int s = c % kStagesRadI;
      if (!mbar_wait(empty + s, ((c / kStagesRadI) & 1) ^ 1, abort_flag)) break;
      // B operand: per half of 64 columns, 64 hi rows then 64 lo rows
      unsigned char* sb = st + s * 4 * kChunk + 2 * kChunk;
      if (BF) {
        if (nar) {
          split_store_bf<2>(sb, sb + 64 * ROWB, tid & 63, v, 2 * (tid >> 6));
        } else {
          unsigned char* hb = sb + ((tid >> 6) & 1) * (128 * ROWB);
          split_store_bf<4>(hb, hb + 64 * ROWB, tid & 63, v, 4 * (tid >> 7));
        }
      } else if (nar) {
        split_store<2>(sb, sb + 64 * ROWB, tid & 63, v, 2 * (tid >> 6), a.nprod == 3);
      } else {
        unsigned char* hb = sb + ((tid >> 6) & 1) * (128 * ROWB);
        split_store<4>(hb, hb + 64 * ROWB, tid & 63, v, 4 * (tid >> 7), a.nprod == 3);
      }
      fence_proxy_async();
      mbar_arrive(split + s);
#pragma unroll
      for (int k = 0; k < 16; ++k) v[k] = vn[k];
      t = tn;
      kc = kcn_next;
    }
  } else {
    const int quarter = warp & 3;
    const int ehalf = (warp - kFirstEpiWarp) >> 2;  // alternate 16-column blocks
    const int i = quarter * 32 + lane;   // TMEM lane = radius index
    uint32_t tcount = 0;
    for (int t = 0; t < nt; ++t, ++tcount) {
      const int2 tl = s_tiles[t];
      const int acc = tcount & 1;
      if (!mbar_wait(accf + acc, (tcount >> 1) & 1, abort_flag)) break;
      tc_after();
      const int l = tl.x;
      const bool nar = tl.y & 1;
      const int col0 = tl.y & ~1;
      const int width = nar ? 64 : 128;
      const int per_b = (2 * l + 1) * 2;
      const uint32_t dq = tmem + (uint32_t)(acc * 256) + ((uint32_t)(quarter * 32) << 16);
      for (int c0 = 16 * ehalf; c0 < width; c0 += 32) {
        // lane k < 16 finds the S offset of column c0 + k (b, m, c); the
        // stores take it by shuffle
        int64_t o = -1;
        {
          const int col = col0 + c0 + (lane & 15);
          if (col < NB * per_b) {
            const int b = col / per_b, rem = col - b * per_b;
            const int m = (rem >> 1) - l, cc = rem & 1;
            const int am = m < 0 ? -m : m;
            const int p = (l - am) & 1;
            const int64_t srow = s_si[2 * (m + B - 1) + p] + ((l - am - p) >> 1);
            o = srow * ((int64_t)NB * 2 * B) + ((int64_t)b * 2 + cc) * B;
          }
        }
        float v[16];
        if (nar) {
          const uint32_t tc = dq + (uint32_t)c0;
          if (a.nprod == 3) {
            tmem_ld16_sum4(tc, tc + 128u, tc + 64u, tc + 192u, v);
          } else {
            tmem_ld16_sum(tc, tc + 128u, v);  // main0 + main1
          }
        } else {  // columns 64h + c: [main_h | corr_h] at 128 h
          const uint32_t tc = dq + (uint32_t)((c0 >> 6) * 128 + (c0 & 63));
          if (a.nprod == 3) tmem_ld16_sum(tc, tc + 64u, v);
          else tmem_ld16(tc, v);
        }
#pragma unroll
        for (int k = 0; k < 16; ++k) {
          const int64_t ok = __shfl_sync(0xffffffffu, o, k);
          if (i < B && ok >= 0) a.s[ok + i] = v[k];
        }
      }
      tc_before();
      mbar_arrive(acce + acc);
    }
  }
  __syncthreads();
  if (*abort_flag) {
    if (threadIdx.x == 0) atomicExch(a.err, 1);
    const uint64_t t0 = gtimer();
    while (gtimer() - t0 < 20000000ull) {
    }
  }
  tc_after();
  if (warp == 1) tmem_dealloc(tmem, tmem_cols);
}

// ===========================================================================
// host side
// ===========================================================================
namespace {

uint32_t rna_bits(float x) {
  uint32_t u;
  memcpy(&u, &x, 4);
  return (u + 0x1000u) & 0xFFFFE000u;
}

// Append KC chunks of `rows` x 32 floats, 128-byte swizzled, each as its hi
// rows followed by its lo rows: value(row, k) for k < K.
template <typename F>
void append_planes(std::vector<unsigned char>& img, int rows, int K, int KC, F value) {
  const size_t off = img.size();
  const size_t plane = (size_t)rows * 128;
  img.resize(off + 2 * (size_t)KC * plane, 0);
  for (int r = 0; r < rows; ++r)
    for (int k = 0; k < K; ++k) {
      const double v = value(r, k);
      if (v == 0.0) continue;
      const float f = (float)v;
      const uint32_t hb = rna_bits(f);
      float hi;
      memcpy(&hi, &hb, 4);
      const uint32_t lb = rna_bits((float)(v - (double)hi));
      const int kc = k / 32, kin = k % 32;
      const size_t pos = (size_t)kc * 2 * plane + (size_t)r * 128 + (size_t)((((kin >> 2) ^ (r & 7)) << 4) + (kin & 3) * 4);
      memcpy(&img[off + pos], &hb, 4);
      memcpy(&img[off + plane + pos], &lb, 4);
    }
}

uint16_t bf16_rn_bits(float x) {
  uint32_t u;
  memcpy(&u, &x, 4);
  return (uint16_t)((u + 0x7FFFu + ((u >> 16) & 1u)) >> 16);
}

// BF16 form of append_planes: per chunk the hi rows, then the lo rows, each
// row 32 values in 64 bytes with the 64-byte swizzle.
template <typename F>
void append_planes_bf16(std::vector<unsigned char>& img, int rows, int K, int KC, F value) {
  const size_t off = img.size();
  const size_t plane = (size_t)rows * 64;
  img.resize(off + 2 * (size_t)KC * plane, 0);
  for (int r = 0; r < rows; ++r)
    for (int k = 0; k < K; ++k) {
      const double v = value(r, k);
      if (v == 0.0) continue;
      const uint16_t hb = bf16_rn_bits((float)v);
      const uint32_t hu = (uint32_t)hb << 16;
      float hi;
      memcpy(&hi, &hu, 4);
      const uint16_t lb = bf16_rn_bits((float)(v - (double)hi));
      const int kc = k / 32, kin = k % 32;
      const size_t pos = (size_t)kc * 2 * plane + (size_t)r * 64 + (size_t)((((kin >> 3) ^ ((r >> 1) & 3)) << 4) + (kin & 7) * 2);
      memcpy(&img[off + pos], &hb, 2);
      memcpy(&img[off + plane + pos], &lb, 2);
    }
}

int pad16i(int n) { return n <= 16 ? 16 : (n + 15) / 16 * 16; }

}  // namespace

struct TcInvSeg {
  // Legendre
  CUtensorMap smap;
  int2* leg_tiles = nullptr;
  int* leg_first = nullptr;
  int leg_ntiles = 0, leg_grid = 0;
  size_t leg_smem = 0;
  int64_t* am_off = nullptr;
  int* am_kc = nullptr;
  int npad = 0, kcmax = 0;
  // radial
  int2* rad_tiles = nullptr;
  int* rad_first = nullptr;
  int rad_ntiles = 0, rad_grid = 0;
  size_t rad_smem = 0;
  int64_t* l_off = nullptr;
};

struct TcInvState {
  std::vector<TcInvSeg> segs;
  unsigned char* d_img = nullptr;
};

bool make_map_2d(CUtensorMap* map, void* base, uint64_t inner, uint64_t rows, uint32_t box_inner, uint32_t box_rows,
                 CUtensorMapSwizzle sw);

template <typename T>
static cudaError_t upload(T** dst, const std::vector<T>& v, int64_t& bytes) {
  cudaError_t e = cudaMalloc((void**)dst, v.size() * sizeof(T) + 16);
  if (e != cudaSuccess) return e;
  bytes += v.size() * sizeof(T);
  return cudaMemcpy(*dst, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice);
}

// Inverse radial tiles of segment s: 64 columns with two K chains where
// B - l >= P.radi_narrow, else 128 columns; the CTA slices and shared memory.
static cudaError_t radi_tiles(const Plan& P, size_t s, TcInvSeg& ts, int nsm, int64_t& bytes) {
  const int B = P.segs[s].B, NB = P.segs[s].NB;
  std::vector<int2> rtiles;
  std::vector<double> rc;
  for (int l = 0; l < B; ++l) {
    const int nar = B - l >= P.radi_narrow ? 1 : 0;
    const int width = nar ? 64 : 128;
    const int kcn = (B - l + 31) / 32;
    for (int c0 = 0; c0 < NB * (2 * l + 1) * 2; c0 += width) {
      rtiles.push_back(make_int2(l, c0 | nar));
      // gathered coefficients, table chunks (from L2, half weight), S out
      rc.push_back(kcn * (width * 128.0 + 16384.0) + 512.0 * width);
    }
  }
  cudaError_t e = upload(&ts.rad_tiles, rtiles, bytes);
  ts.rad_ntiles = (int)rtiles.size();
  ts.rad_grid = std::min(ts.rad_ntiles, nsm);
  int rmax = 0;
  const std::vector<int> rf = balance_slices(rc, std::max(ts.rad_grid, 1), &rmax);
  if (e == cudaSuccess) e = upload(&ts.rad_first, rf, bytes);
  const size_t meta = (size_t)2 * (2 * B - 1) * 8 + (size_t)B * 12 + 8;
  ts.rad_smem = 1024 + (size_t)kStagesRadI * 4 * kChunk + 64 * 8 + meta + (size_t)(rmax + 1) * 8;
  if (e == cudaSuccess && ts.rad_smem > 227 * 1024) e = cudaErrorInvalidValue;
  return e;
}

cudaError_t tc_radi_retile(Plan& P) {
  TcInvState* st = (TcInvState*)P.tc_inv_state;
  if (!st) return cudaSuccess;
  int dev = 0, nsm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  int64_t bytes = 0;
  for (size_t s = 0; s < st->segs.size(); ++s) {
    TcInvSeg& ts = st->segs[s];
    if (ts.rad_tiles) {
      cudaFree(ts.rad_tiles);
      P.bytes -= (int64_t)ts.rad_ntiles * sizeof(int2);
    }
    if (ts.rad_first) {
      cudaFree(ts.rad_first);
      P.bytes -= (int64_t)(ts.rad_grid > 0 ? ts.rad_grid + 1 : 2) * sizeof(int);
    }
    ts.rad_tiles = nullptr;
    ts.rad_first = nullptr;
    cudaError_t e = radi_tiles(P, s, ts, nsm, bytes);
    if (e != cudaSuccess) {
      P.bytes += bytes;
      return e;
    }
  }
  P.bytes += bytes;
  return cudaSuccess;
}

cudaError_t tc_inv_prepare(Plan& P) {
  int dev = 0, nsm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  TcInvState* st = new TcInvState();
  const bool bf = tc_bf16(P.prec);
  std::vector<unsigned char> img;
  std::vector<std::vector<int64_t>> am_offs, l_offs;
  std::vector<std::vector<int>> am_kcs;
  std::vector<std::vector<int2>> lt;
  std::vector<std::vector<double>> lcost;  // estimated bytes moved per tile
  for (size_t s = 0; s < P.segs.size(); ++s) {
    const SegDesc& sg = P.segs[s];
    const HostTables& H = P.tables[s];
    const int B = sg.B, NB = sg.NB;
    TcInvSeg ts;
    ts.npad = pad16i(B);
    // Legendre synthesis tables, per (|m|, j'-half of 64 rows):
    // [P hi][P lo][Q hi][Q lo], rows j', K = l'
    const int nh = ts.npad > 64 ? 64 : ts.npad;
    const int halves = (ts.npad + 63) / 64;
    std::vector<int64_t> aoff(2 * B, 0);
    std::vector<int> akc(B, 0);
    int kcmax = 1;
    for (int am = 0; am < B; ++am) {
      int kcs[2];
      for (int p = 0; p < 2; ++p) kcs[p] = (n_par(B, am, p) + 31) / 32;
      for (int jh = 0; jh < halves; ++jh) {
        img.resize((img.size() + 1023) / 1024 * 1024);
        aoff[2 * am + jh] = (int64_t)img.size();
        for (int p = 0; p < 2; ++p) {
          if (kcs[p] == 0) continue;
          auto lam = [&](int jr, int q) -> double {
            const int j = 64 * jh + jr;
            if (j >= B) return 0.0;
            const int l = am + p + 2 * q;
            return H.lam[((size_t)am * B + l) * B + j];
          };
          if (bf) append_planes_bf16(img, nh, n_par(B, am, p), kcs[p], lam);
          else append_planes(img, nh, n_par(B, am, p), kcs[p], lam);
        }
      }
      akc[am] = kcs[0] | (kcs[1] << 8);
      kcmax = std::max(kcmax, kcs[0] + kcs[1]);
    }
    ts.kcmax = kcmax;
    std::vector<int2> ltiles;
    std::vector<double> lc;
    for (int mi = 0; mi < 2 * B - 1; ++mi) {
      const int am = mi < B - 1 ? B - 1 - mi : mi - (B - 1);
      const int kcs = (akc[am] & 0xff) + (akc[am] >> 8);
      for (int jh = 0; jh < halves; ++jh)
        for (int r0 = 0; r0 < NB * 2 * B; r0 += 128) {
          ltiles.push_back(make_int2(mi, r0 | jh));
          // S chunks in, both G halves out, the table on its first tile
          const int ncols = jh ? ts.npad - 64 : nh;
          lc.push_back(kcs * 16384.0 + 1024.0 * ncols + (r0 == 0 ? 2.0 * kcs * nh * 128 : 0.0));
        }
    }
    // radial inverse tables, per l: KC_l x [hi chunk][lo chunk], rows i (128), K = n'
    std::vector<int64_t> loff(B, 0);
    for (int l = 0; l < B; ++l) {
      img.resize((img.size() + 1023) / 1024 * 1024);
      loff[l] = (int64_t)img.size();
      const int K = B - l, KC = (K + 31) / 32;
      for (int kc = 0; kc < KC; ++kc) {
        auto tv = [&](int i, int k) -> double {
          const int np = kc * 32 + k;
          if (i >= B || np >= K) return 0.0;
          return H.T[((size_t)l * B + (l + np)) * B + i];
        };
        if (bf) append_planes_bf16(img, 128, 32, 1, tv);
        else append_planes(img, 128, 32, 1, tv);
      }
    }
    // tensor map over S: [B^2 rows of l'][NB*2*B]
    float* w2 = (float*)P.d_w2 + sg.w2_off;
    if (!make_map_2d(&ts.smap, w2, (uint64_t)NB * 2 * B, (uint64_t)B * B, 128, 32, CU_TENSOR_MAP_SWIZZLE_NONE)) {
      delete st;
      return cudaErrorInvalidValue;
    }
    st->segs.push_back(ts);
    am_offs.push_back(aoff);
    am_kcs.push_back(akc);
    l_offs.push_back(loff);
    lt.push_back(ltiles);
    lcost.push_back(lc);
  }
  int64_t bytes = 0;
  cudaError_t e = upload(&st->d_img, img, bytes);
  for (size_t s = 0; s < st->segs.size() && e == cudaSuccess; ++s) {
    TcInvSeg& ts = st->segs[s];
    const int B = P.segs[s].B;
    e = upload(&ts.am_off, am_offs[s], bytes);
    if (e == cudaSuccess) e = upload(&ts.am_kc, am_kcs[s], bytes);
    if (e == cudaSuccess) e = upload(&ts.l_off, l_offs[s], bytes);
    if (e == cudaSuccess) e = upload(&ts.leg_tiles, lt[s], bytes);
    ts.leg_ntiles = (int)lt[s].size();
    ts.leg_grid = std::min(ts.leg_ntiles, nsm);
    int lmax = 0;
    const std::vector<int> lf = balance_slices(lcost[s], std::max(ts.leg_grid, 1), &lmax);
    if (e == cudaSuccess) e = upload(&ts.leg_first, lf, bytes);
    lmax += 1;
    if (e == cudaSuccess) e = radi_tiles(P, s, ts, nsm, bytes);
    // tables, staging, operand ring, barrier slots, metadata (S row offsets,
    // image offsets, chunk counts), tile slice
    const size_t meta = (size_t)2 * (2 * B - 1) * 8 + (size_t)B * 12 + 8;
    const int nh_s = ts.npad > 64 ? 64 : ts.npad;
    ts.leg_smem = 1024 + (size_t)ts.kcmax * 2 * nh_s * (bf ? 64 : 128) + (size_t)kStagingLegI * kChunk +
                  (size_t)kStagesLegI * 2 * kChunk + 64 * 8 + meta + (size_t)B * 8 + (size_t)lmax * 8;
    if (ts.leg_smem > 227 * 1024) e = cudaErrorInvalidValue;
  }
  P.bytes += bytes;
  if (e != cudaSuccess) {
    P.tc_inv_state = st;
    return e;
  }
  P.tc_inv_state = st;
  return cudaSuccess;
}

void tc_inv_release(Plan& P) {
  TcInvState* st = (TcInvState*)P.tc_inv_state;
  if (!st) return;
  for (TcInvSeg& s : st->segs) {
    void* ptrs[] = {s.leg_tiles, s.leg_first, s.am_off, s.am_kc, s.rad_tiles, s.rad_first, s.l_off};
    for (void* p : ptrs)
      if (p) cudaFree(p);
  }
  if (st->d_img) cudaFree(st->d_img);
  delete st;
  P.tc_inv_state = nullptr;
}

// prob 2: inverse radial (x = coefficients, y = S); prob 3: inverse Legendre (x = S, y = G)
cudaError_t run_tc_inverse(Plan& P, int prob, const void* x, void* y, cudaStream_t s) {
  TcInvState* st = (TcInvState*)P.tc_inv_state;
  if (!st) return cudaErrorNotSupported;
  StageTimer timer(P, prob == 2 ? ST_RAD_I : ST_LEG_I, s);
  for (size_t k = 0; k < st->segs.size(); ++k) {
    TcInvSeg& ts = st->segs[k];
    const SegDesc& sg = P.segs[k];
    cudaError_t e;
    if (prob == 2) {
      RadIArgs a;
      a.tiles = ts.rad_tiles;
      a.cta_first = ts.rad_first;
      a.ntiles = ts.rad_ntiles;
      a.tabimg = st->d_img;
      a.l_off = ts.l_off;
      a.si_rows = P.d_si_rows + sg.si_rows;
      a.coef = (const float*)x;
      a.fn_coef = P.d_fn_coef + sg.fn0;
      a.s = (float*)y + sg.w2_off;
      a.err = P.d_err;
      a.B = sg.B;
      a.NB = sg.NB;
      a.nprod = tc_products(P.prec);
      void (*fn)(RadIArgs) = tc_bf16(P.prec) ? tc_rad_inv_kernel<true> : tc_rad_inv_kernel<false>;
      e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)ts.rad_smem);
      if (e != cudaSuccess) return e;
      fn<<<ts.rad_grid, kThreadsInv, ts.rad_smem, s>>>(a);
    } else {
      LegIArgs a;
      a.tiles = ts.leg_tiles;
      a.cta_first = ts.leg_first;
      a.ntiles = ts.leg_ntiles;
      a.tabimg = st->d_img;
      a.am_off = ts.am_off;
      a.am_kc = ts.am_kc;
      a.si_rows = P.d_si_rows + sg.si_rows;
      a.g = (float*)y + sg.w1_off;
      a.err = P.d_err;
      a.B = sg.B;
      a.NB = sg.NB;
      a.npad = ts.npad;
      a.kcmax = ts.kcmax;
      a.nprod = tc_products(P.prec);
      void (*fn)(const CUtensorMap, LegIArgs) = tc_bf16(P.prec) ? tc_leg_inv_kernel<true> : tc_leg_inv_kernel<false>;
      e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)ts.leg_smem);
      if (e != cudaSuccess) return e;
      fn<<<ts.leg_grid, kThreadsInv, ts.leg_smem, s>>>(ts.smap, a);
    }
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  timer.finish();
  return cudaSuccess;
}

}  // namespace sgl
