// Tensor-core inverse stages (tcgen05, TMEM, TMA) of the SGL transform:
// TF32x3 (and its hi*hi-only and BF16 hi/lo variants).
//
// Inverse radial stage (iDRT, R_l^T of Sect. 3.3.2), one GEMM per degree l:
//   S[i][col] = sum_{n'} T_{l+1+n',l}(i) fhat[col][n'],  col = (b, m, c)
//   A operand: the table, M = 128 rows i, streamed per K chunk by bulk copy;
//   B operand: coefficients gathered by the split warps (N = 128 columns).
//   S is stored [l'][b][i][c]: the (re, im) columns of one (b, m) go out as
//   one 8-byte pair per radius.
// Inverse Legendre stage (the inner sum of Eq. iSFFT_rearranged), one tile
// per (m, 128 rows (b, i, c)) with both theta-parities:
//   P[row][j'] = sum_{l' even} S[row][l'] Lambda(theta_j'),  Q likewise for odd,
//   G_j' = P + Q,  G_{2B-1-j'} = P - Q   (Lambda(pi - theta) = (-1)^{l+m} Lambda(theta)).
//   A operand: S rows, loaded l'-major by TMA into a staging ring and
//   transposed to K-major hi/lo by the split warps; B operand: the table.
// Same role layout as the forward kernels (tc_ptx.cuh): producer warp, two
// MMA-issuing warps (the first owns tensor memory), split warps, epilogue
// warps; bounded waits.  Each launch covers every bandlimit segment of the
// plan: tiles carry their segment.
#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include <algorithm>
#include <cmath>
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
constexpr int kStagesRadI = 2;
// coefficient gather of the inverse radial stage: chunks in flight per split
// thread (asynchronous copies), and staging slots ([16 values][256 threads])
constexpr int kGatherDepth = 2;
constexpr int kGatherSlots = kGatherDepth + 1;
constexpr int kGatherSlotBytes = 16 * 256 * 4;

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

// 16-bit form: 4*NQ consecutive K values of one row (NQ even) as BF16 hi/lo
// pairs, or (F16) FP16 pairs of the values times the power of two f, at
// 16-byte chunks q0/2 .. q0/2 + NQ/2 - 1 of 64-byte rows.
template <int NQ, bool F16>
__device__ __forceinline__ void split_store_bf(unsigned char* hi, unsigned char* lo, int row, const float* v,
                                               int q0, float f) {
#pragma unroll
  for (int j = 0; j < NQ / 2; ++j) {
    uint32_t hw[4], lw[4];
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      const float x0 = v[8 * j + 2 * e], x1 = v[8 * j + 2 * e + 1];
      if constexpr (F16) {
        fp16_split2(x0, x1, f, hw[e], lw[e]);
      } else {
        const uint32_t a = bf16_split(x0), b = bf16_split(x1);
        hw[e] = (a & 0xFFFFu) | (b << 16);
        lw[e] = (a >> 16) | (b & 0xFFFF0000u);
      }
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
// read once per half.  The first MMA issuer takes the P chunks, the second
// the Q chunks.

// One bandlimit segment of a launch; a launch covers every segment of the
// plan.  Aligned as its tensor map.
struct LegISeg {
  CUtensorMap smap;           // the segment's S: [B^2 rows of l'][NB*2*B]
  int B, NB, npad, fn0;       // bandlimit, functions, padded j' count, first function
  float sb;                   // FP16x3: bound on |S| / largest |coefficient| (radial table)
  int pad;
  int64_t w1_off;             // the segment's G block
};
struct LegISegSmall {
  int B, NB, npad, fn0;
  float sb;
  int pad;
  int64_t w1_off;
};

struct LegIArgs {
  // per tile, two int4: (m_idx, row0, j'-half | segment << 8, KC_P | KC_Q << 8)
  // and (table image offset, S row of the P block, S row of the Q block, 0);
  // ordered by (segment, m_idx, half, row0)
  const int4* tiles;
  const int* slice_first;     // first tile of each work-queue slice (nslices + 1 offsets)
  int nslices;
  int* queue;                 // next slice to take; zero at launch
  int ntiles;
  const unsigned char* tabimg;
  const LegISeg* segs;
  int nseg;
  float* g;                   // output, per segment layout [m_idx][b][j < 2B][i][c]
  int* err;
  int npad_max, kcmax;        // over the segments
  int nprod;                  // TF32 products per K step: 3 or 1 (hi*hi)
  const unsigned* amax;       // FP16x3: per-function largest |coefficient| (segment order)
};

// OP: the operand format (TcOperand): TF32, or BF16 / scaled FP16 hi/lo pairs
// (kind::f16, 64-byte rows, K = 16 per MMA).  FP16 tables are scaled per image
// (exponent in the tile record), S per function (the coefficients' largest
// magnitude times the radial table's growth bound).
template <int OP>
__global__ void __launch_bounds__(kThreadsInv, 1) tc_leg_inv_kernel(LegIArgs a) {
  constexpr bool BF = OP != TC_OP_TF32;
  constexpr bool F16 = OP == TC_OP_FP16;
  constexpr int ROWB = BF ? 64 : 128;  // bytes of one operand row of a 32-value K chunk
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char* base = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  // rows (j') of one table half: per segment min(npad, 64); buffers sized for the largest
  const int nhm = a.npad_max > 64 ? 64 : a.npad_max;
  unsigned char* tab = base;                               // [P hi][P lo][Q hi][Q lo] of one half
  unsigned char* stg = tab + (size_t)a.kcmax * 2 * nhm * ROWB;   // staging ring: 32 l' x 128 rows each
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
  uint64_t* drain = bars + 62;                  // [2] MMA issuers' own barriers, used after an abort
  uint32_t* issued = (uint32_t*)(bars + 61);  // producer: [copies issued into the ring, table copies]
  // the segments, copied once, and the tiles of the current slice of the
  // work queue (two records per tile, capacity a.slice_cap), copied per slice
  // (see tc_gemm_kernel: slices from a global counter, role counters carried
  // over through s_cnt)
  LegISegSmall* s_seg = (LegISegSmall*)(bars + 64);
  int4* s_tiles = (int4*)(((uintptr_t)(s_seg + a.nseg) + 15) & ~(uintptr_t)15);
  // [0, 1] producer copies and tables; [2 + 3p, 3 + 3p, 4 + 3p] MMA issuer p
  // chunks, tiles, tables; [8] split chunks; [9] epilogue tiles
  uint32_t* s_cnt = (uint32_t*)(bars + 48);
  volatile int* s_slice = (volatile int*)(bars + 53);
  for (int k = threadIdx.x; k < a.nseg; k += blockDim.x) {
    const LegISeg& g = a.segs[k];
    s_seg[k] = LegISegSmall{g.B, g.NB, g.npad, g.fn0, g.sb, 0, g.w1_off};
  }

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  uint32_t tmem_cols = 32;
  while (tmem_cols < (uint32_t)(8 * nhm)) tmem_cols <<= 1;  // 2 buffers x {P, Q} x {main, corr}
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
    mbar_init(drain, 1);
    mbar_init(drain + 1, 1);
    issued[0] = issued[1] = 0u;
    for (int k = 0; k < 10; ++k) s_cnt[k] = 0u;
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) tmem_alloc(tmem_slot, tmem_cols);
  tc_before();
  __syncthreads();
  tc_after();
  const uint32_t tmem = *tmem_slot;

  for (;;) {
  if (threadIdx.x == 0) *s_slice = atomicAdd(a.queue, 1);
  __syncthreads();
  const int sl = *s_slice;
  if (sl >= a.nslices || *abort_flag) break;
  const int g_begin = a.slice_first[sl];
  const int nt = a.slice_first[sl + 1] - g_begin;
  for (int k = threadIdx.x; k < 2 * nt; k += blockDim.x) s_tiles[k] = a.tiles[2 * g_begin + k];
  tc_before();
  __syncthreads();
  tc_after();
  // tile t: s_tiles[2t] = (m_idx, row0, half | seg << 8, KC_P | KC_Q << 8),
  //         s_tiles[2t+1] = (table image offset, S row of P, S row of Q, 0);
  // the resident table changes with its image offset

  if (warp == 0) {
    if (lane == 0) {
      int cur = -1, ngrp = (int)s_cnt[1], cur_seg = -1;
      uint32_t c = s_cnt[0];
      for (int t = 0; t < nt && !*abort_flag; ++t) {
        const int4 ta = s_tiles[2 * t], tb = s_tiles[2 * t + 1];
        const int seg = ta.z >> 8;
        const int nh = min(s_seg[seg].npad, 64);
        const int kcp = ta.w & 0xff, kcq = ta.w >> 8;
        const CUtensorMap* smap = &a.segs[seg].smap;
        if (seg != cur_seg) {  // the tensor map lives in global memory
          asm volatile("fence.proxy.tensormap::generic.acquire.gpu [%0], 128;" ::"l"(smap) : "memory");
          cur_seg = seg;
        }
        if (tb.x != cur) {
          if (ngrp > 0 && !mbar_wait(tabe, (ngrp - 1) & 1, abort_flag)) break;
          const uint32_t bytes = (uint32_t)((kcp + kcq) * 2 * nh * ROWB);
          mbar_arrive_tx(tabf, bytes);
          bulk_load(tab, a.tabimg + (uint32_t)tb.x, bytes, tabf);
          cur = tb.x;
          ++ngrp;
        }
        bool ok = true;
        for (int p = 0; p < 2 && ok; ++p) {
          const int kcn = p ? kcq : kcp;
          const int r0 = p ? tb.z : tb.y;
          for (int kc = 0; kc < kcn; ++kc, ++c) {
            const int s = c % kStagingLegI;
            if (!mbar_wait(stge + s, ((c / kStagingLegI) & 1) ^ 1, abort_flag)) { ok = false; break; }
            mbar_arrive_tx(stgf + s, kChunk);
            tma_load_2d(stg + s * kChunk, smap, stgf + s, ta.y, r0 + kc * 32);
          }
        }
        if (!ok) break;
      }
      issued[0] = s_cnt[0] = c;
      issued[1] = s_cnt[1] = (uint32_t)ngrp;
    }
  } else if (warp == 1 || warp == kMma2Warp) {
    // MMA issuer `me` takes the chunks of parity p = me (P or Q accumulators)
    if (lane == 0) {
      const int p = warp == 1 ? 0 : 1;
      int cur = -1, ngrp = (int)s_cnt[4 + 3 * p];
      uint32_t c = s_cnt[2 + 3 * p], tcount = s_cnt[3 + 3 * p];
      // the table image stacks nh hi rows over nh lo rows per K chunk: one
      // MMA of width 2 nh gives [X_hi T_hi | X_hi T_lo], a second of width nh
      // adds X_lo T_hi to the correction
      const uint64_t xdesc0 = BF ? sw64_desc(smem_u32(xs)) : sw128_desc(smem_u32(xs));
      const uint64_t tdesc0 = BF ? sw64_desc(smem_u32(tab)) : sw128_desc(smem_u32(tab));
      for (int t = 0; t < nt && !*abort_flag; ++t, ++tcount) {
        const int4 ta = s_tiles[2 * t], tb = s_tiles[2 * t + 1];
        const int nh = min(s_seg[ta.z >> 8].npad, 64);
        const int chunk_tab = nh * ROWB;
        const uint32_t idesc2 = F16 ? idesc_f16(2 * nh) : BF ? idesc_bf16(2 * nh) : idesc_tf32(2 * nh);
        const uint32_t idesc1 = F16 ? idesc_f16(nh) : BF ? idesc_bf16(nh) : idesc_tf32(nh);
        const int kcp = ta.w & 0xff, kcq = ta.w >> 8;
        if (tb.x != cur) {
          if (!mbar_wait(tabf, ngrp & 1, abort_flag)) break;
          cur = tb.x;
          ++ngrp;
        }
        const int acc = tcount & 1;
        if (!mbar_wait(acce + acc, ((tcount >> 1) & 1) ^ 1, abort_flag)) break;
        tc_after();
        bool ok = true;
        // accumulators of this buffer (4 nhm columns apart): [P main][P corr][Q main][Q corr], nh columns each
        const uint32_t d = tmem + (uint32_t)(4 * acc * nhm + 2 * p * nh);
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
        if (t + 1 >= nt || s_tiles[2 * t + 3].x != cur) mma_commit(tabe);
      }
      s_cnt[2 + 3 * p] = c;
      s_cnt[3 + 3 * p] = tcount;
      s_cnt[4 + 3 * p] = (uint32_t)ngrp;
    }
  } else if (warp < kFirstEpiWarp) {
    // staging [32 l'][128 rows] -> K-major hi/lo rows; thread (r, h) converts
    // the 16 values l' = 16h .. 16h+15 of row r
    const int tid = threadIdx.x - 32 * kFirstSplitWarp;
    const int r = tid & 127, h = tid >> 7;
    // FP16x3: largest magnitude of the function of row r of tile tt (~0u past
    // the rows), loaded a tile ahead
    auto row_amax = [&](int tt) -> unsigned {
      const int4 ta = s_tiles[2 * tt];
      const LegISegSmall sg = s_seg[ta.z >> 8];
      const int grow = ta.y + r;
      return grow < sg.NB * 2 * sg.B ? a.amax[sg.fn0 + grow / (2 * sg.B)] : ~0u;
    };
    unsigned amx = 0u;
    if (F16 && nt > 0) amx = row_amax(0);
    uint32_t c = s_cnt[8];
    for (int t = 0; t < nt; ++t) {
      const int kcw = s_tiles[2 * t].w;
      const int kcp = kcw & 0xff, kcq = kcw >> 8;
      bool ok = true;
      // FP16x3: data scale of row r (its function's), zero past the rows
      float xf = 0.f;
      if constexpr (F16) {
        const float sb = s_seg[s_tiles[2 * t].z >> 8].sb;
        xf = amx == ~0u ? 0.f : pow2f(fp16_data_exp(amx, sb));
        if (t + 1 < nt) amx = row_amax(t + 1);
      }
      for (int ch = 0; ch < kcp + kcq; ++ch, ++c) {
        const int st = c % kStagingLegI;
        if (!mbar_wait(stgf + st, (c / kStagingLegI) & 1, abort_flag)) { ok = false; break; }
        float v[16];
        const float* sp = (const float*)(stg + st * kChunk) + 16 * h * 128;
#pragma unroll
        for (int k = 0; k < 16; ++k) v[k] = sp[k * 128 + r];
        fence_proxy_async();  // reads before the next bulk tensor copy into the slot
        mbar_arrive(stge + st);
        const int s = c % kStagesLegI;
        if (!mbar_wait(empty + s, ((c / kStagesLegI) & 1) ^ 1, abort_flag)) { ok = false; break; }
        if constexpr (BF) split_store_bf<4, F16>(xs + s * 2 * kChunk, xs + s * 2 * kChunk + kChunk, r, v, 4 * h, xf);
        else split_store<4>(xs + s * 2 * kChunk, xs + s * 2 * kChunk + kChunk, r, v, 4 * h, a.nprod == 3);
        fence_proxy_async();
        mbar_arrive(split + s);
      }
      if (!ok) break;
    }
    if (tid == 0) s_cnt[8] = c;
  } else {
    const int quarter = warp & 3;
    const int ehalf = (warp - kFirstEpiWarp) >> 2;  // alternate 16-column blocks
    const int r_in = quarter * 32 + lane;
    uint32_t tcount = s_cnt[9];
    for (int t = 0; t < nt; ++t, ++tcount) {
      const int4 ta = s_tiles[2 * t];
      const int acc = tcount & 1;
      // FP16x3: the magnitude of this row's function, loaded before the wait
      unsigned amx_row = 0u;
      if constexpr (F16) {
        const LegISegSmall sq = s_seg[ta.z >> 8];
        const int gr = ta.y + r_in;
        if (gr < sq.NB * 2 * sq.B) amx_row = a.amax[sq.fn0 + gr / (2 * sq.B)];
      }
      if (!mbar_wait(accf + acc, (tcount >> 1) & 1, abort_flag)) break;
      tc_after();
      const LegISegSmall sg = s_seg[ta.z >> 8];
      const int B = sg.B, NB = sg.NB, npad = sg.npad;
      const int nh = min(npad, 64);
      const int m_idx = ta.x;
      const int m = m_idx - (B - 1);
      const int am = m < 0 ? -m : m;
      const int kcp = ta.w & 0xff, kcq = ta.w >> 8;
      const float sgn = (m < 0 && (am & 1)) ? -1.f : 1.f;
      const int jh = ta.z & 1;
      const int ncols = jh ? npad - 64 : nh;
      // row (b, i, c): G element (m_idx, b, j, i, c) at stride 2B in j
      const int grow = ta.y + r_in;
      const bool valid = grow < NB * 2 * B;
      const int b = grow / (2 * B), ic = grow - b * (2 * B);
      // FP16x3: take out the table image's scale (tile record) and the row's data scale
      const float unscale = F16 && valid ? pow2f(-s_tiles[2 * t + 1].w) * pow2f(-fp16_data_exp(amx_row, sg.sb)) : 1.f;
      float* out = a.g + sg.w1_off + ((int64_t)m_idx * NB + b) * (2 * B) * (2 * B) + ic;
      const uint32_t lanes = (uint32_t)(quarter * 32) << 16;
      const uint32_t dP = tmem + (uint32_t)(4 * acc * nhm) + lanes;
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
        if constexpr (F16) {
#pragma unroll
          for (int k = 0; k < 16; ++k) {
            P[k] *= unscale;
            Q[k] *= unscale;
          }
        }
        if (valid) {
#pragma unroll
          for (int k = 0; k < 16; ++k) {
            const int j = jh * 64 + c0 + k;
            if (j < B) {
              out[(int64_t)j * (2 * B)] = sgn * (P[k] + Q[k]);
              out[(int64_t)(2 * B - 1 - j) * (2 * B)] = sgn * (P[k] - Q[k]);
            }
          }
        }
      }
      tc_before();
      mbar_arrive(acce + acc);
    }
    if (threadIdx.x == 32 * kFirstEpiWarp) s_cnt[9] = tcount;
  }
  // the slice is done in every role: its shared-memory copies may be replaced
  tc_before();
  __syncthreads();
  tc_after();
  }  // slices
  // Every role has left its loop.  After an abort the producer waits,
  // bounded, for the copies it issued and each MMA issuer for its MMAs,
  // before shared and tensor memory are released.
  __syncthreads();
  if (*abort_flag) {
    if (threadIdx.x == 0) atomicExch(a.err, 1);
    if (warp == 0 && lane == 0) {
      const uint32_t* cnt = (const uint32_t*)(bars + 61);
      drain_ring(stgf, kStagingLegI, cnt[0]);
      if (cnt[1] > 0) mbar_drain(tabf, (cnt[1] - 1) & 1);
    }
    if ((warp == 1 || warp == kMma2Warp) && lane == 0) drain_mma(bars + 62 + (warp == 1 ? 0 : 1));
    __syncthreads();
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
// One bandlimit segment of an inverse radial launch (a launch covers every
// segment of the plan).
struct RadISeg {
  int B, NB, fn0, si0;        // bandlimit, functions, first function, first S row entry in si_rows
  int64_t w2_off;             // the segment's S block
  int lb;                     // the segment's first entry in the per-degree table arrays (texp)
  int pad;
};

struct RadIArgs {
  const int4* tiles;          // (l, col0 | narrow, segment, table image offset of l), by segment and l
  const int* slice_first;     // first tile of each work-queue slice (nslices + 1 offsets)
  int nslices;
  int slice_cap;              // most tiles of one slice
  int* queue;                 // next slice to take; zero at launch
  int ntiles;
  const unsigned char* tabimg;
  const RadISeg* segs;
  int nseg;
  const int64_t* si_rows;     // S row offset per (m_idx, p), per segment from si0
  const float* coef;          // complex interleaved coefficients
  const int64_t* fn_coef;     // coefficient offset per function (plan order of segments)
  float* s;                   // output S, per segment layout [m_idx][p][l'][b][i][c]
  int* err;
  int si_max;                 // shared-memory entries for the S row offsets of one CTA's segments
  int nprod;                  // TF32 products per K step: 3 or 1 (hi*hi)
  const int* texp;            // FP16x3: table scale exponent per (segment, l) (RadISeg::lb + l)
  const unsigned* amax;       // FP16x3: per-function largest |coefficient| (segment order)
};

// Function of split thread tid's column (b, m, c) in tile tl (fn0 + b), or
// -1 past the segment's columns.  PAIR: the thread's column pair (b, m, re)
// and (b, m, im).
template <bool PAIR>
__device__ __forceinline__ int rad_fn_of(const RadISeg& sg, int4 tl, int tid) {
  const int l = tl.x;
  const bool nar = tl.y & 1;
  const int per_b = (2 * l + 1) * 2;
  const int col = (tl.y & ~1) + (PAIR ? 2 * (nar ? (tid & 31) : (tid & 63)) : (nar ? (tid & 63) : (tid & 127)));
  return col < sg.NB * per_b ? sg.fn0 + col / per_b : -1;
}

// Coefficients of one K chunk (32 degrees n) of one tile column, gathered by
// split thread tid: 16 (wide tile) or 8 (narrow tile) consecutive degrees,
// copied asynchronously to slot[k * 256 + tid] (zeros past the degree range
// or the segment's columns).  fco is the coefficient offset of the column's
// function (fn_coef, fetched a tile ahead by the caller).
__device__ __forceinline__ void rad_gather_async(const RadIArgs& a, const RadISeg& sg, int4 tl, int kc, int tid,
                                                 int64_t fco, float* slot) {
  const int B = sg.B, l = tl.x;
  const bool nar = tl.y & 1;
  const int col_in = nar ? (tid & 63) : (tid & 127);
  const int h = nar ? (tid >> 6) : (tid >> 7);
  const int nv = nar ? 8 : 16;
  const int per_b = (2 * l + 1) * 2;
  const int col = (tl.y & ~1) + col_in;
  const bool valid = col < sg.NB * per_b;
  const int b = valid ? col / per_b : 0;
  const int rem = col - b * per_b;
  const int m = (rem >> 1) - l, cc = rem & 1;
  const float* cf = a.coef + 2 * fco + cc;
  const int np0 = kc * 32 + h * nv;        // degree n = l + 1 + n'
  int n = l + 1 + np0;
  int64_t off = omega_of(n, l, m);          // omega(n + 1) - omega(n) = n^2
#pragma unroll
  for (int k = 0; k < 16; ++k) {
    if (k < nv) {
      const bool in = valid && np0 + k < B - l;
      cp_async4(slot + k * 256 + tid, in ? cf + 2 * off : a.coef, in);
      off += (int64_t)n * n;
      ++n;
    }
  }
}

// TF32 form: the coefficients of one K chunk of one column pair (b, m, re)
// and (b, m, im) — one complex value, one 8-byte copy per degree — gathered
// by split thread tid: pair tid & 63 (wide tile) or tid & 31 (narrow tile),
// 8 or 4 consecutive degrees from kc * 32 + (tid >> 6 or tid >> 5) * nv,
// copied asynchronously to slot[k * 256 + tid] (zeros past the degree range or
// the segment's columns).  Half the copies of the one-column form.
__device__ __forceinline__ void rad_gather_pairs_async(const RadIArgs& a, const RadISeg& sg, int4 tl, int kc,
                                                       int tid, int64_t fco, float2* slot) {
  const int B = sg.B, l = tl.x;
  const bool nar = tl.y & 1;
  const int pi = nar ? (tid & 31) : (tid & 63);
  const int h = nar ? (tid >> 5) : (tid >> 6);
  const int nv = nar ? 4 : 8;
  const int per_b = (2 * l + 1) * 2;
  const int col = (tl.y & ~1) + 2 * pi;
  const bool valid = col < sg.NB * per_b;
  const int b = valid ? col / per_b : 0;
  const int rem = col - b * per_b;
  const int m = (rem >> 1) - l;
  const float2* cf = (const float2*)a.coef + fco;
  const int np0 = kc * 32 + h * nv;        // degree n = l + 1 + n'
  int n = l + 1 + np0;
  int64_t off = omega_of(n, l, m);          // omega(n + 1) - omega(n) = n^2
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    if (k < nv) {
      const bool in = valid && np0 + k < B - l;
      cp_async8(slot + k * 256 + tid, in ? cf + off : (const float2*)a.coef, in);
      off += (int64_t)n * n;
      ++n;
    }
  }
}

template <int OP>
__global__ void __launch_bounds__(kThreadsInv, 1) tc_rad_inv_kernel(RadIArgs a) {
  constexpr bool BF = OP != TC_OP_TF32;  // 16-bit hi/lo pairs (kind::f16)
  constexpr bool F16 = OP == TC_OP_FP16;
  constexpr bool PAIR = !BF;           // coefficient gather by (re, im) pairs
  constexpr int ROWB = BF ? 64 : 128;  // bytes of one operand row of a 32-value K chunk
  constexpr int TCH = 128 * ROWB;      // one table chunk (hi or lo): 128 rows i
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char* base = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  // stage s: [table hi][table lo][data], 16 KB each part (BF16: the table
  // parts use their first 8 KB; data halves of 64 columns are 64 hi rows over
  // 64 lo rows, 16 KB (TF32) or 8 KB (BF16) each)
  unsigned char* st = base;
  float* gslots = (float*)(st + kStagesRadI * 4 * kChunk);  // gather staging slots
  uint64_t* bars = (uint64_t*)((unsigned char*)gslots + kGatherSlots * kGatherSlotBytes);
  uint64_t* tfull = bars;                   // [S] table chunk landed
  uint64_t* split = tfull + kStagesRadI;    // [S] data ready (split threads)
  uint64_t* empty = split + kStagesRadI;    // [S] MMAs done
  uint64_t* accf = empty + kStagesRadI;     // [2]
  uint64_t* acce = accf + 2;                // [2] (epilogue threads)
  uint32_t* tmem_slot = (uint32_t*)(acce + 2);
  volatile int* abort_flag = (volatile int*)(tmem_slot + 1);
  uint64_t* drain = bars + 62;              // [2] MMA issuers' own barriers, used after an abort
  uint32_t* issued = (uint32_t*)(bars + 61);  // producer: [copies issued into the ring, table copies]
  // Work queue (see tc_gemm_kernel): per slice the slice's tiles, the
  // segments they touch (seg_lo ..) and those segments' S row offsets are
  // copied to shared memory (capacities a.nseg segments, a.si_max offsets,
  // a.slice_cap tiles); role counters carry over through s_cnt.
  RadISeg* s_seg = (RadISeg*)(bars + 64);                  // [nseg]
  int* s_sib = (int*)(s_seg + a.nseg);                      // [nseg] first entry in s_si
  int64_t* s_si = (int64_t*)(((uintptr_t)(s_sib + a.nseg) + 7) & ~(uintptr_t)7);  // [si_max]
  int4* s_tiles = (int4*)(((uintptr_t)(s_si + a.si_max) + 15) & ~(uintptr_t)15);  // [slice_cap]
  // [0] producer table copies; [1 + 2k, 2 + 2k] MMA issuer k chunks, tiles;
  // [5] gather chunks; [6] epilogue tiles
  uint32_t* s_cnt = (uint32_t*)(bars + 48);
  volatile int* s_slice = (volatile int*)(bars + 53);

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
    mbar_init(drain, 1);
    mbar_init(drain + 1, 1);
    issued[0] = issued[1] = 0u;
    for (int k = 0; k < 8; ++k) s_cnt[k] = 0u;
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) tmem_alloc(tmem_slot, tmem_cols);
  tc_before();
  __syncthreads();
  tc_after();
  const uint32_t tmem = *tmem_slot;

  for (;;) {
  if (threadIdx.x == 0) *s_slice = atomicAdd(a.queue, 1);
  __syncthreads();
  const int sl = *s_slice;
  if (sl >= a.nslices || *abort_flag) break;
  const int g_begin = a.slice_first[sl];
  const int nt = a.slice_first[sl + 1] - g_begin;
  const int seg_lo = nt > 0 ? a.tiles[g_begin].z : 0;
  const int nseg_cta = nt > 0 ? a.tiles[g_begin + nt - 1].z - seg_lo + 1 : 0;
  if (threadIdx.x == 0) {
    int e = 0;
    for (int k = 0; k < nseg_cta; ++k) {
      s_seg[k] = a.segs[seg_lo + k];
      s_sib[k] = e;
      e += 2 * (2 * s_seg[k].B - 1);
    }
  }
  __syncthreads();
  for (int k = 0; k < nseg_cta; ++k) {
    const int n = 2 * (2 * s_seg[k].B - 1);
    for (int q = threadIdx.x; q < n; q += blockDim.x) s_si[s_sib[k] + q] = a.si_rows[s_seg[k].si0 + q];
  }
  for (int k = threadIdx.x; k < nt; k += blockDim.x) {
    int4 tl = a.tiles[g_begin + k];
    tl.z -= seg_lo;  // segment within this CTA's copy
    s_tiles[k] = tl;
  }
  tc_before();
  __syncthreads();
  tc_after();

  if (warp == 0) {
    if (lane == 0) {
      uint32_t c = s_cnt[0];
      for (int t = 0; t < nt && !*abort_flag; ++t) {
        const int4 tl = s_tiles[t];
        const int l = tl.x;
        const int kcn = (s_seg[tl.z].B - l + 31) / 32;
        const unsigned char* img = a.tabimg + (uint32_t)tl.w;
        bool ok = true;
        for (int kc = 0; kc < kcn; ++kc, ++c) {
          const int s = c % kStagesRadI;
          if (!mbar_wait(empty + s, ((c / kStagesRadI) & 1) ^ 1, abort_flag)) { ok = false; break; }
          // hi and lo chunk of the image, contiguous; the lo part lands at +kChunk
          mbar_arrive_tx(tfull + s, 2 * TCH);
          bulk_load(st + s * 4 * kChunk, img + (int64_t)kc * 2 * TCH, TCH, tfull + s);
          bulk_load(st + s * 4 * kChunk + kChunk, img + (int64_t)kc * 2 * TCH + TCH, TCH, tfull + s);
        }
        if (!ok) break;
      }
      issued[0] = s_cnt[0] = c;
    }
  } else if (warp == 1 || warp == kMma2Warp) {
    // MMA issuer `me`: narrow tiles, the K steps of parity me into
    // [main_me | corr_me]; wide tiles, the columns 64 me .. 64 me + 63
    if (lane == 0) {
      const int me = warp == 1 ? 0 : 1;
      uint32_t c = s_cnt[1 + 2 * me], tcount = s_cnt[2 + 2 * me];
      const uint64_t sdesc0 = BF ? sw64_desc(smem_u32(st)) : sw128_desc(smem_u32(st));
      // B operand of each half: 64 hi rows over 64 lo rows.  One MMA of width
      // 128 gives [T_hi X_hi | T_hi X_lo], a second of width 64 adds T_lo X_hi.
      const uint32_t idesc2 = F16 ? idesc_f16(128) : BF ? idesc_bf16(128) : idesc_tf32(128);
      const uint32_t idesc1 = F16 ? idesc_f16(64) : BF ? idesc_bf16(64) : idesc_tf32(64);
      for (int t = 0; t < nt && !*abort_flag; ++t, ++tcount) {
        const int4 tl = s_tiles[t];
        const int l = tl.x;
        const bool nar = tl.y & 1;
        const int kcn = (s_seg[tl.z].B - l + 31) / 32;
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
      s_cnt[1 + 2 * me] = c;
      s_cnt[2 + 2 * me] = tcount;
    }
  } else if (warp < kFirstEpiWarp) {
    // gather: thread (column, h) copies 16 (wide) or 8 (narrow) consecutive
    // degrees of its column per chunk into a staging slot (TF32: thread
    // (column pair, h) copies 8 or 4 degrees of its pair's complex values),
    // kGatherDepth chunks ahead of the chunk it splits and stores
    // (asynchronous copies: no registers held while they are in flight).  The
    // coefficient offset of the column's function is fetched a tile ahead of
    // the copies.
    const int tid = threadIdx.x - 32 * kFirstSplitWarp;
    auto fetch_fco = [&](int tt) -> int64_t {
      if (tt >= nt) return 0;
      const int f = rad_fn_of<PAIR>(s_seg[s_tiles[tt].z], s_tiles[tt], tid);
      return f >= 0 ? a.fn_coef[f] : 0;
    };
    // copy cursor: tile ti, chunk kci, chunks issued ci (starting from the
    // chunks consumed before this slice, so that slots and stages line up)
    const uint32_t c_begin = s_cnt[5];
    int ti = 0, kci = 0;
    uint32_t ci = c_begin;
    int64_t fco_i = 0, fco_n = 0;  // tiles ti and ti + 1
    if (nt > 0) {
      fco_i = fetch_fco(0);
      fco_n = fetch_fco(1);
    }
    auto issue_next = [&]() {
      if (ti < nt) {
        const int4 tl = s_tiles[ti];
        const RadISeg& sg = s_seg[tl.z];
        float* slot = gslots + (ci % kGatherSlots) * (kGatherSlotBytes / 4);
        if constexpr (PAIR) rad_gather_pairs_async(a, sg, tl, kci, tid, fco_i, (float2*)slot);
        else rad_gather_async(a, sg, tl, kci, tid, fco_i, slot);
        if (++kci == (sg.B - tl.x + 31) / 32) {
          kci = 0;
          ++ti;
          fco_i = fco_n;
          fco_n = fetch_fco(ti + 1);
        }
      }
      cp_async_commit();  // one group per chunk, empty past the end
      ++ci;
    };
#pragma unroll
    for (int d = 0; d < kGatherDepth; ++d) issue_next();
    int t = 0, kc = 0;
    // FP16x3: data scale of this thread's column (its function's), from the
    // magnitude loaded a tile ahead (~0u past the columns)
    auto col_amax = [&](int tt) -> unsigned {
      const int f = rad_fn_of<PAIR>(s_seg[s_tiles[tt].z], s_tiles[tt], tid);
      return f >= 0 ? a.amax[f] : ~0u;
    };
    unsigned amx = 0u;
    if (F16 && nt > 0) amx = col_amax(0);
    float xf = 0.f;
    uint32_t c = c_begin;
    for (; t < nt; ++c) {
      const int4 tl = s_tiles[t];
      const bool nar = tl.y & 1;
      if constexpr (F16) {
        if (kc == 0) {
          xf = amx == ~0u ? 0.f : pow2f(fp16_data_exp(amx, 1.f));
          if (t + 1 < nt) amx = col_amax(t + 1);
        }
      }
      int tn = t, kcn_next = kc + 1;
      if (kcn_next == (s_seg[tl.z].B - tl.x + 31) / 32) {
        tn = t + 1;
        kcn_next = 0;
      }
      // chunk c landed (the kGatherDepth - 1 later groups may still be in
      // flight); its values to registers, then the slot read one chunk ago
      // is refilled with chunk c + kGatherDepth
      cp_async_wait<kGatherDepth - 1>();
      float v[16];
      const float* gs = gslots + (c % kGatherSlots) * (kGatherSlotBytes / 4);  // the chunk's slot
      if constexpr (PAIR) {  // v[2k], v[2k + 1] = re, im of degree k: slot as float2 [k][tid]
        const float2* gv2 = (const float2*)gs + tid;
#pragma unroll
        for (int k = 0; k < 8; ++k) {
          const float2 w = gv2[k * 256];
          v[2 * k] = w.x;
          v[2 * k + 1] = w.y;
        }
      } else {  // slot as float [k][tid]
        const float* gv = gs + tid;
#pragma unroll
        for (int k = 0; k < 16; ++k) v[k] = gv[k * 256];
      }
      issue_next();
      const int s = c % kStagesRadI;
      if (!mbar_wait(empty + s, ((c / kStagesRadI) & 1) ^ 1, abort_flag)) break;
      // B operand: per half of 64 columns, 64 hi rows then 64 lo rows
      unsigned char* sb = st + s * 4 * kChunk + 2 * kChunk;
      if constexpr (BF) {
        if (nar) {
          split_store_bf<2, F16>(sb, sb + 64 * ROWB, tid & 63, v, 2 * (tid >> 6), xf);
        } else {
          unsigned char* hb = sb + ((tid >> 6) & 1) * (128 * ROWB);
          split_store_bf<4, F16>(hb, hb + 64 * ROWB, tid & 63, v, 4 * (tid >> 7), xf);
        }
      } else {
        // rows 2 pi (re) and 2 pi + 1 (im) of the pair's half; lanes whose
        // pair has bit 2 set store the im row first, so that each store
        // instruction's rows cover all eight 16-byte bank groups of the
        // 128-byte swizzle (conflict-free)
        const int pi = nar ? (tid & 31) : (tid & 63);
        unsigned char* hb = sb + (nar ? 0 : (pi >> 5) * (128 * ROWB));
        const int r0 = (2 * pi) & 63;
        const bool sw = (pi >> 2) & 1;
        float va[8], vb[8];
#pragma unroll
        for (int k = 0; k < 8; ++k) {
          va[k] = sw ? v[2 * k + 1] : v[2 * k];
          vb[k] = sw ? v[2 * k] : v[2 * k + 1];
        }
        if (nar) {
          split_store<1>(hb, hb + 64 * ROWB, r0 + (sw ? 1 : 0), va, tid >> 5, a.nprod == 3);
          split_store<1>(hb, hb + 64 * ROWB, r0 + (sw ? 0 : 1), vb, tid >> 5, a.nprod == 3);
        } else {
          split_store<2>(hb, hb + 64 * ROWB, r0 + (sw ? 1 : 0), va, 2 * (tid >> 6), a.nprod == 3);
          split_store<2>(hb, hb + 64 * ROWB, r0 + (sw ? 0 : 1), vb, 2 * (tid >> 6), a.nprod == 3);
        }
      }
      fence_proxy_async();
      mbar_arrive(split + s);
      t = tn;
      kc = kcn_next;
    }
    cp_async_wait_all();  // no copy may land after the CTA has left (or the slice is replaced)
    if (tid == 0) s_cnt[5] = c;
  } else {
    const int quarter = warp & 3;
    const int ehalf = (warp - kFirstEpiWarp) >> 2;  // alternate 16-column blocks
    const int i = quarter * 32 + lane;   // TMEM lane = radius index
    uint32_t tcount = s_cnt[6];
    for (int t = 0; t < nt; ++t, ++tcount) {
      const int4 tl = s_tiles[t];
      const int acc = tcount & 1;
      // FP16x3: magnitudes of the functions of this lane's column pairs (one
      // per block of 16 columns), loaded before the wait
      unsigned ramx[4] = {0u, 0u, 0u, 0u};
      if constexpr (F16) {
        const RadISeg sq = s_seg[tl.z];
        const int per_b = (2 * tl.x + 1) * 2;
#pragma unroll
        for (int it = 0; it < 4; ++it) {
          const int col = (tl.y & ~1) + 16 * ehalf + 32 * it + 2 * (lane & 7);
          if (col < sq.NB * per_b) ramx[it] = a.amax[sq.fn0 + col / per_b];
        }
      }
      if (!mbar_wait(accf + acc, (tcount >> 1) & 1, abort_flag)) break;
      tc_after();
      const RadISeg sg = s_seg[tl.z];
      const int B = sg.B, NB = sg.NB;
      const int64_t* si = s_si + s_sib[tl.z];
      float* sout = a.s + sg.w2_off;
      const int l = tl.x;
      const bool nar = tl.y & 1;
      const int col0 = tl.y & ~1;
      const int width = nar ? 64 : 128;
      const int per_b = (2 * l + 1) * 2;
      const uint32_t dq = tmem + (uint32_t)(acc * 256) + ((uint32_t)(quarter * 32) << 16);
      const float tscale = F16 ? pow2f(-a.texp[sg.lb + l]) : 1.f;  // FP16x3 table scale out
#pragma unroll
      for (int it = 0; it < 4; ++it) {
        const int c0 = 16 * ehalf + 32 * it;
        if (c0 >= width) break;
        // lane k < 8 finds the S offset of the column pair c0 + 2k, c0 + 2k + 1
        // ((b, m), re and im: column pairs never straddle (b, m), as tiles
        // start at even columns) and, for FP16x3, the pair's unscale factor;
        // the stores take both by shuffle
        int64_t o = -1;
        float un = tscale;
        {
          const int col = col0 + c0 + 2 * (lane & 7);
          if (col < NB * per_b) {
            const int b = col / per_b, rem = col - b * per_b;
            const int m = (rem >> 1) - l;
            const int am = m < 0 ? -m : m;
            const int p = (l - am) & 1;
            const int64_t srow = si[2 * (m + B - 1) + p] + ((l - am - p) >> 1);
            o = srow * ((int64_t)NB * 2 * B) + (int64_t)b * 2 * B;
            if (F16) un *= pow2f(-fp16_data_exp(ramx[it], 1.f));
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
        for (int k = 0; k < 8; ++k) {
          const int64_t ok = __shfl_sync(0xffffffffu, o, k);
          if constexpr (F16) {
            const float uk = __shfl_sync(0xffffffffu, un, k);
            if (i < B && ok >= 0) *(float2*)(sout + ok + 2 * i) = make_float2(v[2 * k] * uk, v[2 * k + 1] * uk);
          } else {
            if (i < B && ok >= 0) *(float2*)(sout + ok + 2 * i) = make_float2(v[2 * k], v[2 * k + 1]);
          }
        }
      }
      tc_before();
      mbar_arrive(acce + acc);
    }
    if (threadIdx.x == 32 * kFirstEpiWarp) s_cnt[6] = tcount;
  }
  // the slice is done in every role: its shared-memory copies may be replaced
  tc_before();
  __syncthreads();
  tc_after();
  }  // slices
  // Every role has left its loop (the gather threads have waited for their
  // asynchronous copies).  After an abort the producer waits, bounded, for
  // the table copies it issued and each MMA issuer for its MMAs, before
  // shared and tensor memory are released.
  __syncthreads();
  if (*abort_flag) {
    if (threadIdx.x == 0) atomicExch(a.err, 1);
    if (warp == 0 && lane == 0) drain_ring(tfull, kStagesRadI, ((const uint32_t*)(bars + 61))[0]);
    if ((warp == 1 || warp == kMma2Warp) && lane == 0) drain_mma(bars + 62 + (warp == 1 ? 0 : 1));
    __syncthreads();
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

// FP16 form of append_planes_bf16: the values times 2^e, as FP16 hi/lo pairs
// (hi = RN(v 2^e), lo = RN(v 2^e - hi)), same layout.
template <typename F>
void append_planes_f16(std::vector<unsigned char>& img, int rows, int K, int KC, int e, F value) {
  const size_t off = img.size();
  const size_t plane = (size_t)rows * 64;
  img.resize(off + 2 * (size_t)KC * plane, 0);
  for (int r = 0; r < rows; ++r)
    for (int k = 0; k < K; ++k) {
      const double v = std::ldexp(value(r, k), e);
      if (v == 0.0) continue;
      const __half h = __float2half_rn((float)v);
      const __half l = __float2half_rn((float)(v - (double)__half2float(h)));
      const uint16_t hb = __half_as_ushort(h), lb = __half_as_ushort(l);
      const int kc = k / 32, kin = k % 32;
      const size_t pos = (size_t)kc * 2 * plane + (size_t)r * 64 + (size_t)((((kin >> 3) ^ ((r >> 1) & 3)) << 4) + (kin & 7) * 2);
      memcpy(&img[off + pos], &hb, 2);
      memcpy(&img[off + plane + pos], &lb, 2);
    }
}

// Largest |value(r, k)| over r < rows, k < K.
template <typename F>
double table_max(int rows, int K, F value) {
  double mx = 0.0;
  for (int r = 0; r < rows; ++r)
    for (int k = 0; k < K; ++k) mx = std::max(mx, std::fabs(value(r, k)));
  return mx;
}

// Appends a table in the plan's operand format (FP16 scaled by 2^e).
template <typename F>
void append_table(std::vector<unsigned char>& img, int op, int rows, int K, int KC, int e, F value) {
  if (op == TC_OP_FP16) append_planes_f16(img, rows, K, KC, e, value);
  else if (op == TC_OP_BF16) append_planes_bf16(img, rows, K, KC, value);
  else append_planes(img, rows, K, KC, value);
}

int pad16i(int n) { return n <= 16 ? 16 : (n + 15) / 16 * 16; }

}  // namespace

// The two inverse stages over every segment of the plan, one launch each.
struct TcInvState {
  unsigned char* d_img = nullptr;
  // Legendre synthesis
  int4* leg_tiles = nullptr;      // two records per tile
  int* leg_first = nullptr;       // work-queue slice offsets
  int* leg_queue = nullptr;       // the queue's counter
  LegISeg* leg_segs = nullptr;
  int leg_ntiles = 0, leg_grid = 0, leg_nslices = 0, npad_max = 16, kcmax = 1;
  size_t leg_smem = 0;
  // radial
  int4* rad_tiles = nullptr;
  int* rad_first = nullptr;
  int* rad_queue = nullptr;
  RadISeg* rad_segs = nullptr;
  int rad_ntiles = 0, rad_grid = 0, rad_nslices = 0, rad_cap = 0, si_max = 0;
  size_t rad_smem = 0;
  std::vector<int64_t> l_off;     // image offset of the radial table of (segment, l)
  std::vector<int> l_base;        // first entry of each segment in l_off
  int* rad_texp = nullptr;        // FP16x3 scale exponent of the radial table of (segment, l)
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

// Work queue of a tile list: one wave of CTAs taking `per_cta` cost-balanced
// slices each on average, more slices while the largest one's share of shared
// memory does not fit.
static std::vector<int> slices_for(const std::vector<double>& cost, int nsm, int per_cta, size_t fixed,
                                   size_t per_tile, int* grid, int* nslices, int* max_tiles) {
  const int n = (int)cost.size();
  *grid = std::max(1, std::min(n, nsm));
  *nslices = std::max(1, std::min(n, *grid * per_cta));
  std::vector<int> first = balance_slices(cost, *nslices, max_tiles);
  while (fixed + (size_t)*max_tiles * per_tile > 227 * 1024 && *nslices < n) {
    *nslices = std::min(n, *nslices + *grid);
    first = balance_slices(cost, *nslices, max_tiles);
  }
  return first;
}

// Inverse radial tiles of every segment: 64 columns with two K chains where
// B - l >= P.radi_narrow, else 128 columns; the CTA slices and shared memory.
static cudaError_t radi_tiles(const Plan& P, TcInvState& st, int nsm, int64_t& bytes) {
  std::vector<int4> rtiles;
  std::vector<double> rc;
  for (size_t s = 0; s < P.segs.size(); ++s) {
    const int B = P.segs[s].B, NB = P.segs[s].NB;
    for (int l = 0; l < B; ++l) {
      const int nar = B - l >= P.radi_narrow ? 1 : 0;
      const int width = nar ? 64 : 128;
      const int kcn = (B - l + 31) / 32;
      const int img = (int)st.l_off[st.l_base[s] + l];
      for (int c0 = 0; c0 < NB * (2 * l + 1) * 2; c0 += width) {
        rtiles.push_back(make_int4(l, c0 | nar, (int)s, img));
        // gathered coefficients, table chunks (from L2, half weight), S out
        rc.push_back(kcn * (width * 128.0 + 16384.0) + 512.0 * width);
      }
    }
  }
  cudaError_t e = upload(&st.rad_tiles, rtiles, bytes);
  st.rad_ntiles = (int)rtiles.size();
  // shared memory: stages, barrier slots, the segments of the slice, their S
  // row offsets (si_max entries: the most any CTA's segments need), the tile
  // slice; more waves of CTAs while that does not fit
  const size_t fixed = 1024 + (size_t)kStagesRadI * 4 * kChunk + (size_t)kGatherSlots * kGatherSlotBytes + 64 * 8 +
                       (P.segs.size() + 1) * (sizeof(RadISeg) + 4) + 8 + 16;
  // work queue: P.queue_slices[2] cost-balanced slices per CTA of one wave, more
  // while a slice's copies do not fit
  const int n = (int)rc.size();
  st.rad_grid = std::max(1, std::min(n, nsm));
  st.rad_nslices = std::max(1, std::min(n, st.rad_grid * P.queue_slices[2]));
  std::vector<int> rf;
  for (;;) {
    int rmax = 0;
    rf = balance_slices(rc, st.rad_nslices, &rmax);
    int si_max = 0;
    for (int k = 0; k < st.rad_nslices; ++k) {
      if (rf[k + 1] <= rf[k]) continue;
      int need = 0;
      for (int sg = rtiles[rf[k]].z; sg <= rtiles[rf[k + 1] - 1].z; ++sg) need += 2 * (2 * P.segs[sg].B - 1);
      si_max = std::max(si_max, need);
    }
    st.si_max = si_max;
    st.rad_cap = std::max(1, rmax);
    st.rad_smem = fixed + (size_t)si_max * 8 + (size_t)(st.rad_cap + 1) * 16;
    if (st.rad_smem <= 227 * 1024 || st.rad_nslices >= n) break;
    st.rad_nslices = std::min(n, st.rad_nslices + st.rad_grid);
  }
  if (e == cudaSuccess) e = upload(&st.rad_first, rf, bytes);
  if (e == cudaSuccess && !st.rad_queue) e = cudaMalloc((void**)&st.rad_queue, sizeof(int));
  if (e == cudaSuccess && st.rad_smem > 227 * 1024) e = cudaErrorInvalidValue;
  return e;
}

cudaError_t tc_radi_retile(Plan& P) {
  TcInvState* st = (TcInvState*)P.tc_inv_state;
  if (!st) return cudaSuccess;
  int dev = 0, nsm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  if (st->rad_tiles) {
    cudaFree(st->rad_tiles);
    P.bytes -= (int64_t)st->rad_ntiles * sizeof(int4);
  }
  if (st->rad_first) {
    cudaFree(st->rad_first);
    P.bytes -= (int64_t)(st->rad_nslices + 1) * sizeof(int);
  }
  st->rad_tiles = nullptr;
  st->rad_first = nullptr;
  int64_t bytes = 0;
  const cudaError_t e = radi_tiles(P, *st, nsm, bytes);
  P.bytes += bytes;
  return e;
}

cudaError_t tc_inv_prepare(Plan& P) {
  int dev = 0, nsm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  TcInvState* st = new TcInvState();
  P.tc_inv_state = st;
  const bool bf = tc_bf16(P.prec);
  const int op = tc_operand(P.prec);
  std::vector<unsigned char> img;
  std::vector<int> texp;      // FP16x3 radial table exponents, as l_off
  std::vector<int4> lt;
  std::vector<double> lcost;  // estimated bytes moved per tile
  std::vector<LegISeg> lsegs;
  std::vector<RadISeg> rsegs;
  for (size_t s = 0; s < P.segs.size(); ++s) {
    const SegDesc& sg = P.segs[s];
    const HostTables& H = P.tables[s];
    const int B = sg.B, NB = sg.NB;
    LegISeg ls;
    memset(&ls, 0, sizeof(ls));
    ls.B = B, ls.NB = NB, ls.npad = pad16i(B), ls.fn0 = sg.fn0, ls.w1_off = sg.w1_off;
    st->npad_max = std::max(st->npad_max, ls.npad);
    // Legendre synthesis tables, per (|m|, j'-half of 64 rows):
    // [P hi][P lo][Q hi][Q lo], rows j', K = l'
    const int nh = ls.npad > 64 ? 64 : ls.npad;
    const int halves = (ls.npad + 63) / 64;
    std::vector<int64_t> aoff(2 * B, 0);
    std::vector<int> aexp(2 * B, 0);
    std::vector<int> akc(B, 0);
    for (int am = 0; am < B; ++am) {
      int kcs[2];
      for (int p = 0; p < 2; ++p) kcs[p] = (n_par(B, am, p) + 31) / 32;
      for (int jh = 0; jh < halves; ++jh) {
        img.resize((img.size() + 1023) / 1024 * 1024);
        aoff[2 * am + jh] = (int64_t)img.size();
        auto lam_p = [&](int p) {
          return [&, p](int jr, int q) -> double {
            const int j = 64 * jh + jr;
            if (j >= B) return 0.0;
            const int l = am + p + 2 * q;
            return H.lam[((size_t)am * B + l) * B + j];
          };
        };
        // one FP16 scale for the image (both parities)
        const double mx = std::max(table_max(nh, n_par(B, am, 0), lam_p(0)), table_max(nh, n_par(B, am, 1), lam_p(1)));
        const int e = op == TC_OP_FP16 ? fp16_scale_exp(mx) : 0;
        aexp[2 * am + jh] = e;
        for (int p = 0; p < 2; ++p) {
          if (kcs[p] == 0) continue;
          append_table(img, op, nh, n_par(B, am, p), kcs[p], e, lam_p(p));
        }
      }
      akc[am] = kcs[0] | (kcs[1] << 8);
      st->kcmax = std::max(st->kcmax, kcs[0] + kcs[1]);
    }
    for (int mi = 0; mi < 2 * B - 1; ++mi) {
      const int am = mi < B - 1 ? B - 1 - mi : mi - (B - 1);
      const int kcs = (akc[am] & 0xff) + (akc[am] >> 8);
      const int siP = (int)si_rows_before(B, mi, 0), siQ = (int)si_rows_before(B, mi, 1);
      for (int jh = 0; jh < halves; ++jh)
        for (int r0 = 0; r0 < NB * 2 * B; r0 += 128) {
          lt.push_back(make_int4(mi, r0, jh | ((int)s << 8), akc[am]));
          lt.push_back(make_int4((int)aoff[2 * am + jh], siP, siQ, aexp[2 * am + jh]));
          // S chunks in, both G halves out, the table on its first tile
          const int ncols = jh ? ls.npad - 64 : nh;
          lcost.push_back(kcs * 16384.0 + 1024.0 * ncols + (r0 == 0 ? 2.0 * kcs * nh * 128 : 0.0));
        }
    }
    // radial inverse tables, per l: KC_l x [hi chunk][lo chunk], rows i (128), K = n'
    st->l_base.push_back((int)st->l_off.size());
    double sbound = 0.0;  // bound on |S| / max |coefficient|: largest sum over n of |T_nl(i)|
    for (int l = 0; l < B; ++l) {
      img.resize((img.size() + 1023) / 1024 * 1024);
      st->l_off.push_back((int64_t)img.size());
      const int K = B - l, KC = (K + 31) / 32;
      double mx = 0.0;
      for (int i = 0; i < B; ++i) {
        double rs = 0.0;
        for (int np = 0; np < K; ++np) {
          const double t = std::fabs(H.T[((size_t)l * B + (l + np)) * B + i]);
          rs += t;
          mx = std::max(mx, t);
        }
        sbound = std::max(sbound, rs);
      }
      const int e = op == TC_OP_FP16 ? fp16_scale_exp(mx) : 0;
      texp.push_back(e);
      for (int kc = 0; kc < KC; ++kc) {
        auto tv = [&](int i, int k) -> double {
          const int np = kc * 32 + k;
          if (i >= B || np >= K) return 0.0;
          return H.T[((size_t)l * B + (l + np)) * B + i];
        };
        append_table(img, op, 128, 32, 1, e, tv);
      }
    }
    ls.sb = (float)sbound;
    // tensor map over S: [B^2 rows of l'][NB*2*B]
    float* w2 = (float*)P.d_w2 + sg.w2_off;
    if (!make_map_2d(&ls.smap, w2, (uint64_t)NB * 2 * B, (uint64_t)B * B, 128, 32, CU_TENSOR_MAP_SWIZZLE_NONE))
      return cudaErrorInvalidValue;
    lsegs.push_back(ls);
    rsegs.push_back(RadISeg{B, NB, sg.fn0, (int)sg.si_rows, sg.w2_off, st->l_base.back(), 0});
  }
  if (img.size() >= (size_t)1 << 31) return cudaErrorInvalidValue;  // image offsets are 32-bit
  int64_t bytes = 0;
  cudaError_t e = upload(&st->d_img, img, bytes);
  if (e == cudaSuccess) e = upload(&st->leg_tiles, lt, bytes);
  if (e == cudaSuccess) e = upload(&st->leg_segs, lsegs, bytes);
  if (e == cudaSuccess) e = upload(&st->rad_segs, rsegs, bytes);
  if (e == cudaSuccess) e = upload(&st->rad_texp, texp, bytes);
  st->leg_ntiles = (int)lcost.size();
  // tables, staging, operand ring, barrier slots, segments, tile slice (32 bytes a tile)
  const int nhm = st->npad_max > 64 ? 64 : st->npad_max;
  const size_t lfixed = 1024 + (size_t)st->kcmax * 2 * nhm * (bf ? 64 : 128) + (size_t)kStagingLegI * kChunk +
                        (size_t)kStagesLegI * 2 * kChunk + 64 * 8 + lsegs.size() * sizeof(LegISegSmall) + 16;
  int lmax = 0;
  const std::vector<int> lf =
      slices_for(lcost, nsm, P.queue_slices[3], lfixed, 32, &st->leg_grid, &st->leg_nslices, &lmax);
  if (e == cudaSuccess) e = upload(&st->leg_first, lf, bytes);
  if (e == cudaSuccess) e = cudaMalloc((void**)&st->leg_queue, sizeof(int));
  st->leg_smem = lfixed + (size_t)(lmax + 1) * 32;
  if (e == cudaSuccess && st->leg_smem > 227 * 1024) e = cudaErrorInvalidValue;
  if (e == cudaSuccess) e = radi_tiles(P, *st, nsm, bytes);
  P.bytes += bytes;
  return e;
}

void tc_inv_release(Plan& P) {
  TcInvState* st = (TcInvState*)P.tc_inv_state;
  if (!st) return;
  void* ptrs[] = {st->d_img,     st->leg_tiles, st->leg_first, st->leg_queue, st->leg_segs,
                  st->rad_tiles, st->rad_first, st->rad_queue, st->rad_segs, st->rad_texp};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  delete st;
  P.tc_inv_state = nullptr;
}

// prob 2: inverse radial (x = coefficients, y = S); prob 3: inverse Legendre (x = S, y = G)
cudaError_t run_tc_inverse(Plan& P, int prob, const void* x, void* y, cudaStream_t s) {
  TcInvState* st = (TcInvState*)P.tc_inv_state;
  if (!st) return cudaErrorNotSupported;
  StageTimer timer(P, prob == 2 ? ST_RAD_I : ST_LEG_I, s);
  cudaError_t e = cudaSuccess;
  if (prob == 2 && st->rad_ntiles > 0) {
    RadIArgs a;
    a.tiles = st->rad_tiles;
    a.slice_first = st->rad_first;
    a.nslices = st->rad_nslices;
    a.slice_cap = st->rad_cap;
    a.queue = st->rad_queue;
    a.ntiles = st->rad_ntiles;
    a.tabimg = st->d_img;
    a.segs = st->rad_segs;
    a.nseg = (int)P.segs.size();
    a.si_rows = P.d_si_rows;
    a.coef = (const float*)x;
    a.fn_coef = P.d_fn_coef;
    a.s = (float*)y;
    a.err = P.d_err;
    a.si_max = st->si_max;
    a.nprod = tc_products(P.prec);
    a.texp = st->rad_texp;
    a.amax = P.d_amax ? P.d_amax + AMAX_COEF * P.nfn : nullptr;
    const int op = tc_operand(P.prec);
    void (*fn)(RadIArgs) = op == TC_OP_FP16   ? tc_rad_inv_kernel<TC_OP_FP16>
                           : op == TC_OP_BF16 ? tc_rad_inv_kernel<TC_OP_BF16>
                                              : tc_rad_inv_kernel<TC_OP_TF32>;
    e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)st->rad_smem);
    if (e == cudaSuccess) e = cudaMemsetAsync(st->rad_queue, 0, sizeof(int), s);
    if (e != cudaSuccess) return e;
    fn<<<st->rad_grid, kThreadsInv, st->rad_smem, s>>>(a);
  } else if (prob == 3 && st->leg_ntiles > 0) {
    LegIArgs a;
    a.tiles = st->leg_tiles;
    a.slice_first = st->leg_first;
    a.nslices = st->leg_nslices;
    a.queue = st->leg_queue;
    a.ntiles = st->leg_ntiles;
    a.tabimg = st->d_img;
    a.segs = st->leg_segs;
    a.nseg = (int)P.segs.size();
    a.g = (float*)y;
    a.err = P.d_err;
    a.npad_max = st->npad_max;
    a.kcmax = st->kcmax;
    a.nprod = tc_products(P.prec);
    a.amax = P.d_amax ? P.d_amax + AMAX_COEF * P.nfn : nullptr;
    const int op = tc_operand(P.prec);
    void (*fn)(LegIArgs) = op == TC_OP_FP16   ? tc_leg_inv_kernel<TC_OP_FP16>
                           : op == TC_OP_BF16 ? tc_leg_inv_kernel<TC_OP_BF16>
                                              : tc_leg_inv_kernel<TC_OP_TF32>;
    e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)st->leg_smem);
    if (e == cudaSuccess) e = cudaMemsetAsync(st->leg_queue, 0, sizeof(int), s);
    if (e != cudaSuccess) return e;
    fn<<<st->leg_grid, kThreadsInv, st->leg_smem, s>>>(a);
  }
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  timer.finish();
  return cudaSuccess;
}

}  // namespace sgl
