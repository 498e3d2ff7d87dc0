// Tensor-core forward stages (tcgen05, TMEM, TMA) of the SGL transform:
// TF32x3 (and its hi*hi-only and BF16 hi/lo variants).  Each launch covers
// every bandlimit segment of the plan: tiles carry their segment.
//
// Forward Legendre stage (Eq. DLT, one GEMM per order m and theta-parity p)
// and forward radial stage (Eq. DRT_matrix, one GEMM per degree l):
//   D[row][n] = sum_k X[row][k] A[n][k]
// X: the stage's FP32 input rows (E/O spectra, or per-degree spectra), K-major;
// A: the FP64 table rounded to a hi + lo pair of TF32 values.  Three TF32
// products per K step, X_hi A_hi + X_hi A_lo + X_lo A_hi, accumulate in FP32 in
// tensor memory (the lo*lo term is below FP32 round-off).  The table image
// stacks the hi rows over the lo rows of each K chunk, so that one MMA of
// width 2N gives X_hi A_hi and X_hi A_lo side by side and a second of width N
// adds X_lo A_hi to the latter: two MMAs per K step.
//
// One persistent CTA per SM, warp-specialized (608 threads):
//   warp 0      TMA producer: 128-row x 32-float X chunks (SWIZZLE_128B) into a
//               staged ring; the group's pre-swizzled hi/lo table by bulk copy
//   warp 1      TMEM owner and MMA issuer of the even K steps (one thread)
//   warps 2-9   split: X -> hi (in place, TF32 round to nearest) and lo = X - hi
//   warps 10-17 epilogue: tcgen05.ld of the double-buffered accumulators, sign,
//               scatter to the next stage's layout
//   warp 18     MMA issuer of the odd K steps (one thread)
// Every wait on an mbarrier is bounded: after ~2 s the CTA sets the plan's
// error flag, stops, and frees its tensor memory.
#include <cuda.h>
#include <cuda_runtime.h>
#include <cudaTypedefs.h>
#include <stdint.h>
#include <string.h>

#include <algorithm>
#include <cmath>
#include <type_traits>
#include <vector>

#include "sgl_internal.h"
#include "tc_ptx.cuh"

namespace sgl {

// inverse tensor-core stages (tc_inv.cu)
cudaError_t tc_inv_prepare(Plan& P);
void tc_inv_release(Plan& P);
cudaError_t run_tc_inverse(Plan& P, int prob, const void* x, void* y, cudaStream_t s);

// cuTensorMapEncodeTiled from the driver (no link-time dependency on libcuda)
PFN_cuTensorMapEncodeTiled_v12000 get_encode() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  if (!fn) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = (PFN_cuTensorMapEncodeTiled_v12000)p;
  }
  return fn;
}

// 2-D FP32 tensor map: `rows` rows of `inner` floats (row pitch inner*4 bytes),
// boxes of box_inner x box_rows, zero fill outside the tensor.
bool make_map_2d(CUtensorMap* map, void* base, uint64_t inner, uint64_t rows, uint32_t box_inner, uint32_t box_rows,
                 CUtensorMapSwizzle sw) {
  PFN_cuTensorMapEncodeTiled_v12000 enc = get_encode();
  if (!enc) return false;
  cuuint64_t dims[2] = {(cuuint64_t)inner, (cuuint64_t)rows};
  cuuint64_t strides[1] = {(cuuint64_t)inner * 4};
  cuuint32_t box[2] = {box_inner, box_rows};
  cuuint32_t es[2] = {1, 1};
  CUresult r = enc(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, base, dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
                   sw, CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

namespace {

enum { TC_LEG_F = 0, TC_RAD_F = 1 };

// Ring depths.  Both tables are at most 64 rows (radial degrees with more
// than 64 terms are cut into groups), at most 64 KB of hi/lo TF32 (32 KB of
// 16-bit pairs), which leaves room for 5 raw TMA chunks next to the two
// operand chunks of TF32 (8 raw chunks for 16-bit pairs, whose operand
// chunks are half the size).
constexpr int kRawTf32 = 5;
constexpr int kRaw16 = 8;
constexpr int kOps = 2;
constexpr int kChunkBytes = 128 * 128;  // 128 rows x 32 floats
constexpr int kThreads = tcx::kRoleThreads;

using namespace tcx;
}  // namespace

// One bandlimit segment of a launch; a launch covers every segment of the
// plan (the tiles carry their segment).  Aligned as its tensor map.
struct TcSegInfo {
  CUtensorMap xmap;             // the segment's stage input, [rows][B] floats
  int B, NB, KC, fn0;           // bandlimit, functions, K chunks, first function in fn_coef
  int64_t w2_off;               // the segment's S_f block (forward Legendre output)
  int g0;                       // the segment's first group in the launch's group list
  float bw, bp;                 // FP16x3, radial stage: bound on |S_f| / largest |E/O|
                                // (weighted and plain Legendre tables)
};

// per-segment values the roles read per tile, staged in shared memory
struct SegSmall {
  int B, NB, KC, fn0;
  int64_t w2_off;
  int g0;
  float bw, bp;
  int pad;
};

struct TcArgs {
  const int2* tiles;            // (group | segment << 20, row0), groups in order
  const int* slice_first;       // first tile of each slice (nslices + 1 offsets)
  int nslices;                  // slices of the work queue
  int slice_cap;                // most tiles of one slice (shared-memory capacity)
  int group_cap;                // most groups one slice's tiles span (groups without
                                // tiles in between count: a slice may span more groups
                                // than it has tiles)
  int* queue;                   // next slice to take; zero at launch
  int ntiles;
  const unsigned char* tabimg;  // pre-swizzled hi/lo tables
  const int64_t* grp_off;       // byte offset of each group's image (weighted set, then plain set)
  const int* grp_npad;          // padded N of each group | l << 8 | n0 << 16 (radial)
  int ngroups;
  const TcSegInfo* segs;        // [nseg]
  int nseg;
  void* y;
  const int64_t* fn_coef;
  int* err;
  int KCmax;                    // largest K chunk count over the segments
  int weighted;
  int npmax;
  int nprod;                    // TF32 products per K step: 3 (hi*hi + hi*lo + lo*hi) or 1 (hi*hi)
  const int* grp_exp;           // FP16x3: table scale exponent of each group image (as grp_off)
  const unsigned* amax;         // FP16x3: per-function largest |E/O| (segment order)
  int rad_rows;                 // radial stage: rows n' of the largest table group (tile width)
};

// OP: the operand format (TcOperand).  TF32: kind::tf32, 128-byte rows, K = 8
// per MMA.  BF16 and FP16 hi/lo pairs: kind::f16, 64-byte rows, K = 16 per
// MMA; FP16 values are scaled by powers of two (tables per group image on the
// host, data per function here) and the epilogue takes the scales out.
template <int PROB, int RAW, int OP>
__global__ void __launch_bounds__(kThreads, 1) tc_gemm_kernel(TcArgs a) {
  constexpr bool BF = OP != TC_OP_TF32;  // a 16-bit operand path
  constexpr bool F16 = OP == TC_OP_FP16;
  constexpr int ROWB = BF ? 64 : 128;  // bytes of one operand row of a 32-value K chunk
  // Two rings: RAW chunks of TMA data (16 KB, the input rows as they are in
  // HBM), each released as soon as the split warps have read it (their
  // shared-memory reads fenced against the next bulk copy), and OPS
  // chunks of split hi/lo operands for the MMAs (hi then lo: 16 + 16 KB for
  // TF32, 8 + 8 KB for 16-bit pairs), so that more input is in flight than
  // the MMAs hold.
  constexpr int OPS = kOps;
  constexpr int OPB = BF ? kChunkBytes : 2 * kChunkBytes;
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char* base = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  const int tab_bytes = 2 * a.KCmax * a.npmax * ROWB;      // hi + lo for the largest group
  unsigned char* tab = base;                                 // [hi: KC][npad][128 B] [lo: same]
  unsigned char* xs = base + tab_bytes;                      // RAW x 16 KB of TMA chunks
  unsigned char* ops = xs + RAW * kChunkBytes;               // OPS x OPB of split operands
  uint64_t* bars = (uint64_t*)(ops + OPS * OPB);
  uint64_t* full = bars;                 // [RAW] TMA landed
  uint64_t* rfree = bars + RAW;          // [RAW] raw chunk read by the split warps
  uint64_t* split = bars + 2 * RAW;      // [OPS] hi/lo ready
  uint64_t* empty = split + OPS;         // [OPS] MMAs done with the operands
  uint64_t* accf = empty + OPS;          // [2] accumulator complete
  uint64_t* acce = accf + 2;             // [2] accumulator drained (128 arrivals)
  uint64_t* tabf = acce + 2;             // table landed
  uint64_t* tabe = tabf + 1;             // table no longer read
  uint32_t* tmem_slot = (uint32_t*)(tabe + 1);
  volatile int* abort_flag = (volatile int*)(tmem_slot + 1);
  uint64_t* drain = bars + 62;           // [2] MMA issuers' own barriers, used after an abort
  uint32_t* issued = (uint32_t*)(bars + 61);  // producer: [copies issued into the ring, table copies]
  // Work queue: the tile list is cut into a.nslices contiguous slices of
  // about equal estimated cost; each CTA takes the next slice from a global
  // counter (cleared before the launch) until none is left.  Per slice the
  // CTA copies the slice's tiles and the metadata of the groups they touch
  // to shared memory (fixed capacity a.slice_cap), so that no role waits on
  // a global load per tile; the segments are copied once.  The roles' barrier
  // phase counters carry over from slice to slice through s_cnt.
  SegSmall* s_seg = (SegSmall*)(bars + 64);                // [nseg]
  const int cap = a.slice_cap, gcap = a.group_cap;           // most tiles, groups of one slice
  int64_t* s_off = (int64_t*)(s_seg + a.nseg);              // [gcap] table image offsets
  int* s_npad = (int*)(s_off + gcap);                       // [gcap] padded N (| l, n0 for radial)
  int* s_exp = s_npad + gcap;                                // [gcap] FP16x3 table exponents
  int4* s_tiles = (int4*)(((uintptr_t)(s_exp + gcap) + 15) & ~(uintptr_t)15);  // [cap] (group, row0, segment)
  // [0, 1] producer chunks and tables; [2 + 3k, 3 + 3k, 4 + 3k] MMA issuer k
  // chunks, tiles, tables; [8] split chunks; [9] epilogue tiles
  uint32_t* s_cnt = (uint32_t*)(bars + 48);
  volatile int* s_slice = (volatile int*)(bars + 53);      // the slice being worked on

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  // Per tile two pairs of a main accumulator (hi*hi) and a correction
  // accumulator (hi*lo + lo*hi), [main0 | corr0 | main1 | corr1], npmax
  // columns each, double-buffered: pair k takes the K steps of parity k and is
  // fed by MMA issuer k.  The tensor cores round partial sums toward zero;
  // keeping the small corrections apart, and the K steps in two chains, cuts
  // the truncating additions into each main accumulator by six, and the four
  // are added with round-to-nearest in the epilogue.  Groups have at most 64
  // rows, so a buffer is at most 256 columns.
  const uint32_t bufcols = (uint32_t)(4 * a.npmax);
  uint32_t tmem_cols = 32;
  while (tmem_cols < 2 * bufcols) tmem_cols <<= 1;  // power of two >= 32

  if (threadIdx.x == 0) {
    for (int s = 0; s < RAW; ++s) {
      mbar_init(full + s, 1);
      mbar_init(rfree + s, kSplitThreads);
    }
    for (int o = 0; o < OPS; ++o) {
      mbar_init(split + o, kSplitThreads);
      mbar_init(empty + o, 2);  // both MMA issuers
    }
    for (int k = 0; k < 2; ++k) {
      mbar_init(accf + k, 2);
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
  for (int k = threadIdx.x; k < a.nseg; k += blockDim.x) {
    const TcSegInfo& g = a.segs[k];
    s_seg[k] = SegSmall{g.B, g.NB, g.KC, g.fn0, g.w2_off, g.g0, g.bw, g.bp, 0};
  }
  tc_before();
  __syncthreads();
  tc_after();
  const uint32_t tmem = *tmem_slot;
  const int64_t wsel = a.weighted ? 0 : a.ngroups;

  for (;;) {
  if (threadIdx.x == 0) *s_slice = atomicAdd(a.queue, 1);
  __syncthreads();
  const int sl = *s_slice;
  if (sl >= a.nslices || *abort_flag) break;
  // the slice's tile range (re-based to 0 in shared memory), group indices
  // re-based to g_lo
  const int g_begin = a.slice_first[sl];
  const int g_end = a.slice_first[sl + 1];
  const int t_begin = 0, t_end = g_end - g_begin;
  const int g_lo = t_end > 0 ? (a.tiles[g_begin].x & 0xFFFFF) : 0;
  const int ngr = t_end > 0 ? (a.tiles[g_end - 1].x & 0xFFFFF) - g_lo + 1 : 0;
  for (int k = threadIdx.x; k < t_end; k += blockDim.x) {
    const int2 tl = a.tiles[g_begin + k];
    s_tiles[k] = make_int4((tl.x & 0xFFFFF) - g_lo, tl.y, tl.x >> 20, 0);
  }
  for (int k = threadIdx.x; k < ngr; k += blockDim.x) {
    s_off[k] = a.grp_off[wsel + g_lo + k];
    s_npad[k] = a.grp_npad[g_lo + k];
    s_exp[k] = F16 ? a.grp_exp[wsel + g_lo + k] : 0;
  }
  tc_before();
  __syncthreads();
  tc_after();

  if (warp == 0) {
    // ---------------- producer ----------------
    if (lane == 0) {
      int cur = -1, ngrp = (int)s_cnt[1], cur_seg = -1;
      uint32_t c = s_cnt[0];
      for (int t = t_begin; t < t_end && !*abort_flag; ++t) {
        const int4 tl = s_tiles[t];
        const SegSmall sg = s_seg[tl.z];
        const CUtensorMap* xmap = &a.segs[tl.z].xmap;
        if (tl.z != cur_seg) {  // the tensor map lives in global memory
          asm volatile("fence.proxy.tensormap::generic.acquire.gpu [%0], 128;" ::"l"(xmap) : "memory");
          cur_seg = tl.z;
        }
        if (tl.x != cur) {
          if (ngrp > 0 && !mbar_wait(tabe, (ngrp - 1) & 1, abort_flag)) break;
          const uint32_t bytes = (uint32_t)(2 * sg.KC * (s_npad[tl.x] & 0xff) * ROWB);
          mbar_arrive_tx(tabf, bytes);
          bulk_load(tab, a.tabimg + s_off[tl.x], bytes, tabf);
          cur = tl.x;
          ++ngrp;
        }
        // tensor rows of this tile
        int64_t row;
        if (PROB == TC_LEG_F) {
          row = (int64_t)(tl.x + g_lo - sg.g0) * sg.NB * 2 * sg.B + tl.y;
        } else {
          const int l = (s_npad[tl.x] >> 8) & 0xff;
          row = (int64_t)sg.NB * 2 * l * l + tl.y;
        }
        for (int kc = 0; kc < sg.KC; ++kc, ++c) {
          const int s = c % RAW;
          if (!mbar_wait(rfree + s, ((c / RAW) & 1) ^ 1, abort_flag)) break;
          mbar_arrive_tx(full + s, kChunkBytes);
          tma_load_2d(xs + s * kChunkBytes, xmap, full + s, kc * 32, (int)row);
        }
      }
      issued[0] = s_cnt[0] = c;
      issued[1] = s_cnt[1] = (uint32_t)ngrp;
    }
  } else if (warp == 1 || warp == kMma2Warp) {
    // ---------------- MMA issuers: K steps of parity `me` ----------------
    if (lane == 0) {
      const int me = warp == 1 ? 0 : 1;
      int cur = -1, ngrp = (int)s_cnt[4 + 3 * me];
      uint32_t c = s_cnt[2 + 3 * me], tcount = s_cnt[3 + 3 * me];
      // operand chunk o: X_hi, then X_lo (16 KB each for TF32, 8 KB for 16-bit)
      const uint64_t xdesc0 = BF ? sw64_desc(smem_u32(ops)) : sw128_desc(smem_u32(ops));
      const uint64_t tdesc0 = BF ? sw64_desc(smem_u32(tab)) : sw128_desc(smem_u32(tab));
      for (int t = t_begin; t < t_end && !*abort_flag; ++t, ++tcount) {
        const int4 tl = s_tiles[t];
        const int KC = s_seg[tl.z].KC;
        if (tl.x != cur) {
          if (!mbar_wait(tabf, ngrp & 1, abort_flag)) break;
          cur = tl.x;
          ++ngrp;
        }
        const int npad = s_npad[tl.x] & 0xff;
        const uint32_t idesc2 = F16 ? idesc_f16(2 * npad) : BF ? idesc_bf16(2 * npad) : idesc_tf32(2 * npad);
        const uint32_t idesc1 = F16 ? idesc_f16(npad) : BF ? idesc_bf16(npad) : idesc_tf32(npad);
        const int acc = tcount & 1;
        if (!mbar_wait(acce + acc, ((tcount >> 1) & 1) ^ 1, abort_flag)) break;
        tc_after();
        // [main_me | corr_me]: one MMA of width 2 npad gives X_hi A_hi and
        // X_hi A_lo side by side, a second of width npad adds X_lo A_hi
        const uint32_t dm = tmem + (uint32_t)acc * bufcols + (uint32_t)(me * 2 * npad);
        const uint32_t dc = dm + (uint32_t)npad;
        bool ok = true;
        for (int kc = 0; kc < KC; ++kc, ++c) {
          const int o = c % OPS;
          if (!mbar_wait(split + o, (c / OPS) & 1, abort_flag)) { ok = false; break; }
          tc_after();
          const uint64_t xh = xdesc0 + (uint64_t)((o * OPB) >> 4) + 2 * me;
          const uint64_t xl = xh + (uint64_t)((BF ? kChunkBytes / 2 : kChunkBytes) >> 4);
          const uint64_t tb = tdesc0 + (uint64_t)((kc * 2 * npad * ROWB) >> 4) + 2 * me;
          const uint32_t first = kc > 0 ? 1u : 0u;
          if (BF) {  // kind::f16, K = 16 per MMA: one K step of the chunk per issuer
            mma_bf16(dm, xh, tb, idesc2, first);
            mma_bf16(dc, xl, tb, idesc1, 1u);
          } else if (a.nprod == 3) {
            mma_tf32(dm, xh, tb, idesc2, first);
            mma_tf32(dc, xl, tb, idesc1, 1u);
            mma_tf32(dm, xh + 4, tb + 4, idesc2, 1u);
            mma_tf32(dc, xl + 4, tb + 4, idesc1, 1u);
          } else {  // hi*hi only: the table's hi rows, main accumulator
            mma_tf32(dm, xh, tb, idesc1, first);
            mma_tf32(dm, xh + 4, tb + 4, idesc1, 1u);
          }
          mma_commit(empty + o);
        }
        if (!ok) break;
        mma_commit(accf + acc);
        const bool last_of_group = (t + 1 >= t_end) || (s_tiles[t + 1].x != cur);
        if (last_of_group) mma_commit(tabe);
      }
      s_cnt[2 + 3 * me] = c;
      s_cnt[3 + 3 * me] = tcount;
      s_cnt[4 + 3 * me] = (uint32_t)ngrp;
    }
  } else if (warp < kFirstEpiWarp) {
    // ---------------- split: X -> (hi, lo) ----------------
    const int tid = threadIdx.x - 32 * kFirstSplitWarp;  // 0 .. kSplitThreads-1
    constexpr int kPer = kChunkBytes / 16 / kSplitThreads;  // 16-byte pieces of a chunk per thread
    // FP16x3: largest magnitudes of the functions of this thread's rows of
    // tile tt (~0u past the stage's rows)
    unsigned amx[kPer];
    auto split_amax_load = [&](int tt, unsigned* out) {
      const int4 tl = s_tiles[tt];
      const SegSmall sg = s_seg[tl.z];
      const int per_f = PROB == TC_LEG_F ? 2 * sg.B : (2 * ((s_npad[tl.x] >> 8) & 0xff) + 1) * 2;
#pragma unroll
      for (int v = 0; v < kPer; ++v) {
        const int grow = tl.y + ((v * kSplitThreads + tid) >> 3);
        out[v] = grow < sg.NB * per_f ? a.amax[sg.fn0 + grow / per_f] : ~0u;
      }
    };
    (void)split_amax_load;
    uint32_t c = s_cnt[8];
    for (int t = t_begin; t < t_end; ++t) {
      bool ok = true;
      const int KC = s_seg[s_tiles[t].z].KC;
      // FP16x3: the data scale 2^e of each row this thread splits (row r =
      // piece index / 8), from the largest magnitude of the row's function
      // (times the growth bound through the Legendre table for the radial
      // stage); rows past the stage's rows are zeroed.  The magnitudes are
      // loaded a tile ahead.
      float xf[kPer];
      if constexpr (F16) {
        const SegSmall sg = s_seg[s_tiles[t].z];
        const float bound = PROB == TC_LEG_F ? 1.f : (a.weighted ? sg.bw : sg.bp);
        if (t == t_begin) split_amax_load(t, amx);
#pragma unroll
        for (int v = 0; v < kPer; ++v) xf[v] = amx[v] == ~0u ? 0.f : pow2f(fp16_data_exp(amx[v], bound));
        if (t + 1 < t_end) split_amax_load(t + 1, amx);
      }
      for (int kc = 0; kc < KC; ++kc, ++c) {
        const int s = c % RAW, o = c % OPS;
        if (!mbar_wait(full + s, (c / RAW) & 1, abort_flag)) { ok = false; break; }
        // the raw chunk to registers, and back to the producer
        float4 x[kPer];
        const float4* in = (const float4*)(xs + s * kChunkBytes);
#pragma unroll
        for (int v = 0; v < kPer; ++v) x[v] = in[v * kSplitThreads + tid];
        // the reads (generic proxy) ordered before the producer's next bulk
        // tensor copy into the slot (async proxy)
        fence_proxy_async();
        mbar_arrive(rfree + s);
        // the operand chunk, once the MMAs of chunk c - OPS are done with it
        if (!mbar_wait(empty + o, ((c / OPS) & 1) ^ 1, abort_flag)) { ok = false; break; }
        unsigned char* ob = ops + o * OPB;
        if constexpr (BF) {
          // raw chunk (128-byte rows, 32 floats) -> 16-bit hi/lo rows of 64 bytes
#pragma unroll
          for (int v = 0; v < kPer; ++v) {
            const int idx = v * kSplitThreads + tid;
            const int r = idx >> 3, q = (idx & 7) ^ (r & 7);  // values 4q .. 4q+3 of row r
            uint2 h2, l2;
            if constexpr (F16) {
              fp16_split2(x[v].x, x[v].y, xf[v], h2.x, l2.x);
              fp16_split2(x[v].z, x[v].w, xf[v], h2.y, l2.y);
            } else {
              const uint32_t s0 = bf16_split(x[v].x), s1 = bf16_split(x[v].y), s2 = bf16_split(x[v].z),
                             s3 = bf16_split(x[v].w);
              h2 = {(s0 & 0xFFFFu) | (s1 << 16), (s2 & 0xFFFFu) | (s3 << 16)};
              l2 = {(s0 >> 16) | (s1 & 0xFFFF0000u), (s2 >> 16) | (s3 & 0xFFFF0000u)};
            }
            const int off = sw64_off(r, q >> 1) + (q & 1) * 8;
            *(uint2*)(ob + off) = h2;
            *(uint2*)(ob + kChunkBytes / 2 + off) = l2;
          }
        } else {
          // same 128-byte swizzled positions as the TMA chunk: hi, then lo
          float4* hi = (float4*)ob;
          float4* lo = (float4*)(ob + kChunkBytes);
#pragma unroll
          for (int v = 0; v < kPer; ++v) {
            const int idx = v * kSplitThreads + tid;
            const float4 h = {tf32_rna(x[v].x), tf32_rna(x[v].y), tf32_rna(x[v].z), tf32_rna(x[v].w)};
            hi[idx] = h;
            if (a.nprod == 3) {
              // lo rounded to TF32 too, so that the tensor core uses it unchanged
              const float4 l = {tf32_rna(x[v].x - h.x), tf32_rna(x[v].y - h.y), tf32_rna(x[v].z - h.z),
                                tf32_rna(x[v].w - h.w)};
              lo[idx] = l;
            }
          }
        }
        fence_proxy_async();
        mbar_arrive(split + o);
      }
      if (!ok) break;
    }
    if (tid == 0) s_cnt[8] = c;
  } else {
    // ---------------- epilogue ----------------
    const int quarter = warp & 3;               // TMEM lanes 32*quarter .. +31
    const int ehalf = (warp - kFirstEpiWarp) >> 2;  // which 16-column blocks
    const int r_in = quarter * 32 + lane;       // tile row of this thread
    uint32_t tcount = s_cnt[9];
    float* Y = reinterpret_cast<float*>(a.y);
    for (int t = t_begin; t < t_end; ++t, ++tcount) {
      const int4 tl = s_tiles[t];
      const SegSmall sg = s_seg[tl.z];
      const int B = sg.B, NB = sg.NB;
      const int acc = tcount & 1;
      // FP16x3: the magnitude of this row's function, loaded before the wait
      unsigned amx_row = 0u;
      if constexpr (F16) {
        const int per_f = PROB == TC_LEG_F ? 2 * B : (2 * ((s_npad[tl.x] >> 8) & 0xff) + 1) * 2;
        const int gr = tl.y + r_in;
        if (gr < NB * per_f) amx_row = a.amax[sg.fn0 + gr / per_f];
      }
      if (!mbar_wait(accf + acc, (tcount >> 1) & 1, abort_flag)) break;
      tc_after();
      const int npad = s_npad[tl.x] & 0xff;
      const uint32_t taddr = tmem + (uint32_t)acc * bufcols + ((uint32_t)(quarter * 32) << 16);
      const uint32_t np = (uint32_t)npad;
      const int grow = tl.y + r_in;
      if (PROB == TC_LEG_F) {
        const int g = tl.x + g_lo - sg.g0;  // group within the segment
        const int m_idx = g >> 1, p = g & 1;
        const int m = m_idx - (B - 1);
        const int am = m < 0 ? -m : m;
        const int ncol = (am + p >= B) ? 0 : (B - 1 - am - p) / 2 + 1;
        const float sgn = (m < 0 && (am & 1)) ? -1.f : 1.f;
        const bool valid = grow < NB * 2 * B;
        const int b = grow / (2 * B), cc = (grow / B) & 1, i = grow % B;
        const int64_t rbase = sg.w2_off + (int64_t)cc * B + i;
        // FP16x3: take out the table's and the row's data scale
        const float unscale = F16 && valid ? pow2f(-s_exp[tl.x]) * pow2f(-fp16_data_exp(amx_row, 1.f)) : 1.f;
        for (int c0 = 16 * ehalf; c0 < npad; c0 += 32) {
          float v[16];
          const uint32_t tc = taddr + (uint32_t)c0;
          if (a.nprod == 3) {
            tmem_ld16_sum4(tc, tc + 2 * np, tc + np, tc + 3 * np, v);
          } else {
            float w[16];
            tmem_ld16x2(tc, tc + 2 * np, v, w);
#pragma unroll
            for (int k = 0; k < 16; ++k) v[k] += w[k];
          }
          if constexpr (F16) {
#pragma unroll
            for (int k = 0; k < 16; ++k) v[k] *= unscale;
          }
          if (valid) {
            // S_f[l][b][m+l][c][i] = 2B (NB l^2 + b(2l+1) + m + l) + c B + i, stepped in
            // l += 2 by first and second differences
            const int l = am + p + 2 * c0;
            const int64_t t = (int64_t)NB * l * l + (int64_t)(2 * b + 1) * l + b + m;
            float* yp = Y + rbase + 2 * (int64_t)B * t;
            int64_t d = 2 * (int64_t)B * ((int64_t)NB * (4 * l + 4) + 2 * (2 * b + 1));
            const int64_t dd = 16 * (int64_t)B * NB;
#pragma unroll
            for (int k = 0; k < 16; ++k) {
              if (c0 + k < ncol) *yp = sgn * v[k];
              yp += d;
              d += dd;
            }
          }
        }
      } else {
        const int l = (s_npad[tl.x] >> 8) & 0xff, n0 = s_npad[tl.x] >> 16;
        const int per_b = (2 * l + 1) * 2;
        const bool valid = grow < NB * per_b;
        const int b = grow / per_b;
        const int rem = grow - b * per_b;
        const int mm = rem >> 1, cc = rem & 1;
        const int ncol = min(B - l - n0, a.rad_rows);
        const int64_t cbase = valid ? a.fn_coef[sg.fn0 + b] : 0;
        const float unscale =
            F16 && valid ? pow2f(-s_exp[tl.x]) * pow2f(-fp16_data_exp(amx_row, a.weighted ? sg.bw : sg.bp)) : 1.f;
        for (int c0 = 16 * ehalf; c0 < npad; c0 += 32) {
          float v[16];
          const uint32_t tc = taddr + (uint32_t)c0;
          if (a.nprod == 3) {
            tmem_ld16_sum4(tc, tc + 2 * np, tc + np, tc + 3 * np, v);
          } else {
            float w[16];
            tmem_ld16x2(tc, tc + 2 * np, v, w);
#pragma unroll
            for (int k = 0; k < 16; ++k) v[k] += w[k];
          }
          if constexpr (F16) {
#pragma unroll
            for (int k = 0; k < 16; ++k) v[k] *= unscale;
          }
          if (valid) {
            // omega(n + 1, l, m) - omega(n, l, m) = n^2
            int n = l + 1 + n0 + c0;
            int64_t off = cbase + omega_of(n, l, mm - l);
#pragma unroll
            for (int k = 0; k < 16; ++k) {
              if (c0 + k < ncol) Y[2 * off + cc] = v[k];
              off += (int64_t)n * n;
              ++n;
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

  // Every role has left its loop.  After an abort (whichever role gave up,
  // and when) the producer waits, bounded, for the copies it issued and each
  // MMA issuer for its MMAs, before shared and tensor memory are released.
  __syncthreads();
  if (*abort_flag) {
    if (threadIdx.x == 0) atomicExch(a.err, 1);
    if (warp == 0 && lane == 0) {
      const uint32_t* cnt = (const uint32_t*)(bars + 61);
      drain_ring(full, RAW, cnt[0]);
      if (cnt[1] > 0) mbar_drain(tabf, (cnt[1] - 1) & 1);
    }
    if ((warp == 1 || warp == kMma2Warp) && lane == 0) drain_mma(bars + 62 + (warp == 1 ? 0 : 1));
    __syncthreads();
  }
  tc_after();
  if (warp == 1) tmem_dealloc(tmem, tmem_cols);
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
namespace {

// One stage (forward Legendre or forward radial) of every segment of the
// plan, run as one launch.
struct TcStage {
  int2* d_tiles = nullptr;
  int* d_first = nullptr;       // slice offsets of the work queue
  int* d_queue = nullptr;       // the queue's counter
  int nslices = 0, cap = 0, gcap = 0;
  int ntiles = 0;
  int64_t* d_off = nullptr;
  int* d_npad = nullptr;
  int* d_exp = nullptr;
  int ngroups = 0;
  TcSegInfo* d_segs = nullptr;
  int nseg = 0;
  int npmax = 16;
  int KCmax = 1;
  size_t smem = 0;
  int grid = 0;
};

struct TcState {
  TcStage leg, rad;
  unsigned char* d_img = nullptr;
};

// 2-D FP32 tensor [rows][B] with 128-row x 32-float boxes, 128-byte swizzle.
bool make_xmap(CUtensorMap* map, void* base, int B, int64_t rows) {
  return make_map_2d(map, base, (uint64_t)B, (uint64_t)rows, 32, 128, CU_TENSOR_MAP_SWIZZLE_128B);
}

uint32_t rna_tf32_bits(float x) {
  uint32_t u;
  memcpy(&u, &x, 4);
  u = (u + 0x1000u) & 0xFFFFE000u;
  return u;
}

// Append the swizzled hi/lo image of a table A[n][k] (n < N, k < K; zero
// padded to npad rows and KC*32 columns): per K chunk the npad hi rows, then
// the npad lo rows.
void append_image(std::vector<unsigned char>& img, int N, int K, int npad, int KC,
                  const std::vector<double>& A /* N x K */) {
  const size_t off = img.size();
  const size_t plane = (size_t)npad * 128;
  img.resize(off + 2 * (size_t)KC * plane, 0);
  for (int n = 0; n < N; ++n)
    for (int k = 0; k < K; ++k) {
      const double v = A[(size_t)n * K + k];
      const float f = (float)v;
      const uint32_t hb = rna_tf32_bits(f);
      float hi;
      memcpy(&hi, &hb, 4);
      const uint32_t lb = rna_tf32_bits((float)(v - (double)hi));
      float lo;
      memcpy(&lo, &lb, 4);
      const int kc = k / 32, kin = k % 32;
      const int chunk = kin / 4, w = kin % 4;
      const size_t pos = (size_t)kc * 2 * plane + (size_t)n * 128 + (size_t)((chunk ^ (n & 7)) * 16) + w * 4;
      memcpy(&img[off + pos], &hi, 4);
      memcpy(&img[off + plane + pos], &lo, 4);
    }
}

// BF16 round to nearest even of a float (finite values)
uint16_t bf16_bits(float x) {
  uint32_t u;
  memcpy(&u, &x, 4);
  return (uint16_t)((u + 0x7FFFu + ((u >> 16) & 1u)) >> 16);
}

// BF16 image of the same table: per K chunk the npad hi rows, then the npad
// lo rows, each row 32 values in 64 bytes with the 64-byte swizzle.
void append_image_bf16(std::vector<unsigned char>& img, int N, int K, int npad, int KC,
                       const std::vector<double>& A /* N x K */) {
  const size_t off = img.size();
  const size_t plane = (size_t)npad * 64;
  img.resize(off + 2 * (size_t)KC * plane, 0);
  for (int n = 0; n < N; ++n)
    for (int k = 0; k < K; ++k) {
      const double v = A[(size_t)n * K + k];
      const uint16_t hb = bf16_bits((float)v);
      uint32_t hu = (uint32_t)hb << 16;
      float hi;
      memcpy(&hi, &hu, 4);
      const uint16_t lb = bf16_bits((float)(v - (double)hi));
      const int kc = k / 32, kin = k % 32;
      const int q = kin / 8, w = kin % 8;  // 16-byte chunk of the 64-byte row, element in it
      const size_t pos = (size_t)kc * 2 * plane + (size_t)n * 64 + (size_t)((q ^ ((n >> 1) & 3)) * 16) + w * 2;
      memcpy(&img[off + pos], &hb, 2);
      memcpy(&img[off + plane + pos], &lb, 2);
    }
}

// FP16 image of the same table, scaled by 2^e (e = fp16_scale_exp of its
// largest magnitude, returned): hi = RN(v 2^e), lo = RN(v 2^e - hi), laid out
// as the BF16 image.
int append_image_f16(std::vector<unsigned char>& img, int N, int K, int npad, int KC,
                     const std::vector<double>& A /* N x K */) {
  double mx = 0.0;
  for (double v : A) mx = std::max(mx, std::fabs(v));
  const int e = fp16_scale_exp(mx);
  const size_t off = img.size();
  const size_t plane = (size_t)npad * 64;
  img.resize(off + 2 * (size_t)KC * plane, 0);
  for (int n = 0; n < N; ++n)
    for (int k = 0; k < K; ++k) {
      const double v = std::ldexp(A[(size_t)n * K + k], e);
      const __half h = __float2half_rn((float)v);
      const __half l = __float2half_rn((float)(v - (double)__half2float(h)));
      const uint16_t hb = __half_as_ushort(h), lb = __half_as_ushort(l);
      const int kc = k / 32, kin = k % 32;
      const int q = kin / 8, w = kin % 8;
      const size_t pos = (size_t)kc * 2 * plane + (size_t)n * 64 + (size_t)((q ^ ((n >> 1) & 3)) * 16) + w * 2;
      memcpy(&img[off + pos], &hb, 2);
      memcpy(&img[off + plane + pos], &lb, 2);
    }
  return e;
}

// Appends table A's image in the plan's operand format; returns the FP16
// scale exponent (0 for the other formats).
int append_table(std::vector<unsigned char>& img, int op, int N, int K, int npad, int KC,
                 const std::vector<double>& A) {
  if (op == TC_OP_FP16) return append_image_f16(img, N, K, npad, KC, A);
  if (op == TC_OP_BF16) append_image_bf16(img, N, K, npad, KC, A);
  else append_image(img, N, K, npad, KC, A);
  return 0;
}

int pad16(int n) { return n <= 16 ? 16 : (n + 15) / 16 * 16; }

}  // namespace

static cudaError_t tc_prepare_impl(Plan& P);

// Builds the tensor-core state of both directions and records its device
// bytes, so that tc_release can take them off the plan's count again.
cudaError_t tc_prepare(Plan& P) {
  const int64_t before = P.bytes;
  const cudaError_t e = tc_prepare_impl(P);
  P.tc_bytes = P.bytes - before;
  return e;
}

static cudaError_t tc_prepare_impl(Plan& P) {
  if (!get_encode()) return cudaErrorNotSupported;
  int dev = 0, nsm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  TcState* st = new TcState();
  const bool bf = tc_bf16(P.prec);
  const int op = tc_operand(P.prec);
  std::vector<unsigned char> img;
  // group lists of both stages over all segments: image offsets (weighted
  // set, plain set), padded widths, tiles and their estimated cost
  struct Pending {
    std::vector<int64_t> off[2];
    std::vector<int> exp[2];   // FP16 scale exponents, as off
    std::vector<int> npad;
    std::vector<int2> tiles;   // (group | segment << 20, row0)
    std::vector<double> cost;  // estimated bytes moved per tile (slice balancing)
    std::vector<TcSegInfo> segs;
  } pl, pr;
  for (size_t s = 0; s < P.segs.size(); ++s) {
    const SegDesc& sg = P.segs[s];
    const HostTables& H = P.tables[s];
    const int B = sg.B, NB = sg.NB;
    const int KC = (B + 31) / 32;
    float* w1 = (float*)P.d_w1 + sg.w1_off;
    float* w2 = (float*)P.d_w2 + sg.w2_off;
    // Legendre: groups g = m_idx*2 + p; images per (|m|, p), shared by +-m
    TcSegInfo li;
    memset(&li, 0, sizeof(li));
    li.B = B, li.NB = NB, li.KC = KC, li.fn0 = sg.fn0, li.w2_off = sg.w2_off, li.g0 = (int)pl.npad.size();
    if (!make_xmap(&li.xmap, w1, B, (int64_t)(2 * B - 1) * 2 * NB * 2 * B)) {
      delete st;
      return cudaErrorInvalidValue;
    }
    // bound on |S_f| / max |E/O| for the FP16x3 radial stage: the largest
    // absolute row sum of the (weighted, plain) Legendre table over the folded
    // grid, since S_f[l] = sum_j' A[l][j'] X[j']
    double rowsum[2] = {0.0, 0.0};
    for (int w = 0; w < 2; ++w) {
      std::vector<int64_t> am_off(2 * B, 0);
      std::vector<int> am_exp(2 * B, 0);
      for (int am = 0; am < B; ++am)
        for (int p = 0; p < 2; ++p) {
          const int N = n_par(B, am, p);
          if (N == 0) continue;
          const int np = pad16(N);
          std::vector<double> A((size_t)N * B);
          for (int q = 0; q < N; ++q) {
            const int l = am + p + 2 * q;
            double rs = 0.0;
            for (int j = 0; j < B; ++j) {
              const double v = H.lam[((size_t)am * B + l) * B + j];
              A[(size_t)q * B + j] = w == 0 ? H.beta[j] * v : v;
              rs += std::fabs(A[(size_t)q * B + j]);
            }
            rowsum[w] = std::max(rowsum[w], rs);
          }
          img.resize((img.size() + 1023) / 1024 * 1024);
          am_off[am * 2 + p] = (int64_t)img.size();
          am_exp[am * 2 + p] = append_table(img, op, N, B, np, KC, A);
        }
      for (int mi = 0; mi < 2 * B - 1; ++mi) {
        const int am = mi < B - 1 ? B - 1 - mi : mi - (B - 1);
        for (int p = 0; p < 2; ++p) {
          pl.off[w].push_back(am_off[am * 2 + p]);
          pl.exp[w].push_back(am_exp[am * 2 + p]);
        }
      }
    }
    li.bw = (float)rowsum[0];
    li.bp = (float)rowsum[1];
    for (int mi = 0; mi < 2 * B - 1; ++mi) {
      const int am = mi < B - 1 ? B - 1 - mi : mi - (B - 1);
      for (int p = 0; p < 2; ++p) {
        const int N = n_par(B, am, p);
        const int g = li.g0 + mi * 2 + p;
        pl.npad.push_back(pad16(N));
        st->leg.npmax = std::max(st->leg.npmax, pad16(N));
        if (N == 0) continue;
        for (int r0 = 0; r0 < NB * 2 * B; r0 += 128) {
          pl.tiles.push_back(make_int2(g | ((int)s << 20), r0));
          // X chunks in, S columns out, the group's table on its first tile
          pl.cost.push_back(KC * 16384.0 + 512.0 * N + (r0 == 0 ? 256.0 * KC * pad16(N) : 0.0));
        }
      }
    }
    pl.segs.push_back(li);
    // radial: groups (l, n0); degrees with more than P.rad_rows terms n' are
    // cut into groups of P.rad_rows rows n' (the tuned tile width) and the rest
    TcSegInfo ri = li;
    ri.g0 = (int)pr.npad.size();
    if (!make_xmap(&ri.xmap, w2, B, (int64_t)2 * NB * B * B)) {
      delete st;
      return cudaErrorInvalidValue;
    }
    std::vector<int2> rgrp;  // (l, n0)
    for (int l = 0; l < B; ++l)
      for (int n0 = 0; n0 < B - l; n0 += P.rad_rows) rgrp.push_back(make_int2(l, n0));
    for (int w = 0; w < 2; ++w)
      for (size_t g = 0; g < rgrp.size(); ++g) {
        const int l = rgrp[g].x, n0 = rgrp[g].y;
        const int N = std::min(B - l - n0, P.rad_rows);
        const int np = pad16(N);
        std::vector<double> A((size_t)N * B);
        for (int q = 0; q < N; ++q)
          for (int i = 0; i < B; ++i) {
            const double v = H.T[((size_t)l * B + (l + n0 + q)) * B + i];
            A[(size_t)q * B + i] = w == 0 ? H.what[i] * v : v;
          }
        img.resize((img.size() + 1023) / 1024 * 1024);
        pr.off[w].push_back((int64_t)img.size());
        if (w == 0) {
          pr.npad.push_back(np | (l << 8) | (n0 << 16));
          st->rad.npmax = std::max(st->rad.npmax, np);
        }
        pr.exp[w].push_back(append_table(img, op, N, B, np, KC, A));
      }
    for (size_t g = 0; g < rgrp.size(); ++g) {
      const int l = rgrp[g].x, n0 = rgrp[g].y;
      const int N = std::min(B - l - n0, P.rad_rows);
      for (int r0 = 0; r0 < NB * (2 * l + 1) * 2; r0 += 128) {
        pr.tiles.push_back(make_int2((ri.g0 + (int)g) | ((int)s << 20), r0));
        pr.cost.push_back(KC * 16384.0 + 512.0 * N + (r0 == 0 ? 256.0 * KC * pad16(N) : 0.0));
      }
    }
    pr.segs.push_back(ri);
    st->leg.KCmax = std::max(st->leg.KCmax, KC);
    st->rad.KCmax = std::max(st->rad.KCmax, KC);
  }
  cudaError_t e = cudaMalloc(&st->d_img, img.size());
  if (e != cudaSuccess) { delete st; return e; }
  P.bytes += img.size();
  e = cudaMemcpy(st->d_img, img.data(), img.size(), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) { delete st; return e; }
  auto upload = [&](auto** dst, const auto& v) -> cudaError_t {
    using T = typename std::decay<decltype(v[0])>::type;
    cudaError_t r = cudaMalloc((void**)dst, std::max<size_t>(v.size(), 1) * sizeof(T));
    if (r == cudaSuccess && !v.empty()) r = cudaMemcpy(*dst, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice);
    P.bytes += v.size() * sizeof(T);
    return r;
  };
  Pending* pend[2] = {&pl, &pr};
  TcStage* stg[2] = {&st->leg, &st->rad};
  for (int k = 0; k < 2 && e == cudaSuccess; ++k) {
    Pending& pd = *pend[k];
    TcStage& S = *stg[k];
    S.ntiles = (int)pd.tiles.size();
    S.ngroups = (int)pd.npad.size();
    S.nseg = (int)pd.segs.size();
    std::vector<int64_t> off = pd.off[0];
    off.insert(off.end(), pd.off[1].begin(), pd.off[1].end());
    std::vector<int> ex = pd.exp[0];
    ex.insert(ex.end(), pd.exp[1].begin(), pd.exp[1].end());
    e = upload(&S.d_tiles, pd.tiles);
    if (e == cudaSuccess) e = upload(&S.d_off, off);
    if (e == cudaSuccess) e = upload(&S.d_exp, ex);
    if (e == cudaSuccess) e = upload(&S.d_npad, pd.npad);
    if (e == cudaSuccess) e = upload(&S.d_segs, pd.segs);
    // tables, raw and operand rings, 64 barrier/flag slots, segments, then
    // per slice the group metadata and the tiles
    const size_t rings = bf ? (size_t)kRaw16 * kChunkBytes + (size_t)kOps * kChunkBytes
                            : (size_t)kRawTf32 * kChunkBytes + (size_t)kOps * 2 * kChunkBytes;
    const size_t fixed = 1024 + (size_t)2 * S.KCmax * S.npmax * (bf ? 64 : 128) + rings + 64 * 8 +
                         (size_t)S.nseg * sizeof(SegSmall) + 16 + 12 + 16;
    // work queue: P.queue_slices[k] cost-balanced slices per CTA of one wave
    // (more while one slice's shared-memory copies would not fit)
    // shared memory per slice: 16 bytes a tile, 16 bytes a group the tiles
    // span (counted exactly: groups without tiles may lie in between)
    S.grid = std::max(1, std::min(S.ntiles, nsm));
    S.nslices = std::max(1, std::min(S.ntiles, S.grid * P.queue_slices[k]));
    auto group_span = [&](const std::vector<int>& fst) {
      int g = 1;
      for (int k = 0; k < (int)fst.size() - 1; ++k)
        if (fst[k + 1] > fst[k])
          g = std::max(g, (pd.tiles[fst[k + 1] - 1].x & 0xFFFFF) - (pd.tiles[fst[k]].x & 0xFFFFF) + 1);
      return g;
    };
    int max_tiles = 0;
    std::vector<int> first = balance_slices(pd.cost, S.nslices, &max_tiles);
    int max_groups = group_span(first);
    while (fixed + (size_t)max_tiles * 16 + (size_t)max_groups * 16 > 227 * 1024 && S.nslices < S.ntiles) {
      S.nslices = std::min(S.ntiles, S.nslices + S.grid);
      first = balance_slices(pd.cost, S.nslices, &max_tiles);
      max_groups = group_span(first);
    }
    S.cap = std::max(1, max_tiles);
    S.gcap = max_groups;
    S.smem = fixed + (size_t)S.cap * 16 + (size_t)S.gcap * 16;
    if (e == cudaSuccess) e = upload(&S.d_first, first);
    if (e == cudaSuccess) e = cudaMalloc((void**)&S.d_queue, sizeof(int));
    if (e == cudaSuccess && S.smem > 227 * 1024) e = cudaErrorInvalidValue;
  }
  P.tc_state = st;
  if (e != cudaSuccess) return e;
  return tc_inv_prepare(P);
}

void tc_release(Plan& P) {
  P.bytes -= P.tc_bytes;
  P.tc_bytes = 0;
  tc_inv_release(P);
  TcState* st = (TcState*)P.tc_state;
  if (!st) return;
  for (TcStage* S : {&st->leg, &st->rad}) {
    void* ptrs[] = {S->d_tiles, S->d_first, S->d_queue, S->d_off, S->d_npad, S->d_exp, S->d_segs};
    for (void* q : ptrs)
      if (q) cudaFree(q);
  }
  if (st->d_img) cudaFree(st->d_img);
  delete st;
  P.tc_state = nullptr;
}

cudaError_t run_tc_stage(Plan& P, int prob, const void* x, void* y, int weighted, cudaStream_t s) {
  if (prob != 0 && prob != 1) return run_tc_inverse(P, prob, x, y, s);
  TcState* st = (TcState*)P.tc_state;
  if (!st) return cudaErrorNotSupported;
  static const int stage_of[2] = {ST_LEG_F, ST_RAD_F};
  StageTimer timer(P, stage_of[prob], s);
  TcStage& S = prob == 0 ? st->leg : st->rad;
  if (S.ntiles > 0) {
    TcArgs a;
    a.tiles = S.d_tiles;
    a.slice_first = S.d_first;
    a.nslices = S.nslices;
    a.slice_cap = S.cap;
    a.group_cap = S.gcap;
    a.queue = S.d_queue;
    a.ntiles = S.ntiles;
    a.tabimg = st->d_img;
    a.grp_off = S.d_off;
    a.grp_npad = S.d_npad;
    a.ngroups = S.ngroups;
    a.segs = S.d_segs;
    a.nseg = S.nseg;
    a.y = y;
    a.fn_coef = P.d_fn_coef;
    a.err = P.d_err;
    a.KCmax = S.KCmax;
    a.weighted = weighted;
    a.npmax = S.npmax;
    a.nprod = tc_products(P.prec);
    a.grp_exp = S.d_exp;
    a.rad_rows = P.rad_rows;
    a.amax = P.d_amax ? P.d_amax + AMAX_EO * P.nfn : nullptr;
    (void)x;
    void (*fn)(TcArgs);
    switch (tc_operand(P.prec)) {
      case TC_OP_FP16:
        fn = prob == 0 ? tc_gemm_kernel<TC_LEG_F, kRaw16, TC_OP_FP16> : tc_gemm_kernel<TC_RAD_F, kRaw16, TC_OP_FP16>;
        break;
      case TC_OP_BF16:
        fn = prob == 0 ? tc_gemm_kernel<TC_LEG_F, kRaw16, TC_OP_BF16> : tc_gemm_kernel<TC_RAD_F, kRaw16, TC_OP_BF16>;
        break;
      default:
        fn = prob == 0 ? tc_gemm_kernel<TC_LEG_F, kRawTf32, TC_OP_TF32>
                       : tc_gemm_kernel<TC_RAD_F, kRawTf32, TC_OP_TF32>;
    }
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)S.smem);
    if (e == cudaSuccess) e = cudaMemsetAsync(S.d_queue, 0, sizeof(int), s);
    if (e != cudaSuccess) return e;
    fn<<<S.grid, kThreads, S.smem, s>>>(a);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  timer.finish();
  return cudaSuccess;
}

}  // namespace sgl
