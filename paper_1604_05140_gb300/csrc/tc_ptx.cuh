// PTX wrappers for the tcgen05 / TMA / mbarrier kernels (sm_103a).
#pragma once

#include <cuda.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace sgl {
namespace tcx {

constexpr uint64_t kWaitNs = 2000000000ull;  // bound of every mbarrier wait

// Warp roles of the tensor-core kernels: warp 0 producer, warp 1 TMEM owner
// and first MMA issuer, then kSplitWarps operand-split warps, kEpiWarps
// epilogue warps and the second MMA issuer.  Epilogue warp w reads TMEM lanes
// 32*(w%4) .. +31; the two warps of one lane quarter take alternate 16-column
// blocks.  Each issuer owns its own accumulators (one thread issues an MMA
// only every ~60 cycles, less than the tensor core takes for the small tiles
// here, so two threads on two schedulers keep it busier).
constexpr int kSplitWarps = 8;
constexpr int kEpiWarps = 8;
constexpr int kFirstSplitWarp = 2;
constexpr int kFirstEpiWarp = kFirstSplitWarp + kSplitWarps;
constexpr int kMma2Warp = kFirstEpiWarp + kEpiWarps;
constexpr int kSplitThreads = 32 * kSplitWarps;
constexpr int kEpiThreads = 32 * kEpiWarps;
constexpr int kRoleThreads = 32 * (kMma2Warp + 1);

static __device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// 4-byte asynchronous copy global -> shared, zero-filled (nothing read) when
// !pred; copies are tracked per thread in commit groups
static __device__ __forceinline__ void cp_async4(void* dst, const void* src, bool pred) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;" ::"r"(smem_u32(dst)), "l"(src), "r"(pred ? 4 : 0)
               : "memory");
}
static __device__ __forceinline__ void cp_async8(void* dst, const void* src, bool pred) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;" ::"r"(smem_u32(dst)), "l"(src), "r"(pred ? 8 : 0)
               : "memory");
}
static __device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
// wait until at most N of this thread's most recent groups are pending
template <int N>
static __device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}
static __device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

static __device__ __forceinline__ uint64_t gtimer() {
  uint64_t t;
  asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
  return t;
}

static __device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

static __device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

static __device__ __forceinline__ void mbar_arrive_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}

static __device__ __forceinline__ bool mbar_try(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// As mbar_try, but the thread may sleep in the instruction until the phase
// completes or about `ns` nanoseconds have passed, so that waiting warps take
// no issue slots from the working ones.
static __device__ __forceinline__ bool mbar_try_sleep(uint64_t* bar, uint32_t parity, uint32_t ns) {
  uint32_t ok;
  asm volatile(
      "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\nselp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity), "r"(ns)
      : "memory");
  return ok != 0;
}

// Bounded wait for the phase of the given parity.  On timeout (limit_ns,
// 2 s by default), or when another role already aborted, sets the abort flag
// and returns false.
static __device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, volatile int* abort_flag,
                                                 uint64_t limit_ns = kWaitNs) {
  if (mbar_try(bar, parity)) return true;
  const uint64_t t0 = gtimer();
  while (true) {
    if (mbar_try_sleep(bar, parity, 100000u)) return true;
    if (*abort_flag) return false;
    if (gtimer() - t0 > limit_ns) {
      *abort_flag = 1;
      return false;
    }
  }
}

// Bound of each wait while a CTA winds down after an abort.
constexpr uint64_t kDrainNs = 200000000ull;

// Wait, bounded by limit_ns, for the phase of the given parity without
// looking at the abort flag (used after an abort, to let operations that were
// already issued finish).  Returns whether the phase completed.
static __device__ __noinline__ bool mbar_drain(uint64_t* bar, uint32_t parity, uint64_t limit_ns = kDrainNs) {
  const uint64_t t0 = gtimer();
  while (!mbar_try_sleep(bar, parity, 100000u))
    if (gtimer() - t0 > limit_ns) return false;
  return true;
}

// After an abort: wait for the last asynchronous copy that landed, or will
// land, on each barrier of a ring of `stages` barriers, when `issued` copies
// were issued in all (copy k completes phase k / stages of bars[k % stages]).
// Returns whether every one of them finished within the bound.
static __device__ __noinline__ bool drain_ring(uint64_t* bars, int stages, uint32_t issued) {
  bool ok = true;
  for (int s = 0; s < stages && (uint32_t)s < issued; ++s) {
    const uint32_t last = (uint32_t)s + (uint32_t)stages * ((issued - 1 - (uint32_t)s) / (uint32_t)stages);
    ok = mbar_drain(bars + s, (last / (uint32_t)stages) & 1) && ok;
  }
  return ok;
}

static __device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, uint64_t* bar, int x, int y) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4}], [%2];" ::"r"(
          smem_u32(dst)),
      "l"(map), "r"(smem_u32(bar)), "r"(x), "r"(y)
      : "memory");
}

static __device__ __forceinline__ void bulk_load(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   smem_u32(dst)),
               "l"(src), "r"(bytes), "r"(smem_u32(bar))
               : "memory");
}

static __device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
static __device__ __forceinline__ void tc_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
static __device__ __forceinline__ void tc_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

static __device__ __forceinline__ void tmem_alloc(uint32_t* slot, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(slot)),
               "r"(ncols)
               : "memory");
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}

static __device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}

static __device__ __forceinline__ void mma_tf32(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
      "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(d),
      "l"(a), "l"(b), "r"(idesc), "r"(acc)
      : "memory");
}

static __device__ __forceinline__ void mma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
               : "memory");
}

// After an abort: an MMA-issuing thread commits every MMA it issued to its
// own barrier (count 1, not used before) and waits, bounded, until they have
// finished reading shared memory and writing tensor memory.
static __device__ __noinline__ bool drain_mma(uint64_t* bar) {
  mma_commit(bar);
  return mbar_drain(bar, 0);
}

static __device__ __forceinline__ void tmem_ld16(uint32_t taddr, float* v) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int k = 0; k < 16; ++k) v[k] = __uint_as_float(r[k]);
}

// Two 16-column loads issued together, one wait.
static __device__ __forceinline__ void tmem_ld16x2(uint32_t ta, uint32_t tb, float* va, float* vb) {
  uint32_t r[32];
  asm volatile(
      "{\n"
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%32];\n"
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, "
      "[%33];\n"
      "tcgen05.wait::ld.sync.aligned;\n"
      "}\n"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
        "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
        "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(ta), "r"(tb)
      : "memory");
#pragma unroll
  for (int k = 0; k < 16; ++k) {
    va[k] = __uint_as_float(r[k]);
    vb[k] = __uint_as_float(r[16 + k]);
  }
}

// main + correction accumulators, 16 columns each, summed with round-to-nearest
static __device__ __forceinline__ void tmem_ld16_sum(uint32_t tmain, uint32_t tcorr, float* v) {
  float c[16];
  tmem_ld16x2(tmain, tcorr, v, c);
#pragma unroll
  for (int k = 0; k < 16; ++k) v[k] += c[k];
}

// two main and two correction accumulators: (main0 + main1) + (corr0 + corr1)
static __device__ __forceinline__ void tmem_ld16_sum4(uint32_t tm0, uint32_t tm1, uint32_t tc0, uint32_t tc1,
                                                      float* v) {
  float w[16], c[16], d[16];
  tmem_ld16x2(tm0, tm1, v, w);
  tmem_ld16x2(tc0, tc1, c, d);
#pragma unroll
  for (int k = 0; k < 16; ++k) v[k] = (v[k] + w[k]) + (c[k] + d[k]);
}

// Round to TF32 (10 fraction bits), to nearest with ties away from zero: add
// half a unit of the 11th significant bit to the magnitude bits and clear the
// 13 bits below it (a carry into the exponent gives the correctly rounded
// power of two).  Finite inputs only.
static __device__ __forceinline__ float tf32_rna(float x) {
  return __uint_as_float((__float_as_uint(x) + 0x1000u) & 0xFFFFE000u);
}

// K-major, 128-byte swizzled operand: 8-row groups 1024 B apart.  The start
// address is the low field (address / 16), so a descriptor moves by `bytes`
// (a multiple of 16, staying inside shared memory) with desc + bytes / 16.
static __device__ __forceinline__ uint64_t sw128_desc(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr & 0x3FFFF) >> 4);       // start address
  d |= (uint64_t)1 << 16;                        // leading byte offset (unused for this layout)
  d |= (uint64_t)(1024 >> 4) << 32;              // stride byte offset
  d |= (uint64_t)1 << 46;                        // descriptor version
  d |= (uint64_t)2 << 61;                        // 128-byte swizzle
  return d;
}

// K-major, 64-byte swizzled operand (rows of 64 bytes, the BF16 operands):
// 8-row groups 512 B apart.
static __device__ __forceinline__ uint64_t sw64_desc(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr & 0x3FFFF) >> 4);       // start address
  d |= (uint64_t)1 << 16;                        // leading byte offset (unused for this layout)
  d |= (uint64_t)(512 >> 4) << 32;               // stride byte offset
  d |= (uint64_t)1 << 46;                        // descriptor version
  d |= (uint64_t)4 << 61;                        // 64-byte swizzle
  return d;
}

// kind::f16 instruction descriptor: D f32, A and B bf16, both K-major, M = 128.
static __device__ __forceinline__ uint32_t idesc_bf16(int n) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(128 >> 4) << 24);
}

static __device__ __forceinline__ void mma_bf16(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d),
      "l"(a), "l"(b), "r"(idesc), "r"(acc)
      : "memory");
}

// Split x into BF16 hi = RN(x) and lo = RN(x - hi) (round to nearest even);
// returns hi in the low and lo in the high half-word.
static __device__ __forceinline__ uint32_t bf16_split(float x) {
  uint32_t u = __float_as_uint(x);
  const uint32_t hb = (u + 0x7FFFu + ((u >> 16) & 1u)) >> 16;
  const float r = x - __uint_as_float(hb << 16);
  u = __float_as_uint(r);
  const uint32_t lb = (u + 0x7FFFu + ((u >> 16) & 1u)) >> 16;
  return hb | (lb << 16);
}

// kind::f16 instruction descriptor with FP16 A and B (format 0): D f32,
// both K-major, M = 128.
static __device__ __forceinline__ uint32_t idesc_f16(int n) {
  return (1u << 4) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(128 >> 4) << 24);
}

// FP16 hi/lo split of x * f (f a power of two, so the product is exact).
// With the scales used here |x f| < 2^14, so hi never overflows, and lo keeps
// 11 significant bits down to |x f| ~ 2^-3.
// Two values at once, packed as the operand rows want them: hi = {hi(x0) in
// the low half, hi(x1) in the high half}, lo likewise.  hi is x f rounded to
// 11 significant bits by the integer TF32 rounding (an FP16 value whenever
// |x f| is in FP16's normal range, which the scales guarantee for all but
// the negligible values), lo = x f - hi in FP32; one packed conversion
// (cvt f16x2) each, instead of three scalar conversions per value.
static __device__ __forceinline__ void fp16_split2(float x0, float x1, float f, uint32_t& hi, uint32_t& lo) {
  const float a = x0 * f, b = x1 * f;
  const float ha = tf32_rna(a), hb = tf32_rna(b);
  const __half2 h = __floats2half2_rn(ha, hb);
  const __half2 l = __floats2half2_rn(a - ha, b - hb);
  hi = *reinterpret_cast<const uint32_t*>(&h);
  lo = *reinterpret_cast<const uint32_t*>(&l);
}

// 2^e as a float, -126 <= e <= 127.
static __device__ __forceinline__ float pow2f(int e) { return __int_as_float((e + 127) << 23); }

// Exponent e of the FP16x3 data scale: the largest magnitude x (a float's
// bits; x >= 0), times a growth bound, lands in [2^13, 2^14) after scaling by
// 2^e; 0 for x = 0; clamped to +-100 (as fp16_scale_exp on the host).
static __device__ __forceinline__ int fp16_data_exp(unsigned amax_bits, float bound) {
  const float x = __uint_as_float(amax_bits) * bound;
  if (!(x > 0.f)) return 0;
  // x = m 2^E with m in [0.5, 1): E = biased exponent - 126 for normal x, so
  // e = 14 - E = 140 - biased exponent; subnormal x (biased 0) clamps to
  // +100, infinite or NaN x (biased 255) to -100
  const int eb = (int)((__float_as_uint(x) >> 23) & 0xffu);
  const int e = 140 - eb;
  return eb == 0 ? 100 : (e > 100 ? 100 : (e < -100 ? -100 : e));
}

// 128-byte swizzled (TF32 rows) and 64-byte swizzled (BF16 rows) byte
// offsets of 16-byte chunk q of row r in a K-major tile.
static __device__ __forceinline__ int sw128_off(int r, int q) { return r * 128 + ((q ^ (r & 7)) << 4); }
static __device__ __forceinline__ int sw64_off(int r, int q) { return r * 64 + ((q ^ ((r >> 1) & 3)) << 4); }

// kind::tf32 instruction descriptor: D f32, A and B tf32, both K-major, M = 128.
static __device__ __forceinline__ uint32_t idesc_tf32(int n) {
  return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(128 >> 4) << 24);
}

static __device__ __forceinline__ int64_t omega_of(int n, int l, int m) {
  return (int64_t)n * (n - 1) * (2 * n - 1) / 6 + (int64_t)l * (l + 1) + m;
}


}  // namespace tcx
}  // namespace sgl
