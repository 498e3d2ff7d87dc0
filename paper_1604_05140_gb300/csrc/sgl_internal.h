// Internal declarations of the SGL transform library (not part of the ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <cmath>
#include <string>
#include <map>
#include <vector>

#include "../../include/sgl.h"

namespace sgl {

// ---------------------------------------------------------------------------
// Host FP64 tables of one bandlimit (tables.cpp)
// ---------------------------------------------------------------------------
struct HostTables {
  int B = 0;
  int R = 0;                               // radii: B, or 2B on the paper's grid
  std::vector<double> t, r, what;          // [R]   radial nodes t_i = r_i^2, weights what_i
  std::vector<double> theta, phi, beta;    // [2B]  sphere rule (Thm 3.1, beta = pi/B b_j)
  std::vector<double> lam;                 // [m][l][j'] m,l < B, j' < B: Lambda_lm(theta_j')
  std::vector<double> T;                   // [l][n-1][i < R]: N_nl R_nl(r_i) exp(-t_i/2)
  // seminaive Legendre transform: cosine coefficients of Lambda_lm / w_m
  // (w_m = sin theta for odd m) in the frequencies 2k' (l - m even) or 2k'+1
  // (l - m odd), k' < B, zero beyond the degree: [m][l][k']
  std::vector<double> lcos;
};

// Builds every table for bandlimit B (1 <= B <= SGL_MAX_B) on the radial grid
// `grid` (an sgl_grid_kind).  Returns false and sets msg on failure.
bool build_tables(int B, int grid, HostTables& out, std::string& msg);

// Radii of the grid of bandlimit B.
inline int n_radial(int B, int grid) { return grid == SGL_GRID_HALF_RANGE_HERMITE ? 2 * B : B; }

// Number of degrees l >= m with (l - m) % 2 == p, l < B.
inline int n_par(int B, int m, int p) {
  int first = m + p;
  return first >= B ? 0 : (B - 1 - first) / 2 + 1;
}

// Largest power of two dividing n, capped at 16.
inline int fft_n1(int n) {
  int p = 1;
  while (p < 16 && n % (2 * p) == 0) p *= 2;
  return p;
}

inline bool bandlimit_supported(int B) {
  if (B < 1 || B > SGL_MAX_B) return false;
  int n = 2 * B;
  return n / fft_n1(n) <= 16;
}

// Plans whose Legendre and radial stages run on the tensor cores, and the
// number of TF32 products per K step they use (hi*hi [+ hi*lo + lo*hi]).
inline bool tc_precision(int prec) {
  return prec == SGL_TF32X3 || prec == SGL_TF32 || prec == SGL_BF16X3 || prec == SGL_FP16X3;
}
inline int tc_products(int prec) { return prec == SGL_TF32 ? 1 : 3; }
// operand format of the tensor-core stages: TF32 (kind::tf32), or 16-bit
// hi/lo pairs on the kind::f16 path, BF16 or scaled FP16
enum TcOperand { TC_OP_TF32 = 0, TC_OP_BF16 = 1, TC_OP_FP16 = 2 };
inline int tc_operand(int prec) {
  return prec == SGL_BF16X3 ? TC_OP_BF16 : prec == SGL_FP16X3 ? TC_OP_FP16 : TC_OP_TF32;
}
inline bool tc_bf16(int prec) { return tc_operand(prec) != TC_OP_TF32; }  // a 16-bit operand path

// FP16x3 scales.  Data: per function, the largest magnitude of a stage's input
// (measured, or a measured magnitude times a bound on the growth through a
// table) as the bits of a non-negative float; slots of Plan::d_amax:
enum AmaxSlot { AMAX_EO = 0, AMAX_COEF = 1, AMAX_SLOTS = 2 };
// Power-of-two exponent e that puts a largest magnitude x into [2^13, 2^14)
// (x * 2^e), so that FP16 hi parts stay below 65504 and small values keep
// 28 binades of normal range; 0 for x = 0, clamped to +-100.
inline int fp16_scale_exp(double x) {
  if (!(x > 0)) return 0;
  int E = 0;
  (void)std::frexp(x, &E);  // x = f 2^E, f in [0.5, 1)
  int e = 14 - E;
  return e > 100 ? 100 : e < -100 ? -100 : e;
}

inline int64_t coeff_count(int B) { return (int64_t)B * (B + 1) * (2 * B + 1) / 6; }
// samples of one function: R radii x 2B x 2B (R = B, or 2B on the paper's grid)
inline int64_t sample_count(int B, int R) { return 4LL * R * B * B; }

// ---------------------------------------------------------------------------
// Table and workspace layouts (reals)
// ---------------------------------------------------------------------------
// Misc block of one bandlimit with R radii:
//   [0, R)            what_i
//   [R, 2R)           exp(-t_i/2)
//   [2R, 3R)          exp(+t_i/2)
//   [3R, 3R+2B)       beta_j, j < 2B
//   [3R+2B, 3R+6B)    twiddles e^{-2 pi i k/(2B)} as (re, im), k < 2B
inline int64_t misc_size(int B, int R) { return 3LL * R + 6LL * B; }

// Legendre block: for m = 0..B-1, p = 0,1: n_par(B,m,p) rows of B reals over
// the half grid j' < B; row q of (m,p) is degree l = m + p + 2q.
inline int64_t leg_rows_before(int B, int m, int p) {
  int64_t rows = (int64_t)m * B - (int64_t)m * (m - 1) / 2;
  if (p == 1) rows += n_par(B, m, 0);
  return rows;
}
inline int64_t leg_table_size(int B) { return (int64_t)B * (B + 1) / 2 * B; }
// Radial block: [l][n' < B-l][i < R], row n' is degree n = l + 1 + n'.
inline int64_t rad_rows_before(int B, int l) { return (int64_t)l * B - (int64_t)l * (l - 1) / 2; }
inline int64_t rad_table_size(int B, int R) { return (int64_t)B * (B + 1) / 2 * R; }

// Workspaces of a segment of NB functions with one bandlimit B and R radii
// (the tensor-core path stores W1 inverse as [m_idx][b][j][i][c] and S_i rows
// as [b][i][c], R = B there):
//   W1 forward "EO":  [m_idx < 2B-1][p<2][b<NB][c<2][i<R][j'<B]      (E = G_j'+G_mirror, O = G_j'-G_mirror)
//   W1 inverse "G":   [m_idx < 2B-1][b<NB][c<2][i<R][j<2B]
//   W2 forward "S_f": block l at NB*2*R*l^2: [b][m+l < 2l+1][c][i<R]
//   W2 inverse "S_i": block (m_idx,p) at NB*2*R*si_rows_before: [l'<n_par][b][c][i<R]
inline int64_t w1_size(int B, int NB, int R) { return 4LL * NB * R * B * (2 * B - 1); }
inline int64_t w2_size(int B, int NB, int R) { return 2LL * NB * B * B * R; }
inline int64_t si_rows_before(int B, int m_idx, int p) {
  int64_t rows = 0;
  for (int mi = 0; mi < m_idx; ++mi) {
    int am = mi - (B - 1);
    rows += B - (am < 0 ? -am : am);
  }
  if (p == 1) {
    int am = m_idx - (B - 1);
    rows += n_par(B, am < 0 ? -am : am, 0);
  }
  return rows;
}

// Contiguous slices of an ordered tile list for `grid` persistent CTAs with
// about equal estimated cost each: tile t goes to the CTA in whose share of
// the total cost the tile's midpoint falls.  Returns grid + 1 offsets (CTA k
// runs tiles first[k] .. first[k+1]-1; a slice may be empty) and the largest
// slice in *max_slice.
inline std::vector<int> balance_slices(const std::vector<double>& cost, int grid, int* max_slice) {
  const int n = (int)cost.size();
  std::vector<int> first(grid + 1, n);
  double total = 0.0;
  for (double c : cost) total += c;
  int k = 0;
  double p = 0.0;
  for (int t = 0; t < n; ++t) {
    const double mid = p + 0.5 * cost[t];
    int c = total > 0.0 ? (int)(mid / total * grid) : 0;
    if (c > grid - 1) c = grid - 1;
    while (k <= c) first[k++] = t;
    p += cost[t];
  }
  while (k <= grid) first[k++] = n;
  int mx = 0;
  for (int j = 0; j < grid; ++j) mx = first[j + 1] - first[j] > mx ? first[j + 1] - first[j] : mx;
  *max_slice = mx;
  return first;
}

// ---------------------------------------------------------------------------
// Segments: functions of one bandlimit processed together
// ---------------------------------------------------------------------------
struct SegDesc {
  int B, NB;          // bandlimit, functions in the segment
  int n1, n2;         // 2B = n1 * n2 (phi-FFT factors)
  int fn0;            // first entry of the segment in the per-function offset arrays
  int R;              // radii: B, or 2B on the paper's grid
  int64_t w1_off, w2_off;               // reals
  int64_t tab_leg_f, tab_leg_i;         // reals: Legendre tables (fwd: * beta, inv: plain)
  int64_t tab_rad_f, tab_rad_i;         // reals: radial tables (fwd: * what, inv: plain)
  int64_t tab_misc;                     // reals
  int64_t si_rows;                      // offset of the segment's S_i row table in d_si_rows
  // seminaive Legendre transform (SIMT plans): cosine coefficients of
  // Lambda_lm / w_m in the Legendre block layout, then 5B reals of DCT
  // twiddles: cos, sin of pi k / 2B; cos, sin of pi (2k+1) / 4B; sin theta_j'
  int64_t tab_leg_s, tab_dct;
};

// Tile of a GEMM stage: (segment, group, row0, col0)
// FFT CTA:            (segment, shell = b*R + i, j'0, 0)

// Tile lists of one SIMT GEMM stage, one per tile shape w: 64 x 64 (w = 0),
// 128 x 32 (1), 256 x 16 (2) and 64 x 48 (3) outputs (rows x columns); a
// group's columns are covered by whole 64-column blocks, the rest by the
// narrowest shape that holds it (kernels.cu).
constexpr int kGemmShapes = 4;
constexpr int kDctVec = 16;  // vectors per CTA of the seminaive DCT kernel
inline int gemm_shape_of(int ncols) { return ncols <= 16 ? 2 : ncols <= 32 ? 1 : ncols <= 48 ? 3 : 0; }
inline int gemm_shape_cols(int w) { return w == 3 ? 48 : 64 >> w; }
inline int gemm_shape_rows(int w) { return w == 3 ? 64 : 64 << w; }
struct GemmSched {
  int4* d_tiles[kGemmShapes] = {nullptr, nullptr, nullptr, nullptr};
  int ntiles[kGemmShapes] = {0, 0, 0, 0};
  int launches() const {
    int n = 0;
    for (int w = 0; w < kGemmShapes; ++w) n += ntiles[w] > 0;
    return n;
  }
};

struct Plan {
  int prec = SGL_FP64;
  int samples = SGL_SAMPLES_WEIGHTED;
  int grid = SGL_GRID_LAGUERRE;  // radial grid (sgl_grid_kind)
  int nfn = 0;
  bool uniform = true;
  int maxB = 0;
  int64_t n_samples = 0, n_coeffs = 0;           // complex elements, whole plan
  std::vector<int> fn_B;                         // user order
  std::vector<int64_t> fn_samp_off, fn_coef_off; // user order, complex elements
  std::vector<SegDesc> segs;
  std::vector<int> seg_fn;                       // per segment order: user function index
  std::vector<HostTables> tables;                // one per segment
  int device = 0;

  // device memory
  void* d_tab = nullptr;        // tables in the plan's real type (hi parts for TF32x3)
  void* d_tab_lo = nullptr;     // TF32x3 lo parts of the Legendre / radial tables
  void* d_w1 = nullptr;
  void* d_w2 = nullptr;
  void* d_stage_in = nullptr;
  void* d_stage_out = nullptr;
  size_t stage_in_bytes = 0, stage_out_bytes = 0;
  SegDesc* d_segs = nullptr;
  int64_t* d_fn_samp = nullptr; // per segment order
  int64_t* d_fn_coef = nullptr;
  int64_t* d_si_rows = nullptr; // per segment: [(2B-1)*2] rows-before of S_i blocks
  int* d_err = nullptr;
  int64_t bytes = 0;
  int64_t w1_elems = 0, w2_elems = 0, tab_elems = 0;

  GemmSched leg_fwd, rad_fwd, rad_inv, leg_inv;
  int4* d_fft_fwd = nullptr;
  int4* d_fft_inv = nullptr;
  int n_fft_fwd = 0, n_fft_inv = 0;
  int launches_per_call = 0;
  void* tc_state = nullptr;      // tensor-core forward stage state (tc_gemm.cu)
  int64_t tc_bytes = 0;          // device bytes of the tensor-core state (both directions)
  void* tc_inv_state = nullptr;  // tensor-core inverse stage state (tc_inv.cu)

  // launch configuration chosen by sgl_autotune: ring pairs per CTA of the
  // forward and inverse phi-FFT (0: default), and the number of radial terms
  // B - l from which the TF32x3 inverse radial stage cuts 64-column tiles
  // with two K chains (smaller counts get 128-column tiles)
  int jp_fwd = 0, jp_inv = 0;
  int radi_narrow = 65;
  // tile shapes chosen by sgl_autotune: the SIMT tile family of each GEMM
  // stage (0 LEG_F, 1 RAD_F, 2 RAD_I, 3 LEG_I; see build_simt_lists in
  // api.cu), and the rows n' of the largest table group of the tensor-core
  // forward radial stage (its MMA tile width; 32, 48 or 64)
  int simt_policy[4] = {0, 0, 0, 0};
  int rad_rows = 64;
  // plans of several register-FFT sizes: one multi-size phi-FFT launch per
  // direction (1) or one launch per size (0)
  int fft_merge = 1;
  // work-queue slices per CTA of each tensor-core stage (1, 2, 4 or 8):
  // forward Legendre, forward radial, inverse radial, Legendre synthesis
  int queue_slices[4] = {2, 2, 2, 2};
  // CTA order of the tensor-core plans' inverse phi-FFT: shell blocks outer
  // (0) or ring pairs outer (1)
  int fft_inv_order = 0;
  std::string tuning;

  // FP16x3 plans: per-function largest magnitudes [AMAX_SLOTS][nfn] (segment
  // order), cleared and measured by every call (the data scales)
  unsigned* d_amax = nullptr;

  // calls with host buffers on single-bandlimit plans run in chunks of
  // functions so that the copies overlap the kernels (api.cu): one sub-plan
  // per chunk size of the schedules (sizes growing from a small first chunk
  // when the input is on the host, shrinking to a small last chunk when the
  // output is), copy streams and events.  Sub-plans share the parent's error
  // flag.
  std::map<int, Plan*> subs;
  cudaStream_t copy_stream = nullptr;       // host-to-device copies of the chunks
  cudaStream_t copy_back_stream = nullptr;  // device-to-host copies (the other direction of the link)
  std::vector<cudaEvent_t> pipe_ev;
  bool owns_err = true;

  // stage timing (sgl_set_profiling): event pairs per stage, and a free pool
  bool profiling = false;
  std::vector<std::pair<cudaEvent_t, cudaEvent_t>> prof_ev[SGL_NUM_STAGES];
  std::vector<cudaEvent_t> ev_pool;

  // real functions (SGL_SAMPLES_REAL): the plan's nfn complex functions
  // carry the nreal user functions in pairs (function 2q as the real part of
  // complex function q, 2q + 1 as its imaginary part); n_samples counts the
  // user's reals, n_coeffs the user's complex coefficients, and the complex
  // coefficients of the pairs live in d_ccoef
  bool real_pairs = false;
  int nreal = 0;
  void* d_ccoef = nullptr;
  // tensor-core plans on the paper's grid: each function's 2B radii run as
  // two functions of B radii (its first and second half of the radial rule:
  // two segments with their own radial tables); nfn counts those halves,
  // nuser the caller's functions.  d_ccoef holds the halves' coefficients:
  // the forward sums each function's two partial sums, the inverse gives both
  // halves the function's coefficients.  Real functions on the paper's grid
  // take both forms: nuser counts the complex pairs, each pair's two halves
  // are functions 2q and 2q + 1 (half h of the pair reads half h of both of
  // its real functions), and d_pcoef holds the pairs' coefficients between
  // the halves' sum (or copy) and the split into real functions.
  bool radial_halves = false;
  int nuser = 0;
  void* d_pcoef = nullptr;

  // forward Legendre stage by the seminaive algorithm (sgl_set_dlt, SIMT
  // plans): DCT CTA list (segment, first vector, vectors, 0)
  bool seminaive = false;
  int4* d_dct_ctas = nullptr;
  int n_dct = 0;

  // CUDA graphs of the plan's own calls (sgl_set_graphs): one per call kind
  // (direction, weights) and device buffer pair, captured on first use on a
  // plan-owned stream and replayed on the caller's stream; the least recently
  // used one is dropped beyond kMaxGraphs
  struct GraphEntry {
    int kind;
    const void* in;
    void* out;
    cudaGraphExec_t exec;
    uint64_t used;
  };
  static constexpr size_t kMaxGraphs = 8;
  bool use_graphs = false;
  cudaStream_t graph_stream = nullptr;
  std::vector<GraphEntry> graphs;
  uint64_t graph_clock = 0;

  std::string err;
  int latched = SGL_OK;
};

enum Stage { ST_FFT_F = 0, ST_LEG_F = 1, ST_RAD_F = 2, ST_RAD_I = 3, ST_LEG_I = 4, ST_FFT_I = 5 };

// Records a start event on construction and a stop event on finish() when the
// plan is profiling; otherwise does nothing.
struct StageTimer {
  Plan& P;
  int stage;
  cudaStream_t s;
  cudaEvent_t a = nullptr;
  StageTimer(Plan& p, int st, cudaStream_t str) : P(p), stage(st), s(str) {
    if (P.profiling) {
      a = take();
      cudaEventRecord(a, s);
    }
  }
  cudaEvent_t take() {
    if (!P.ev_pool.empty()) {
      cudaEvent_t e = P.ev_pool.back();
      P.ev_pool.pop_back();
      return e;
    }
    cudaEvent_t e;
    cudaEventCreate(&e);
    return e;
  }
  void finish() {
    if (P.profiling && a) {
      cudaEvent_t b = take();
      cudaEventRecord(b, s);
      P.prof_ev[stage].push_back({a, b});
      a = nullptr;
    }
  }
};

// Arguments of the specialized phi-FFT kernels for 2B = 16 * N2, N2 in {8, 16}
// (fft16.cu).  mode: forward 0 none, 1 *exp(-t/2), 2 *exp(+t/2); inverse
// 0 none, 1 *exp(+t/2), 2 *what*beta, 3 *what*beta*exp(-t/2).
struct Fft16Args {
  const SegDesc* segs;
  const int64_t* fn_samp;
  const int4* ctas;      // (segment, shell, j'0, 0)
  const void* tab;
  const void* in;
  void* out;
  void* w1;
  int JP;                // ring pairs per CTA; blockDim = 16 * JP
  int mode;
  // real functions in pairs: 0 for complex samples, else the number of
  // reals in the sample array (the second function of the last pair exists
  // only below this limit)
  int64_t pair_limit;
  unsigned* amax;        // forward, FP16x3 plans: per-function largest |E/O| (else null)
  // real functions in pairs: reals from a sample of the pair's first function
  // to the same sample of its second (one function's reals)
  int64_t pair_gap;
};
// Largest magnitude of a CTA's values, folded into *amax (bits of a
// non-negative float, compared as integers) with one atomic per CTA; each
// thread passes the largest |value| it produced.  Every thread of the CTA
// calls it, with the same amax.
#ifdef __CUDACC__
__device__ __forceinline__ void cta_amax(float v, unsigned* amax) {
  __shared__ unsigned s_amax;
  if (threadIdx.x == 0) s_amax = 0u;
  __syncthreads();
  const unsigned w = __reduce_max_sync(__activemask(), __float_as_uint(v));
  if ((threadIdx.x & 31) == 0) atomicMax(&s_amax, w);
  __syncthreads();
  if (threadIdx.x == 0 && s_amax != 0u) atomicMax(amax, s_amax);
}
#endif

// Launches the register FFT when it takes 2B = n1 * n2 (fft16_handles) and
// returns true (launch status in *err); returns false otherwise.
template <typename real>
bool fft16_launch(bool inv, const Fft16Args& a, int n1, int n2, int nctas, cudaStream_t s, cudaError_t* err);
// Whether the register FFT takes rings of 2B = n1 * n2 (fft16.cu).
bool fft16_handles(bool fp64, bool pairs, int n1, int n2);
// One launch of the multi-size register FFT (FP32 complex samples) over
// nctas CTAs of segments with n2 <= max_n2; false when it does not apply.
bool fft16_launch_multi(bool inv, const Fft16Args& a, int max_n2, int nctas, cudaStream_t s, cudaError_t* err);

// Packs the host tables of every segment of P into one array of the plan's
// real type, at the offsets recorded in the segment descriptors (api.cu).
template <typename real>
void pack_tables(const Plan& P, std::vector<real>& tab);

// Stage launchers (kernels.cu)
cudaError_t run_forward(Plan& P, const void* samples, void* coeffs, cudaStream_t s, bool weights);
cudaError_t run_inverse(Plan& P, const void* coeffs, void* samples, cudaStream_t s, bool weights);

// Default ring pairs per phi-FFT CTA (kernels.cu), and the plan's choice for
// one direction (the tuned value where set), at most B.
int fft_pairs_per_cta(int prec, int B);
inline int fft_jp(const Plan& P, int B, bool inv) {
  int jp = inv ? P.jp_inv : P.jp_fwd;
  if (jp <= 0) jp = fft_pairs_per_cta(P.prec, B);
  return jp < B ? jp : B;
}

// phi-FFT launches of one call in direction inv (kernels.cu).
int fft_launches(const Plan& P, bool inv);

// Rebuilds the TF32x3 inverse radial tiles for P.radi_narrow (tc_inv.cu).
cudaError_t tc_radi_retile(Plan& P);

}  // namespace sgl
