// C ABI of the SGL transform library: plans, dispatch, host-buffer staging.
#include <cuda_runtime.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "sgl_internal.h"

namespace sgl {
size_t fft_smem_for(int prec, int n1, int n2, int B);
void gemm_tile_dims(int& tm, int& tn, int& tk);
cudaError_t tc_prepare(Plan& P);   // tensor-core tables and schedules (tc_gemm.cu)
void tc_release(Plan& P);
}  // namespace sgl

using namespace sgl;

// Failures that have no plan to hold their message (plan creation, plan-free
// entry points); one per thread, so concurrent creations keep their own.
static thread_local std::string g_create_error;

namespace sgl {
// Message returned by sgl_last_error(NULL) on the calling thread.
void set_global_error(const std::string& msg) { g_create_error = msg; }
}  // namespace sgl

static sgl_status fail(Plan* P, sgl_status st, const std::string& msg) {
  if (P) P->err = msg; else g_create_error = msg;
  return st;
}

static sgl_status cuda_fail(Plan* P, cudaError_t e, const char* where) {
  std::string msg = std::string(where) + ": " + cudaGetErrorString(e);
  return fail(P, SGL_ERR_CUDA, msg);
}

template <typename T>
static cudaError_t dev_upload(Plan& P, T** dst, const std::vector<T>& src) {
  if (src.empty()) { *dst = nullptr; return cudaSuccess; }
  cudaError_t e = cudaMalloc((void**)dst, src.size() * sizeof(T));
  if (e != cudaSuccess) return e;
  P.bytes += src.size() * sizeof(T);
  return cudaMemcpy(*dst, src.data(), src.size() * sizeof(T), cudaMemcpyHostToDevice);
}

static void clear_profile(Plan& P) {
  for (int st = 0; st < SGL_NUM_STAGES; ++st) {
    for (auto& pr : P.prof_ev[st]) {
      P.ev_pool.push_back(pr.first);
      P.ev_pool.push_back(pr.second);
    }
    P.prof_ev[st].clear();
  }
}

static void release_pipeline(Plan* P);

// Destroys the plan's captured graphs (their launches no longer match the
// plan's schedules, or graphs were switched off).
static void drop_graphs(Plan& P) {
  for (Plan::GraphEntry& g : P.graphs) cudaGraphExecDestroy(g.exec);
  P.graphs.clear();
}

static void release(Plan* P) {
  if (!P) return;
  int cur = 0;
  cudaGetDevice(&cur);
  cudaSetDevice(P->device);
  drop_graphs(*P);
  if (P->graph_stream) cudaStreamDestroy(P->graph_stream);
  release_pipeline(P);
  clear_profile(*P);
  for (cudaEvent_t e : P->ev_pool) cudaEventDestroy(e);
  tc_release(*P);
  if (!P->owns_err) P->d_err = nullptr;
  void* ptrs[] = {P->d_tab, P->d_tab_lo, P->d_w1, P->d_w2, P->d_stage_in, P->d_stage_out, P->d_segs,
                  P->d_fn_samp, P->d_fn_coef, P->d_si_rows, P->d_err, P->d_fft_fwd, P->d_fft_inv, P->d_ccoef,
                  P->d_pcoef, P->d_dct_ctas, P->d_amax};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  for (GemmSched* g : {&P->leg_fwd, &P->rad_fwd, &P->rad_inv, &P->leg_inv})
    for (int w = 0; w < kGemmShapes; ++w)
      if (g->d_tiles[w]) cudaFree(g->d_tiles[w]);
  cudaSetDevice(cur);
  delete P;
}

static void release_pipeline(Plan* P) {
  for (auto& kv : P->subs) release(kv.second);
  P->subs.clear();
  for (cudaEvent_t e : P->pipe_ev) cudaEventDestroy(e);
  P->pipe_ev.clear();
  if (P->copy_stream) cudaStreamDestroy(P->copy_stream);
  if (P->copy_back_stream) cudaStreamDestroy(P->copy_back_stream);
  P->copy_stream = P->copy_back_stream = nullptr;
}

// Host tables depend on the bandlimit and the radial grid only; built once
// per process.
static bool cached_tables(int B, int grid, HostTables& out, std::string& msg) {
  static std::mutex mu;
  static std::map<std::pair<int, int>, HostTables> cache;
  std::lock_guard<std::mutex> lock(mu);
  auto it = cache.find({B, grid});
  if (it == cache.end()) {
    HostTables H;
    if (!build_tables(B, grid, H, msg)) return false;
    it = cache.emplace(std::make_pair(B, grid), std::move(H)).first;
  }
  out = it->second;
  return true;
}

// Half h of a radial rule of 2B nodes (the paper's grid) as a rule of B
// nodes: nodes, weights and radial functions at radii h B .. h B + B - 1
// (the radial sums of Eq. DRT_matrix split into two partial sums); the
// sphere tables are unchanged.
static HostTables radial_half(const HostTables& H, int h) {
  HostTables out = H;
  const int B = H.B, R = H.R, i0 = h * B;
  out.R = B;
  out.t.assign(H.t.begin() + i0, H.t.begin() + i0 + B);
  out.r.assign(H.r.begin() + i0, H.r.begin() + i0 + B);
  out.what.assign(H.what.begin() + i0, H.what.begin() + i0 + B);
  const size_t rows = H.T.size() / (size_t)R;  // (l, n-1) rows of R radii
  out.T.assign(rows * (size_t)B, 0.0);
  for (size_t q = 0; q < rows; ++q)
    std::copy(H.T.begin() + q * R + i0, H.T.begin() + q * R + i0 + B, out.T.begin() + q * B);
  return out;
}

template <typename real>
void sgl::pack_tables(const Plan& P, std::vector<real>& tab) {
  tab.assign(P.tab_elems, real(0));
  for (size_t s = 0; s < P.segs.size(); ++s) {
    const SegDesc& sg = P.segs[s];
    const HostTables& H = P.tables[s];
    const int B = sg.B, R = sg.R;
    real* misc = tab.data() + sg.tab_misc;
    for (int i = 0; i < R; ++i) {
      misc[i] = (real)H.what[i];
      misc[R + i] = (real)exp(-0.5 * H.t[i]);
      misc[2 * R + i] = (real)exp(0.5 * H.t[i]);
    }
    for (int j = 0; j < 2 * B; ++j) misc[3 * R + j] = (real)H.beta[j];
    for (int k = 0; k < 2 * B; ++k) {
      // e^{-2 pi i k / 2B}
      long double ang = 3.141592653589793238462643383279502884L * (long double)k / (long double)B;
      misc[3 * R + 2 * B + 2 * k] = (real)cosl(ang);
      misc[3 * R + 2 * B + 2 * k + 1] = (real)(-sinl(ang));
    }
    for (int m = 0; m < B; ++m)
      for (int p = 0; p < 2; ++p) {
        const int64_t r0 = leg_rows_before(B, m, p);
        for (int q = 0; q < n_par(B, m, p); ++q) {
          const int l = m + p + 2 * q;
          for (int j = 0; j < B; ++j) {
            const double v = H.lam[((size_t)m * B + l) * B + j];
            tab[sg.tab_leg_f + (r0 + q) * B + j] = (real)(H.beta[j] * v);
            tab[sg.tab_leg_i + (r0 + q) * B + j] = (real)v;
          }
        }
      }
    for (int m = 0; m < B; ++m)
      for (int p = 0; p < 2; ++p) {
        const int64_t r0 = leg_rows_before(B, m, p);
        for (int q = 0; q < n_par(B, m, p); ++q) {
          const int l = m + p + 2 * q;
          for (int k = 0; k < B; ++k) tab[sg.tab_leg_s + (r0 + q) * B + k] = (real)H.lcos[((size_t)m * B + l) * B + k];
        }
      }
    for (int k = 0; k < B; ++k) {
      const long double pi = 3.141592653589793238462643383279502884L;
      tab[sg.tab_dct + k] = (real)cosl(pi * k / (2.0L * B));
      tab[sg.tab_dct + B + k] = (real)sinl(pi * k / (2.0L * B));
      tab[sg.tab_dct + 2 * B + k] = (real)cosl(pi * (2.0L * k + 1.0L) / (4.0L * B));
      tab[sg.tab_dct + 3 * B + k] = (real)sinl(pi * (2.0L * k + 1.0L) / (4.0L * B));
      tab[sg.tab_dct + 4 * B + k] = (real)sinl(pi * (2.0L * k + 1.0L) / (4.0L * B));  // sin theta_k
    }
    for (int l = 0; l < B; ++l) {
      const int64_t r0 = rad_rows_before(B, l);
      for (int q = 0; q < B - l; ++q) {
        const int n = l + 1 + q;
        for (int i = 0; i < R; ++i) {
          const double v = H.T[((size_t)l * B + (n - 1)) * R + i];
          tab[sg.tab_rad_f + (r0 + q) * R + i] = (real)(H.what[i] * v);
          tab[sg.tab_rad_i + (r0 + q) * R + i] = (real)v;
        }
      }
    }
  }
}

template void sgl::pack_tables<double>(const Plan& P, std::vector<double>& tab);
template void sgl::pack_tables<float>(const Plan& P, std::vector<float>& tab);

// Kernel launches of one forward (or inverse) call, the larger of the two
// directions: the phi-FFT launches and the stage launches (one per
// tensor-core stage, one per tile shape of a SIMT stage).
static void set_launch_count(Plan& P) {
  int fwd = fft_launches(P, false), inv = fft_launches(P, true);
  if (tc_precision(P.prec)) {
    fwd += 2;
    inv += 2 + (tc_operand(P.prec) == TC_OP_FP16 ? 1 : 0);  // FP16x3: the coefficients' magnitudes
  } else {
    fwd += P.leg_fwd.launches() + P.rad_fwd.launches() + (P.seminaive ? (int)P.segs.size() : 0);
    inv += P.rad_inv.launches() + P.leg_inv.launches();
  }
  P.launches_per_call = std::max(fwd, inv) + (P.real_pairs ? 1 : 0) + (P.radial_halves ? 1 : 0);
}

// FFT CTA lists of both directions (segment order) for the plan's current
// ring pairs per CTA; replaces the previous lists.
static cudaError_t build_fft_lists(Plan& P) {
  std::vector<int4> ff;
  for (size_t s = 0; s < P.segs.size(); ++s) {
    const SegDesc& sg = P.segs[s];
    const int JP = fft_jp(P, sg.B, false);
    for (int sh = 0; sh < sg.NB * sg.R; ++sh)
      for (int j0 = 0; j0 < sg.B; j0 += JP) ff.push_back(make_int4((int)s, sh, j0, 0));
  }
  if (P.d_fft_fwd) {
    cudaFree(P.d_fft_fwd);
    P.d_fft_fwd = nullptr;
    P.bytes -= (int64_t)P.n_fft_fwd * sizeof(int4);
  }
  P.n_fft_fwd = (int)ff.size();
  cudaError_t e = dev_upload(P, &P.d_fft_fwd, ff);
  if (e != cudaSuccess) return e;
  ff.clear();
  for (size_t s = 0; s < P.segs.size(); ++s) {
    const SegDesc& sg = P.segs[s];
    const int JP = fft_jp(P, sg.B, true);
    if (tc_precision(P.prec)) {
      // the tensor-core Legendre synthesis stores spectra [m][b][j][i][c]: each
      // inverse-FFT CTA takes JP consecutive shells of one ring pair (layout 1).
      // CTA order (tuned): shell blocks outer (consecutive CTAs read other
      // rings), or ring pairs outer (consecutive CTAs read the neighbouring
      // pieces of the same runs of shells)
      for (int b = 0; b < sg.NB; ++b) {
        if (P.fft_inv_order == 0) {
          for (int i0 = 0; i0 < sg.R; i0 += JP)
            for (int jp = 0; jp < sg.B; ++jp) ff.push_back(make_int4((int)s, b * sg.R + i0, jp, 1));
        } else {
          for (int jp = 0; jp < sg.B; ++jp)
            for (int i0 = 0; i0 < sg.R; i0 += JP) ff.push_back(make_int4((int)s, b * sg.R + i0, jp, 1));
        }
      }
    } else {
      for (int sh = 0; sh < sg.NB * sg.R; ++sh)
        for (int j0 = 0; j0 < sg.B; j0 += JP) ff.push_back(make_int4((int)s, sh, j0, 0));
    }
  }
  if (P.d_fft_inv) {
    cudaFree(P.d_fft_inv);
    P.d_fft_inv = nullptr;
    P.bytes -= (int64_t)P.n_fft_inv * sizeof(int4);
  }
  P.n_fft_inv = (int)ff.size();
  return dev_upload(P, &P.d_fft_inv, ff);
}

// SIMT GEMM tile lists of every stage (0 LEG_F, 1 RAD_F, 2 RAD_I, 3 LEG_I)
// for the plan's tile-family policy of that stage (Plan::simt_policy):
//   0  whole blocks of 64 columns, the rest in the narrowest shape that holds
//      it (the default: least padding);
//   1  64 x 64 tiles only (fewest tiles);
//   2  blocks of 32 columns (128 x 32 tiles), a rest of <= 16 in 256 x 16.
// Replaces the previous lists.
static cudaError_t build_simt_lists(Plan& P) {
  std::vector<int4> lists[4][kGemmShapes];
  auto add = [&](int stage, int s, int g, int rows, int ncols) {
    const int pol = P.simt_policy[stage];
    for (int c0 = 0; c0 < ncols;) {
      const int rest = ncols - c0;
      const int w = pol == 1 ? 0 : pol == 2 ? (rest <= 16 ? 2 : 1) : gemm_shape_of(rest);
      const int tm = gemm_shape_rows(w), tn = gemm_shape_cols(w);
      for (int r0 = 0; r0 < rows; r0 += tm) lists[stage][w].push_back(make_int4(s, g, r0, c0));
      c0 += tn;
    }
  };
  for (size_t s = 0; s < P.segs.size(); ++s) {
    const SegDesc& sg = P.segs[s];
    const int B = sg.B, NB = sg.NB, R = sg.R;
    for (int g = 0; g < 2 * (2 * B - 1); ++g) {
      const int m = (g >> 1) - (B - 1);
      add(0, (int)s, g, NB * 2 * R, n_par(B, m < 0 ? -m : m, g & 1));
    }
    for (int l = 0; l < B; ++l) {
      const int rows = NB * (2 * l + 1) * 2;
      add(1, (int)s, l, rows, B - l);
      add(2, (int)s, l, rows, R);
    }
    for (int mi = 0; mi < 2 * B - 1; ++mi) add(3, (int)s, mi, NB * 2 * R, B);
  }
  GemmSched* scheds[4] = {&P.leg_fwd, &P.rad_fwd, &P.rad_inv, &P.leg_inv};
  for (int st = 0; st < 4; ++st)
    for (int w = 0; w < kGemmShapes; ++w) {
      if (scheds[st]->d_tiles[w]) {
        cudaFree(scheds[st]->d_tiles[w]);
        P.bytes -= (int64_t)scheds[st]->ntiles[w] * sizeof(int4);
        scheds[st]->d_tiles[w] = nullptr;
      }
      scheds[st]->ntiles[w] = (int)lists[st][w].size();
      const cudaError_t e = dev_upload(P, &scheds[st]->d_tiles[w], lists[st][w]);
      if (e != cudaSuccess) return e;
    }
  return cudaSuccess;
}

static sgl_status build_plan(Plan* P, const std::vector<int>& Bs, bool uniform) {
  cudaGetDevice(&P->device);
  P->nfn = (int)Bs.size();
  P->uniform = uniform;
  P->fn_B = Bs;
  // offsets in user order (radial halves: the halves in order, B radii each)
  const int grid_fn = P->radial_halves ? SGL_GRID_LAGUERRE : P->grid;  // radii of one function
  int64_t so = 0, co = 0;
  for (int B : Bs) {
    P->fn_samp_off.push_back(so);
    P->fn_coef_off.push_back(co);
    so += sample_count(B, n_radial(B, grid_fn));
    co += coeff_count(B);
    P->maxB = std::max(P->maxB, B);
  }
  // real functions on the paper's grid: half h of pair q (function 2q + h)
  // starts, in reals, at half h of the pair's first real function
  if (P->real_pairs && P->radial_halves)
    for (int f = 0; f < P->nfn; ++f) P->fn_samp_off[f] = (2 * (int64_t)f - (f & 1)) * (so / P->nfn) / 2;
  P->n_samples = so;
  P->n_coeffs = co;
  // segments: group by bandlimit, largest first; radial halves: one segment
  // per half (even and odd functions), each with its half of the radial rule
  std::vector<std::pair<int, std::vector<int>>> by_B;
  if (P->radial_halves) {
    for (int h = 0; h < 2; ++h) {
      std::vector<int> fs;
      for (int f = h; f < P->nfn; f += 2) fs.push_back(f);
      by_B.push_back({Bs[0], fs});
    }
  } else {
    std::map<int, std::vector<int>, std::greater<int>> m;
    for (int f = 0; f < P->nfn; ++f) m[Bs[f]].push_back(f);
    for (auto& kv : m) by_B.push_back(kv);
  }
  int half = 0;
  std::vector<int64_t> fn_samp, fn_coef, si_rows;
  int64_t w1 = 0, w2 = 0, tab = 0;
  for (auto& kv : by_B) {
    SegDesc sg;
    memset(&sg, 0, sizeof(sg));
    sg.B = kv.first;
    sg.R = n_radial(sg.B, grid_fn);
    sg.NB = (int)kv.second.size();
    sg.n1 = fft_n1(2 * sg.B);
    sg.n2 = 2 * sg.B / sg.n1;
    sg.fn0 = (int)fn_samp.size();
    for (int f : kv.second) {
      fn_samp.push_back(P->fn_samp_off[f]);
      fn_coef.push_back(P->fn_coef_off[f]);
      P->seg_fn.push_back(f);
    }
    sg.w1_off = w1;
    sg.w2_off = w2;
    w1 += w1_size(sg.B, sg.NB, sg.R);
    w2 += w2_size(sg.B, sg.NB, sg.R);
    sg.tab_misc = tab;
    tab += misc_size(sg.B, sg.R);
    sg.tab_leg_f = tab;
    tab += leg_table_size(sg.B);
    sg.tab_leg_i = tab;
    tab += leg_table_size(sg.B);
    sg.tab_rad_f = tab;
    tab += rad_table_size(sg.B, sg.R);
    sg.tab_rad_i = tab;
    tab += rad_table_size(sg.B, sg.R);
    sg.tab_leg_s = tab;
    tab += leg_table_size(sg.B);
    sg.tab_dct = tab;
    tab += 5 * sg.B;
    tab = (tab + 31) / 32 * 32;
    sg.si_rows = (int64_t)si_rows.size();
    for (int mi = 0; mi < 2 * sg.B - 1; ++mi)
      for (int p = 0; p < 2; ++p) si_rows.push_back(si_rows_before(sg.B, mi, p));
    HostTables H;
    std::string msg;
    if (!cached_tables(sg.B, P->grid, H, msg)) return fail(P, SGL_ERR_ARG, "table generation: " + msg);
    if (P->radial_halves) H = radial_half(H, half++);
    P->tables.push_back(std::move(H));
    P->segs.push_back(sg);
  }
  P->w1_elems = w1;
  P->w2_elems = w2;
  P->tab_elems = tab;

  const size_t rsz = (P->prec == SGL_FP64) ? sizeof(double) : sizeof(float);
  cudaError_t e;
  // tables
  if (P->prec == SGL_FP64) {
    std::vector<double> t;
    pack_tables<double>(*P, t);
    e = dev_upload(*P, (double**)&P->d_tab, t);
  } else {
    std::vector<float> t;
    pack_tables<float>(*P, t);
    e = dev_upload(*P, (float**)&P->d_tab, t);
  }
  if (e != cudaSuccess) return cuda_fail(P, e, "table upload");
  e = dev_upload(*P, &P->d_segs, P->segs);
  if (e != cudaSuccess) return cuda_fail(P, e, "segment upload");
  e = dev_upload(*P, &P->d_fn_samp, fn_samp);
  if (e != cudaSuccess) return cuda_fail(P, e, "offset upload");
  e = dev_upload(*P, &P->d_fn_coef, fn_coef);
  if (e != cudaSuccess) return cuda_fail(P, e, "offset upload");
  e = dev_upload(*P, &P->d_si_rows, si_rows);
  if (e != cudaSuccess) return cuda_fail(P, e, "offset upload");
  // workspaces
  e = cudaMalloc(&P->d_w1, w1 * rsz);
  if (e != cudaSuccess) return fail(P, SGL_ERR_ALLOC, "workspace allocation failed");
  P->bytes += w1 * rsz;
  e = cudaMalloc(&P->d_w2, w2 * rsz);
  if (e != cudaSuccess) return fail(P, SGL_ERR_ALLOC, "workspace allocation failed");
  P->bytes += w2 * rsz;
  e = cudaMalloc((void**)&P->d_err, sizeof(int));
  if (e != cudaSuccess) return fail(P, SGL_ERR_ALLOC, "allocation failed");
  cudaMemset(P->d_err, 0, sizeof(int));
  if (tc_operand(P->prec) == TC_OP_FP16) {  // per-function largest magnitudes (data scales)
    const size_t n = (size_t)AMAX_SLOTS * P->nfn * sizeof(unsigned);
    e = cudaMalloc((void**)&P->d_amax, n);
    if (e != cudaSuccess) return fail(P, SGL_ERR_ALLOC, "allocation failed");
    P->bytes += n;
  }

  // SIMT GEMM schedules
  e = build_simt_lists(*P);
  if (e != cudaSuccess) return cuda_fail(P, e, "schedule upload");
  e = build_fft_lists(*P);
  if (e != cudaSuccess) return cuda_fail(P, e, "schedule upload");
  for (const SegDesc& sg : P->segs) {
    size_t smem = fft_smem_for(P->prec, sg.n1, sg.n2, sg.B);
    if (smem > 227 * 1024) return fail(P, SGL_ERR_UNSUPPORTED, "FFT tile exceeds shared memory");
  }
  if (tc_precision(P->prec)) {
    e = tc_prepare(*P);
    if (e != cudaSuccess) return cuda_fail(P, e, "tensor-core preparation");
  }
  set_launch_count(*P);
  return SGL_OK;
}

static bool is_device_ptr(const void* p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

static size_t complex_bytes(const Plan& P) { return P.prec == SGL_FP64 ? 16 : 8; }
// bytes of one element of the user's sample array (a real for real-function plans)
static size_t sample_bytes(const Plan& P) { return P.real_pairs ? complex_bytes(P) / 2 : complex_bytes(P); }
// functions as the user counts them
static int user_fns(const Plan& P) { return P.real_pairs ? P.nreal : P.radial_halves ? P.nuser : P.nfn; }

// Forward Legendre stage by the seminaive algorithm (or back to the direct
// sums); builds the DCT CTA list on first use.
static sgl_status set_dlt(Plan* P, bool on) {
  if (on && !P->d_dct_ctas) {
    std::vector<int4> v;
    for (size_t s = 0; s < P->segs.size(); ++s) {
      const SegDesc& sg = P->segs[s];
      const int64_t nvec = (int64_t)(2 * sg.B - 1) * 2 * sg.NB * 2 * sg.R;
      if (nvec >= ((int64_t)1 << 31)) return fail(P, SGL_ERR_UNSUPPORTED, "too many spectra for the DCT schedule");
      for (int64_t v0 = 0; v0 < nvec; v0 += kDctVec)
        v.push_back(make_int4((int)s, (int)v0, (int)std::min<int64_t>(kDctVec, nvec - v0), 0));
    }
    const cudaError_t e = dev_upload(*P, &P->d_dct_ctas, v);
    if (e != cudaSuccess) return cuda_fail(P, e, "DCT schedule upload");
    P->n_dct = (int)v.size();
  }
  P->seminaive = on;
  set_launch_count(*P);
  return SGL_OK;
}

static sgl_status ensure_stage(Plan& P, void** buf, size_t* have, size_t need) {
  if (*have >= need) return SGL_OK;
  if (*buf) {
    cudaFree(*buf);
    P.bytes -= *have;
  }
  *buf = nullptr;
  *have = 0;
  if (cudaMalloc(buf, need) != cudaSuccess) return fail(&P, SGL_ERR_ALLOC, "staging allocation failed");
  *have = need;
  P.bytes += need;
  return SGL_OK;
}

// ---------------------------------------------------------------------------
// host-buffer calls in chunks: the copies of one chunk of functions overlap
// the kernels of its neighbours
// ---------------------------------------------------------------------------
constexpr int kPipeMinFunctions = 16;

// Chunk sizes of n functions growing by about 1.6 from n/16: a host-to-device
// copy of a chunk (≈27 µs a function at B = 128 over a 200 GB/s link) then
// ends before the transform of the chunk before it (≈49 µs a function), so
// only the first, small chunk's copy is exposed, and most functions run in
// large, efficient chunks.  The last chunk takes the remainder.
static std::vector<int> grow_schedule(int n) {
  std::vector<int> out;
  int sum = 0;
  double x = std::max(1, n / 16);
  while (sum + (int)x < n) {
    out.push_back((int)x);
    sum += (int)x;
    x = std::ceil(x * 1.6);
  }
  out.push_back(n - sum);
  return out;
}

// The chunk sizes of a call: growing when the input is on the host (its
// first copy is the exposed one), shrinking when only the output is (the
// small chunk last, whose device-to-host copy is the exposed one).  Both
// directions use the same sizes, so one sub-plan per size serves every call.
static std::vector<int> pipe_schedule(int n, bool in_host) {
  std::vector<int> a = grow_schedule(n);
  if (!in_host) std::reverse(a.begin(), a.end());
  return a;
}

static sgl_status ensure_pipeline(Plan* P) {
  if (!P->subs.empty()) return SGL_OK;
  const int NB = P->nfn, B = P->fn_B[0];
  const std::vector<int> sizes = grow_schedule(NB);
  const size_t nchunks = sizes.size();
  auto make = [&](int n, Plan** out) -> sgl_status {
    Plan* S = new Plan();
    S->prec = P->prec;
    S->samples = P->samples;
    S->grid = P->grid;
    S->jp_fwd = P->jp_fwd;
    S->jp_inv = P->jp_inv;
    S->radi_narrow = P->radi_narrow;
    sgl_status st = build_plan(S, std::vector<int>(n, B), true);
    if (st == SGL_OK && P->seminaive) st = set_dlt(S, true);
    if (st != SGL_OK) {
      const std::string m = S->err;
      release(S);
      return fail(P, st, "sub-batch plan: " + m);
    }
    cudaFree(S->d_err);  // the parent's flag collects device-side errors
    S->d_err = P->d_err;
    S->owns_err = false;
    *out = S;
    return SGL_OK;
  };
  sgl_status st = SGL_OK;
  for (int n : sizes) {
    if (st != SGL_OK || P->subs.count(n)) continue;
    Plan* S = nullptr;
    st = make(n, &S);
    if (st == SGL_OK) P->subs[n] = S;
  }
  if (st == SGL_OK && (cudaStreamCreateWithFlags(&P->copy_stream, cudaStreamNonBlocking) != cudaSuccess ||
                       cudaStreamCreateWithFlags(&P->copy_back_stream, cudaStreamNonBlocking) != cudaSuccess))
    st = fail(P, SGL_ERR_CUDA, "copy stream creation failed");
  for (size_t k = 0; st == SGL_OK && k < 2 * nchunks + 2; ++k) {
    cudaEvent_t ev;
    if (cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) != cudaSuccess)
      st = fail(P, SGL_ERR_CUDA, "event creation failed");
    else
      P->pipe_ev.push_back(ev);
  }
  if (st != SGL_OK) {
    release_pipeline(P);
    return st;
  }
  return SGL_OK;
}

static sgl_status execute_pipelined(Plan* P, bool is_fwd, bool weights, const void* in, void* out, bool in_dev,
                                    bool out_dev, cudaStream_t s) {
  sgl_status st = ensure_pipeline(P);
  if (st != SGL_OK) return st;
  const size_t cb = complex_bytes(*P);
  const int B = P->fn_B[0];
  const int64_t spf = sample_count(B, n_radial(B, P->grid));  // samples per function
  const size_t in_per = (size_t)(is_fwd ? spf : coeff_count(B)) * cb;   // bytes per function
  const size_t out_per = (size_t)(is_fwd ? coeff_count(B) : spf) * cb;
  const char* din = (const char*)in;
  char* dout = (char*)out;
  if (!in_dev) {
    st = ensure_stage(*P, &P->d_stage_in, &P->stage_in_bytes, P->nfn * in_per);
    if (st != SGL_OK) return st;
    din = (const char*)P->d_stage_in;
  }
  if (!out_dev) {
    st = ensure_stage(*P, &P->d_stage_out, &P->stage_out_bytes, P->nfn * out_per);
    if (st != SGL_OK) return st;
    dout = (char*)P->d_stage_out;
  }
  const std::vector<int> sched = pipe_schedule(P->nfn, !in_dev);
  const int n = (int)sched.size();
  cudaEvent_t* ev = P->pipe_ev.data();  // [0] start, [1] end, then in/out per chunk
  cudaError_t e = cudaEventRecord(ev[0], s);
  // chunk k: its host-to-device copy on copy_stream (not held back by
  // anything but the start, so it runs while earlier chunks compute), its
  // transform on s once the copy is in, its device-to-host copy on
  // copy_back_stream once the transform is done
  if (e == cudaSuccess) e = cudaStreamWaitEvent(P->copy_stream, ev[0], 0);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(P->copy_back_stream, ev[0], 0);
  for (int k = 0, f0 = 0; k < n && e == cudaSuccess; f0 += sched[k], ++k) {
    const int nk = sched[k];
    Plan* S = P->subs.at(nk);
    const size_t io = (size_t)f0 * in_per, oo = (size_t)f0 * out_per;
    if (!in_dev) {
      e = cudaMemcpyAsync((void*)(din + io), (const char*)in + io, (size_t)nk * in_per, cudaMemcpyHostToDevice,
                          P->copy_stream);
      if (e == cudaSuccess) e = cudaEventRecord(ev[2 + 2 * k], P->copy_stream);
      if (e == cudaSuccess) e = cudaStreamWaitEvent(s, ev[2 + 2 * k], 0);
    }
    if (e == cudaSuccess)
      e = is_fwd ? run_forward(*S, din + io, dout + oo, s, weights) : run_inverse(*S, din + io, dout + oo, s, weights);
    if (e == cudaSuccess && !out_dev) {
      e = cudaEventRecord(ev[3 + 2 * k], s);
      if (e == cudaSuccess) e = cudaStreamWaitEvent(P->copy_back_stream, ev[3 + 2 * k], 0);
      if (e == cudaSuccess)
        e = cudaMemcpyAsync((char*)out + oo, dout + oo, (size_t)nk * out_per, cudaMemcpyDeviceToHost,
                            P->copy_back_stream);
    }
  }
  // the device-to-host copies follow every transform, which follow every
  // host-to-device copy: the end of copy_back_stream is the end of the call
  if (e == cudaSuccess) e = cudaEventRecord(ev[1], P->copy_back_stream);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(s, ev[1], 0);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_fail(P, e, "sub-batch execution");
  return SGL_OK;
}

// Runs the call through the plan's graph for (kind, in, out): replays it on
// s, or first captures the call's launches on the plan's own stream (nothing
// runs during the capture) and instantiates it.
static cudaError_t run_graph(Plan& P, bool is_fwd, bool weights, const void* in, void* out, cudaStream_t s) {
  const int kind = (is_fwd ? 2 : 0) | (weights ? 1 : 0);
  for (Plan::GraphEntry& g : P.graphs)
    if (g.kind == kind && g.in == in && g.out == out) {
      g.used = ++P.graph_clock;
      return cudaGraphLaunch(g.exec, s);
    }
  cudaError_t e = cudaSuccess;
  if (!P.graph_stream) e = cudaStreamCreateWithFlags(&P.graph_stream, cudaStreamNonBlocking);
  if (e != cudaSuccess) return e;
  e = cudaStreamBeginCapture(P.graph_stream, cudaStreamCaptureModeThreadLocal);
  if (e != cudaSuccess) return e;
  const cudaError_t er = is_fwd ? run_forward(P, in, out, P.graph_stream, weights)
                                : run_inverse(P, in, out, P.graph_stream, weights);
  cudaGraph_t graph = nullptr;
  e = cudaStreamEndCapture(P.graph_stream, &graph);  // always ends the capture
  if (er != cudaSuccess || e != cudaSuccess) {
    if (graph) cudaGraphDestroy(graph);
    return er != cudaSuccess ? er : e;
  }
  cudaGraphExec_t exec = nullptr;
  e = cudaGraphInstantiate(&exec, graph, 0);
  cudaGraphDestroy(graph);
  if (e != cudaSuccess) return e;
  if (P.graphs.size() >= Plan::kMaxGraphs) {
    size_t lru = 0;
    for (size_t k = 1; k < P.graphs.size(); ++k)
      if (P.graphs[k].used < P.graphs[lru].used) lru = k;
    cudaGraphExecDestroy(P.graphs[lru].exec);
    P.graphs.erase(P.graphs.begin() + (long)lru);
  }
  P.graphs.push_back({kind, in, out, exec, ++P.graph_clock});
  return cudaGraphLaunch(exec, s);
}

static bool stream_capturing(cudaStream_t s) {
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(s, &cs) != cudaSuccess) {
    cudaGetLastError();
    return true;  // unknown: do not start a capture of our own
  }
  return cs != cudaStreamCaptureStatusNone;
}

// Runs fwd (is_fwd) or inv with in/out that may be host or device memory.
static sgl_status execute(Plan* P, bool is_fwd, bool weights, const void* in, void* out, sgl_stream_t stream) {
  if (!P) return fail(nullptr, SGL_ERR_ARG, "null plan");
  if (!in || !out) return fail(P, SGL_ERR_ARG, "null data pointer");
  if (P->latched != SGL_OK) return (sgl_status)P->latched;
  cudaStream_t s = (cudaStream_t)stream;
  int cur = 0;
  cudaGetDevice(&cur);
  if (cur != P->device) cudaSetDevice(P->device);
  const size_t cb = complex_bytes(*P), sb = sample_bytes(*P);
  const size_t in_bytes = is_fwd ? P->n_samples * sb : P->n_coeffs * cb;
  const size_t out_bytes = is_fwd ? P->n_coeffs * cb : P->n_samples * sb;
  const size_t in_align = is_fwd ? sb : cb, out_align = is_fwd ? cb : sb;
  const bool in_dev = is_device_ptr(in), out_dev = is_device_ptr(out);
  if ((in_dev && (uintptr_t)in % in_align) || (out_dev && (uintptr_t)out % out_align)) {
    if (cur != P->device) cudaSetDevice(cur);
    return fail(P, SGL_ERR_ARG, "device data pointers must be aligned to their element size");
  }
  const void* din = in;
  void* dout = out;
  sgl_status st = SGL_OK;
  cudaError_t e = cudaSuccess;
  if (in_dev && out_dev && P->use_graphs && !P->profiling && !stream_capturing(s)) {
    e = run_graph(*P, is_fwd, weights, in, out, s);
    if (e != cudaSuccess) st = cuda_fail(P, e, "graph launch");
    goto done;
  }
  if ((!in_dev || !out_dev) && P->uniform && !P->real_pairs && !P->radial_halves && P->nfn >= kPipeMinFunctions) {
    st = execute_pipelined(P, is_fwd, weights, in, out, in_dev, out_dev, s);
    goto done;
  }
  if (!in_dev) {
    st = ensure_stage(*P, &P->d_stage_in, &P->stage_in_bytes, in_bytes);
    if (st != SGL_OK) goto done;
    e = cudaMemcpyAsync(P->d_stage_in, in, in_bytes, cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) { st = cuda_fail(P, e, "host-to-device copy"); goto done; }
    din = P->d_stage_in;
  }
  if (!out_dev) {
    st = ensure_stage(*P, &P->d_stage_out, &P->stage_out_bytes, out_bytes);
    if (st != SGL_OK) goto done;
    dout = P->d_stage_out;
  }
  e = is_fwd ? run_forward(*P, din, dout, s, weights) : run_inverse(*P, din, dout, s, weights);
  if (e != cudaSuccess) { st = cuda_fail(P, e, is_fwd ? "forward launch" : "inverse launch"); goto done; }
  if (!out_dev) {
    e = cudaMemcpyAsync(out, dout, out_bytes, cudaMemcpyDeviceToHost, s);
    if (e != cudaSuccess) { st = cuda_fail(P, e, "device-to-host copy"); goto done; }
  }
  if (!in_dev || !out_dev) {
    e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) { st = cuda_fail(P, e, "stream synchronize"); goto done; }
  }
done:
  if (cur != P->device) cudaSetDevice(cur);
  return st;
}

// ---------------------------------------------------------------------------
// autotuning (sgl_autotune)
// ---------------------------------------------------------------------------
static std::string tuning_text(const Plan& P, const char* source) {
  char buf[256];
  snprintf(buf, sizeof buf,
           "fft_fwd_jp=%d fft_inv_jp=%d rad_inv_narrow=%d simt=%d,%d,%d,%d rad_rows=%d fft_merge=%d queue=%d,%d,%d,%d "
           "inv_order=%d source=%s",
           fft_jp(P, P.maxB, false), fft_jp(P, P.maxB, true), P.radi_narrow, P.simt_policy[0], P.simt_policy[1],
           P.simt_policy[2], P.simt_policy[3], P.rad_rows, P.fft_merge, P.queue_slices[0], P.queue_slices[1],
           P.queue_slices[2], P.queue_slices[3], P.fft_inv_order, source);
  return buf;
}

// cache key: GPU model, precision, segments (bandlimit x functions)
static std::string tuning_key(const Plan& P) {
  cudaDeviceProp prop;
  std::string name = "unknown";
  if (cudaGetDeviceProperties(&prop, P.device) == cudaSuccess) name = prop.name;
  std::string k = name + " prec=" + std::to_string(P.prec) + " segs=";
  for (const SegDesc& sg : P.segs) k += std::to_string(sg.B) + "x" + std::to_string(sg.NB) + ",";
  return k;
}

// Best of three timed calls after one warm-up (milliseconds), or a negative
// value if a launch failed.
static double time_calls(Plan& P, bool fwd, void* samples, void* coeffs, cudaStream_t s) {
  cudaEvent_t a = nullptr, b = nullptr;
  if (cudaEventCreate(&a) != cudaSuccess || cudaEventCreate(&b) != cudaSuccess) return -1.0;
  double best = 1e30;
  for (int rep = 0; rep < 4 && best >= 0.0; ++rep) {
    cudaEventRecord(a, s);
    const cudaError_t e = fwd ? run_forward(P, samples, coeffs, s, true) : run_inverse(P, coeffs, samples, s, true);
    cudaEventRecord(b, s);
    if (e != cudaSuccess || cudaEventSynchronize(b) != cudaSuccess) {
      best = -1.0;
      break;
    }
    float ms = 0.f;
    cudaEventElapsedTime(&ms, a, b);
    if (rep > 0 && ms < best) best = ms;
  }
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  return best;
}

static sgl_status autotune(Plan* P, void* samples, void* coeffs, const char* cache_path, cudaStream_t s) {
  cudaError_t e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_fail(P, e, "stream synchronize");
  const std::string key = tuning_key(*P);
  bool cached = false;
  if (cache_path) {
    FILE* f = fopen(cache_path, "r");
    if (f) {
      char line[1024];
      while (fgets(line, sizeof line, f)) {
        const std::string ln(line);
        if (ln.compare(0, key.size() + 3, key + " | ") != 0) continue;
        int jf = 0, ji = 0, rn = 0, sp[4] = {0, 0, 0, 0}, rr = 64, fm = 1, qs[4] = {2, 2, 2, 2}, io = 0;
        const int got = sscanf(ln.c_str() + key.size() + 3,
                               "fft_fwd_jp=%d fft_inv_jp=%d rad_inv_narrow=%d simt=%d,%d,%d,%d rad_rows=%d fft_merge=%d "
                               "queue=%d,%d,%d,%d inv_order=%d",
                               &jf, &ji, &rn, &sp[0], &sp[1], &sp[2], &sp[3], &rr, &fm, &qs[0], &qs[1], &qs[2], &qs[3],
                               &io);
        // lines of fewer fields (older formats) keep the defaults of the rest
        bool valid = (got == 3 || got >= 8) && jf >= 1 && jf <= 16 && ji >= 1 && ji <= 16 && rn >= 1;
        for (int k = 0; k < 4; ++k) valid = valid && sp[k] >= 0 && sp[k] <= 2;
        for (int k = 0; k < 4; ++k) valid = valid && (qs[k] == 1 || qs[k] == 2 || qs[k] == 4 || qs[k] == 8);
        valid = valid && (rr == 32 || rr == 48 || rr == 64) && (fm == 0 || fm == 1) && (io == 0 || io == 1);
        if (valid) {
          P->jp_fwd = jf;
          P->jp_inv = ji;
          P->radi_narrow = rn;
          for (int k = 0; k < 4; ++k) P->simt_policy[k] = sp[k];
          P->rad_rows = rr;
          P->fft_merge = fm;
          for (int k = 0; k < 4; ++k) P->queue_slices[k] = qs[k];
          P->fft_inv_order = io;
          cached = true;
        }
      }
      fclose(f);
    }
  }
  if (!cached) {
    cudaMemsetAsync(samples, 0, (size_t)P->n_samples * sample_bytes(*P), s);
    cudaMemsetAsync(coeffs, 0, (size_t)P->n_coeffs * complex_bytes(*P), s);
    std::vector<int> jps = {4, 8};
    if (P->prec != SGL_FP64) jps.push_back(16);
    for (int dir = 0; dir < 2; ++dir) {
      int& knob = dir == 0 ? P->jp_fwd : P->jp_inv;
      int best = 0;
      double tbest = 1e30;
      for (int jp : jps) {
        knob = jp;
        e = build_fft_lists(*P);
        if (e != cudaSuccess) return cuda_fail(P, e, "autotune schedule upload");
        const double t = time_calls(*P, dir == 0, samples, coeffs, s);
        if (t < 0.0) return cuda_fail(P, cudaGetLastError(), "autotune launch");
        if (t < tbest) {
          tbest = t;
          best = jp;
        }
      }
      knob = best;
    }
    e = build_fft_lists(*P);
    if (e != cudaSuccess) return cuda_fail(P, e, "autotune schedule upload");
    if (tc_precision(P->prec)) {  // CTA order of the inverse phi-FFT (layout 1)
      int best = 0;
      double tbest = 1e30;
      for (int io : {0, 1}) {
        P->fft_inv_order = io;
        e = build_fft_lists(*P);
        if (e != cudaSuccess) return cuda_fail(P, e, "autotune schedule upload");
        const double t = time_calls(*P, false, samples, coeffs, s);
        if (t < 0.0) return cuda_fail(P, cudaGetLastError(), "autotune launch");
        if (t < tbest) {
          tbest = t;
          best = io;
        }
      }
      P->fft_inv_order = best;
      e = build_fft_lists(*P);
      if (e != cudaSuccess) return cuda_fail(P, e, "autotune schedule upload");
    }
    // plans of several register-FFT sizes: one multi-size launch per
    // direction, or one launch per size (timed over both directions)
    const int merge0 = P->fft_merge;
    P->fft_merge = 0;
    const bool several = fft_launches(*P, false) > 1 || fft_launches(*P, true) > 1;
    P->fft_merge = merge0;
    if (several) {
      int best = P->fft_merge;
      double tbest = 1e30;
      for (int fm : {1, 0}) {
        P->fft_merge = fm;
        const double t = time_calls(*P, true, samples, coeffs, s) + time_calls(*P, false, samples, coeffs, s);
        if (t < 0.0) return cuda_fail(P, cudaGetLastError(), "autotune launch");
        if (t < tbest) {
          tbest = t;
          best = fm;
        }
      }
      P->fft_merge = best;
    }
    if (tc_precision(P->prec)) {
      int best = 65;
      double tbest = 1e30;
      for (int rn : {65, 1}) {
        P->radi_narrow = rn;
        e = tc_radi_retile(*P);
        if (e != cudaSuccess) return cuda_fail(P, e, "autotune schedule upload");
        const double t = time_calls(*P, false, samples, coeffs, s);
        if (t < 0.0) return cuda_fail(P, cudaGetLastError(), "autotune launch");
        if (t < tbest) {
          tbest = t;
          best = rn;
        }
      }
      P->radi_narrow = best;
      // tile width of the forward radial stage: the table group height
      int best_rr = 64;
      tbest = 1e30;
      for (int rr : {64, 48, 32}) {
        P->rad_rows = rr;
        tc_release(*P);
        e = tc_prepare(*P);
        if (e != cudaSuccess) return cuda_fail(P, e, "autotune tensor-core preparation");
        const double t = time_calls(*P, true, samples, coeffs, s);
        if (t < 0.0) return cuda_fail(P, cudaGetLastError(), "autotune launch");
        if (t < tbest) {
          tbest = t;
          best_rr = rr;
        }
      }
      P->rad_rows = best_rr;
      // work-queue granularity of each tensor-core stage (slices per CTA),
      // one stage at a time: the forward stages timed on forward calls, the
      // inverse stages on inverse calls
      for (int st = 0; st < 4; ++st) {
        int best_q = P->queue_slices[st];
        tbest = 1e30;
        for (int q : {2, 1, 4, 8}) {
          P->queue_slices[st] = q;
          tc_release(*P);
          e = tc_prepare(*P);
          if (e != cudaSuccess) return cuda_fail(P, e, "autotune tensor-core preparation");
          const double t = time_calls(*P, st < 2, samples, coeffs, s);
          if (t < 0.0) return cuda_fail(P, cudaGetLastError(), "autotune launch");
          if (t < tbest) {
            tbest = t;
            best_q = q;
          }
        }
        P->queue_slices[st] = best_q;
      }
    } else {
      // SIMT tile family of each GEMM stage, one stage at a time (forward
      // stages timed on forward calls, inverse stages on inverse calls)
      for (int st = 0; st < 4; ++st) {
        int best = 0;
        double tbest = 1e30;
        for (int pol = 0; pol < 3; ++pol) {
          P->simt_policy[st] = pol;
          e = build_simt_lists(*P);
          if (e != cudaSuccess) return cuda_fail(P, e, "autotune schedule upload");
          const double t = time_calls(*P, st < 2, samples, coeffs, s);
          if (t < 0.0) return cuda_fail(P, cudaGetLastError(), "autotune launch");
          if (t < tbest) {
            tbest = t;
            best = pol;
          }
        }
        P->simt_policy[st] = best;
      }
    }
  }
  e = build_fft_lists(*P);
  if (e == cudaSuccess) e = build_simt_lists(*P);
  if (e == cudaSuccess && tc_precision(P->prec)) {
    tc_release(*P);
    e = tc_prepare(*P);  // for the chosen radial tile width (and inverse radial policy)
  }
  if (e != cudaSuccess) return cuda_fail(P, e, "autotune schedule upload");
  set_launch_count(*P);
  P->tuning = tuning_text(*P, cached ? "cache" : "timed");
  release_pipeline(P);  // sub-batch plans are rebuilt with the new configuration on next use
  drop_graphs(*P);      // and graphs are captured again
  if (!cached && cache_path) {
    FILE* f = fopen(cache_path, "a");
    if (!f) return fail(P, SGL_ERR_ARG, std::string("cannot append to tuning cache ") + cache_path);
    fprintf(f,
            "%s | fft_fwd_jp=%d fft_inv_jp=%d rad_inv_narrow=%d simt=%d,%d,%d,%d rad_rows=%d fft_merge=%d "
            "queue=%d,%d,%d,%d inv_order=%d\n",
            key.c_str(), P->jp_fwd, P->jp_inv, P->radi_narrow, P->simt_policy[0], P->simt_policy[1],
            P->simt_policy[2], P->simt_policy[3], P->rad_rows, P->fft_merge, P->queue_slices[0], P->queue_slices[1],
            P->queue_slices[2], P->queue_slices[3], P->fft_inv_order);
    fclose(f);
  }
  return SGL_OK;
}

extern "C" {

sgl_status sgl_plan(sgl_plan_t* out, int B, int batch, int prec, int samples) {
  return sgl_plan_grid(out, B, batch, prec, samples, SGL_GRID_LAGUERRE);
}

sgl_status sgl_plan_grid(sgl_plan_t* out, int B, int batch, int prec, int samples, int grid) {
  if (!out) return fail(nullptr, SGL_ERR_ARG, "null output pointer");
  *out = nullptr;
  if (B < 1) return fail(nullptr, SGL_ERR_ARG, "bandlimit must be >= 1");
  if (batch < 1) return fail(nullptr, SGL_ERR_ARG, "batch must be >= 1");
  if (prec < SGL_FP64 || prec > SGL_FP16X3) return fail(nullptr, SGL_ERR_ARG, "unknown precision");
  if (samples != SGL_SAMPLES_WEIGHTED && samples != SGL_SAMPLES_PHYSICAL && samples != SGL_SAMPLES_REAL)
    return fail(nullptr, SGL_ERR_ARG, "unknown sample convention");
  if (samples == SGL_SAMPLES_PHYSICAL && prec != SGL_FP64)
    return fail(nullptr, SGL_ERR_ARG, "physical samples need an FP64 plan");
  if (grid != SGL_GRID_LAGUERRE && grid != SGL_GRID_HALF_RANGE_HERMITE)
    return fail(nullptr, SGL_ERR_ARG, "unknown radial grid");
  if (!bandlimit_supported(B)) return fail(nullptr, SGL_ERR_UNSUPPORTED, "unsupported bandlimit");
  if (tc_precision(prec) && B % 4 != 0)
    return fail(nullptr, SGL_ERR_UNSUPPORTED, "tensor-core plans need a bandlimit divisible by 4");
  Plan* P = new Plan();
  P->prec = prec;
  P->samples = samples;
  P->grid = grid;
  const bool real = samples == SGL_SAMPLES_REAL;
  if (real) {  // the real functions in pairs, one complex function per pair
    P->real_pairs = true;
    P->nreal = batch;
  }
  // tensor-core stages on the paper's grid: the two halves of each
  // function's 2B radii as two functions of B radii
  const bool halves = grid == SGL_GRID_HALF_RANGE_HERMITE && tc_precision(prec);
  const int ncomplex = real ? (batch + 1) / 2 : batch;  // complex functions of 2B radii
  if (halves) {
    P->radial_halves = true;
    P->nuser = ncomplex;
  }
  std::vector<int> Bs(halves ? 2 * ncomplex : ncomplex, B);
  sgl_status st = build_plan(P, Bs, true);
  // coefficient workspaces: d_ccoef the plan's nfn functions (halves or
  // pairs), d_pcoef the pairs when the plan has both
  const int64_t fbytes = coeff_count(B) * (int64_t)complex_bytes(*P);
  if (st == SGL_OK && (halves || real)) {
    P->n_coeffs = (int64_t)batch * coeff_count(B);
    if (cudaMalloc(&P->d_ccoef, P->nfn * fbytes) != cudaSuccess)
      st = fail(P, SGL_ERR_ALLOC, "workspace allocation failed");
    else
      P->bytes += P->nfn * fbytes;
  }
  if (st == SGL_OK && halves && real) {
    if (cudaMalloc(&P->d_pcoef, ncomplex * fbytes) != cudaSuccess)
      st = fail(P, SGL_ERR_ALLOC, "workspace allocation failed");
    else
      P->bytes += ncomplex * fbytes;
  }
  if (st == SGL_OK && real) P->n_samples = (int64_t)batch * sample_count(B, n_radial(B, grid));  // reals
  if (st != SGL_OK) {
    g_create_error = P->err;
    release(P);
    return st;
  }
  *out = (sgl_plan_t)P;
  return SGL_OK;
}

sgl_status sgl_plan_many(sgl_plan_t* out, const int* B_per_fn, int nfn, int prec) {
  if (!out) return fail(nullptr, SGL_ERR_ARG, "null output pointer");
  *out = nullptr;
  if (!B_per_fn || nfn < 1) return fail(nullptr, SGL_ERR_ARG, "need at least one function");
  if (prec < SGL_FP64 || prec > SGL_FP16X3) return fail(nullptr, SGL_ERR_ARG, "unknown precision");
  std::vector<int> Bs(B_per_fn, B_per_fn + nfn);
  for (int B : Bs) {
    if (B < 1) return fail(nullptr, SGL_ERR_ARG, "bandlimit must be >= 1");
    if (!bandlimit_supported(B)) return fail(nullptr, SGL_ERR_UNSUPPORTED, "unsupported bandlimit");
    if (tc_precision(prec) && B % 4 != 0)
      return fail(nullptr, SGL_ERR_UNSUPPORTED, "tensor-core plans need bandlimits divisible by 4");
  }
  Plan* P = new Plan();
  P->prec = prec;
  P->samples = SGL_SAMPLES_WEIGHTED;
  bool uni = true;
  for (int B : Bs) uni = uni && (B == Bs[0]);
  sgl_status st = build_plan(P, Bs, uni);
  if (st != SGL_OK) {
    g_create_error = P->err;
    release(P);
    return st;
  }
  *out = (sgl_plan_t)P;
  return SGL_OK;
}

sgl_status sgl_forward(sgl_plan_t plan, const void* samples, void* coeffs, sgl_stream_t stream) {
  return execute((Plan*)plan, true, true, samples, coeffs, stream);
}

sgl_status sgl_inverse(sgl_plan_t plan, const void* coeffs, void* samples, sgl_stream_t stream) {
  return execute((Plan*)plan, false, false, coeffs, samples, stream);
}

sgl_status sgl_adjoint(sgl_plan_t plan, int of_inverse, const void* in, void* out, sgl_stream_t stream) {
  // adjoint of the forward map: weighted inverse pipeline; adjoint of the
  // inverse map: forward pipeline without weights
  if (of_inverse) return execute((Plan*)plan, true, false, in, out, stream);
  return execute((Plan*)plan, false, true, in, out, stream);
}

sgl_status sgl_grid(sgl_plan_t plan, int fn, double* r, double* theta, double* phi, double* w_r,
                    double* w_theta) {
  Plan* P = (Plan*)plan;
  if (!P) return fail(nullptr, SGL_ERR_ARG, "null plan");
  if (fn < 0 || fn >= user_fns(*P)) return fail(P, SGL_ERR_ARG, "function index out of range");
  const int B = P->fn_B[P->real_pairs || P->radial_halves ? 0 : fn];
  size_t seg = 0;
  while (P->segs[seg].B != B) ++seg;
  HostTables full;  // radial halves: the whole rule, not a segment's half
  if (P->radial_halves) {
    std::string msg;
    if (!cached_tables(B, P->grid, full, msg)) return fail(P, SGL_ERR_ARG, "table generation: " + msg);
  }
  const HostTables& H = P->radial_halves ? full : P->tables[seg];
  if (r) memcpy(r, H.r.data(), H.R * sizeof(double));
  if (theta) memcpy(theta, H.theta.data(), 2 * B * sizeof(double));
  if (phi) memcpy(phi, H.phi.data(), 2 * B * sizeof(double));
  if (w_r) memcpy(w_r, H.what.data(), H.R * sizeof(double));
  if (w_theta) memcpy(w_theta, H.beta.data(), 2 * B * sizeof(double));
  return SGL_OK;
}

int64_t sgl_sample_count(sgl_plan_t plan) { return plan ? ((Plan*)plan)->n_samples : -1; }
int64_t sgl_coeff_count(sgl_plan_t plan) { return plan ? ((Plan*)plan)->n_coeffs : -1; }

int64_t sgl_sample_offset(sgl_plan_t plan, int fn) {
  Plan* P = (Plan*)plan;
  if (!P || fn < 0 || fn >= user_fns(*P)) return -1;
  if (P->real_pairs || P->radial_halves) return (int64_t)fn * sample_count(P->fn_B[0], n_radial(P->fn_B[0], P->grid));
  return P->fn_samp_off[fn];
}

int64_t sgl_coeff_offset(sgl_plan_t plan, int fn) {
  Plan* P = (Plan*)plan;
  if (!P || fn < 0 || fn >= user_fns(*P)) return -1;
  if (P->real_pairs || P->radial_halves) return (int64_t)fn * coeff_count(P->fn_B[0]);
  return P->fn_coef_off[fn];
}

int sgl_num_functions(sgl_plan_t plan) { return plan ? user_fns(*(Plan*)plan) : -1; }

int sgl_bandlimit(sgl_plan_t plan, int fn) {
  Plan* P = (Plan*)plan;
  if (!P || fn < 0 || fn >= user_fns(*P)) return -1;
  return P->fn_B[P->real_pairs || P->radial_halves ? 0 : fn];
}

int sgl_radii(sgl_plan_t plan, int fn) {
  Plan* P = (Plan*)plan;
  if (!P || fn < 0 || fn >= user_fns(*P)) return -1;
  const int B = P->fn_B[P->real_pairs || P->radial_halves ? 0 : fn];
  return n_radial(B, P->grid);
}

int64_t sgl_workspace_bytes(sgl_plan_t plan) {
  if (!plan) return -1;
  const Plan* P = (const Plan*)plan;
  int64_t b = P->bytes;
  for (const auto& kv : P->subs) b += kv.second->bytes;
  return b;
}

int sgl_launches_per_call(sgl_plan_t plan) { return plan ? ((Plan*)plan)->launches_per_call : -1; }

sgl_status sgl_check(sgl_plan_t plan, sgl_stream_t stream) {
  Plan* P = (Plan*)plan;
  if (!P) return fail(nullptr, SGL_ERR_ARG, "null plan");
  int flag = 0;
  cudaError_t e = cudaMemcpyAsync(&flag, P->d_err, sizeof(int), cudaMemcpyDeviceToHost, (cudaStream_t)stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize((cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(P, e, "error flag read");
  if (flag != 0) {
    P->latched = SGL_ERR_TIMEOUT;
    P->err = "a bounded device-side wait gave up";
  }
  return (sgl_status)P->latched;
}

sgl_status sgl_set_graphs(sgl_plan_t plan, int enable) {
  Plan* P = (Plan*)plan;
  if (!P) return fail(nullptr, SGL_ERR_ARG, "null plan");
  int cur = 0;
  cudaGetDevice(&cur);
  if (cur != P->device) cudaSetDevice(P->device);
  P->use_graphs = enable != 0;
  if (!P->use_graphs) drop_graphs(*P);
  if (cur != P->device) cudaSetDevice(cur);
  return SGL_OK;
}

int sgl_graph_count(sgl_plan_t plan) { return plan ? (int)((Plan*)plan)->graphs.size() : -1; }

sgl_status sgl_set_profiling(sgl_plan_t plan, int enable) {
  Plan* P = (Plan*)plan;
  if (!P) return fail(nullptr, SGL_ERR_ARG, "null plan");
  if (!enable) clear_profile(*P);
  P->profiling = enable != 0;
  return SGL_OK;
}

sgl_status sgl_stage_times(sgl_plan_t plan, double* ms, int64_t* launches) {
  Plan* P = (Plan*)plan;
  if (!P) return fail(nullptr, SGL_ERR_ARG, "null plan");
  for (int st = 0; st < SGL_NUM_STAGES; ++st) {
    double sum = 0.0;
    for (auto& pr : P->prof_ev[st]) {
      cudaError_t e = cudaEventSynchronize(pr.second);
      if (e != cudaSuccess) return cuda_fail(P, e, "profiling event");
      float t = 0.f;
      cudaEventElapsedTime(&t, pr.first, pr.second);
      sum += t;
    }
    if (ms) ms[st] = sum;
    if (launches) launches[st] = (int64_t)P->prof_ev[st].size();
  }
  return SGL_OK;
}

const char* sgl_stage_name(int stage) {
  static const char* names[SGL_NUM_STAGES] = {"fft_forward", "legendre_forward", "radial_forward",
                                              "radial_inverse", "legendre_inverse", "fft_inverse"};
  if (stage < 0 || stage >= SGL_NUM_STAGES) return "";
  return names[stage];
}

sgl_status sgl_set_dlt(sgl_plan_t plan, int seminaive) {
  Plan* P = (Plan*)plan;
  if (!P) return fail(nullptr, SGL_ERR_ARG, "null plan");
  if (tc_precision(P->prec))
    return fail(P, SGL_ERR_UNSUPPORTED, "the seminaive Legendre transform is built for FP64 and FP32 plans");
  int cur = 0;
  cudaGetDevice(&cur);
  if (cur != P->device) cudaSetDevice(P->device);
  release_pipeline(P);  // sub-batch plans are rebuilt with the setting on next use
  drop_graphs(*P);
  const sgl_status st = set_dlt(P, seminaive != 0);
  if (cur != P->device) cudaSetDevice(cur);
  return st;
}

sgl_status sgl_autotune(sgl_plan_t plan, void* samples, void* coeffs, const char* cache_path,
                        sgl_stream_t stream) {
  Plan* P = (Plan*)plan;
  if (!P) return fail(nullptr, SGL_ERR_ARG, "null plan");
  if (!samples || !coeffs || !is_device_ptr(samples) || !is_device_ptr(coeffs))
    return fail(P, SGL_ERR_ARG, "sgl_autotune needs device buffers for samples and coefficients");
  if ((uintptr_t)samples % sample_bytes(*P) || (uintptr_t)coeffs % complex_bytes(*P))
    return fail(P, SGL_ERR_ARG, "device data pointers must be aligned to their element size");
  if (P->latched != SGL_OK) return (sgl_status)P->latched;
  int cur = 0;
  cudaGetDevice(&cur);
  if (cur != P->device) cudaSetDevice(P->device);
  const sgl_status st = autotune(P, samples, coeffs, cache_path, (cudaStream_t)stream);
  if (cur != P->device) cudaSetDevice(cur);
  return st;
}

const char* sgl_tuning(sgl_plan_t plan) {
  Plan* P = (Plan*)plan;
  if (!P) return "";
  if (P->tuning.empty()) P->tuning = tuning_text(*P, "default");
  return P->tuning.c_str();
}

const char* sgl_last_error(sgl_plan_t plan) {
  if (!plan) return g_create_error.c_str();
  return ((Plan*)plan)->err.c_str();
}

void sgl_destroy(sgl_plan_t plan) { release((Plan*)plan); }

const char* sgl_version(void) { return "sgl-gb300 0.1"; }

}  // extern "C"
