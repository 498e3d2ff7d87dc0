// sgl_forward_noalloc: the FP64 forward transform without any device
// allocation, for callers that cannot call cudaMalloc.
//
// The three forward kernels of the plan path run unchanged; what differs is
// where their memory comes from.  Their scratch (the E/O spectra and the
// per-degree spectra between the stages) lives in one file-scope static
// __device__ array of fixed size, and their read-only data (tables, segment
// descriptor, offsets, launch schedules) in a second one.  Host code never
// dereferences either array: it asks the runtime for their device addresses
// with cudaGetSymbolAddress, once per device, and passes those addresses on.
//
// The library is built without relocatable device code, so this file is its
// own CUDA module.  Under CUDA's lazy module loading (the default) a module
// is loaded on a device when host code first needs it there: the first
// cudaGetSymbolAddress below loads this one and reserves both arrays (24 MiB)
// on that device, and the first launch of each forward kernel loads that
// kernel's module.  The first call on a device therefore belongs at start-up,
// before the caller's allocator takes the device's memory (or the process
// runs with CUDA_MODULE_LOADING=EAGER, which loads every module up front).
#include <cuda_runtime.h>
#include <string.h>

#include <mutex>
#include <string>
#include <vector>

#include "sgl_internal.h"

namespace sgl {
void set_global_error(const std::string& msg);
int fft_pairs_per_cta(int prec, int B);
void gemm_tile_dims(int& tm, int& tn, int& tk);
size_t fft_smem_for(int prec, int n1, int n2, int B);
}  // namespace sgl

using namespace sgl;

namespace {

constexpr int kMaxB = 32;                                   // largest bandlimit accepted
constexpr size_t kScratchDoubles = size_t(2) << 20;         // 16 MiB of scratch
constexpr size_t kConstBytes = size_t(8) << 20;             // 8 MiB of tables and schedules
constexpr int kMaxDevices = 64;

// Scratch of the forward pipeline: workspace 1 (E/O spectra) followed by
// workspace 2 (per-degree spectra).  Every call overwrites what it reads
// before reading it, so nothing needs clearing between calls.
static __device__ __align__(256) double g_noalloc_scratch[kScratchDoubles];
// Tables, descriptors and schedules of the current (B, batch) on this device.
static __device__ __align__(256) unsigned char g_noalloc_const[kConstBytes];

struct DeviceState {
  bool ready = false;
  double* scratch = nullptr;         // device address of g_noalloc_scratch
  unsigned char* cst = nullptr;      // device address of g_noalloc_const
  int B = 0, batch = 0;              // configuration whose data sits in the const region
  Plan plan;                         // host description; device pointers into the arrays
  std::vector<unsigned char> image;  // host copy of the const region for (B, batch)
};

DeviceState g_dev[kMaxDevices];
std::mutex g_mu;

// failures are reported through sgl_last_error(NULL)
sgl_status fail(sgl_status st, const std::string& msg) {
  set_global_error(msg);
  return st;
}

size_t align256(size_t x) { return (x + 255) / 256 * 256; }

template <typename T>
size_t put(std::vector<unsigned char>& img, const std::vector<T>& v) {
  size_t off = align256(img.size());
  img.resize(off + v.size() * sizeof(T));
  if (!v.empty()) memcpy(img.data() + off, v.data(), v.size() * sizeof(T));
  return off;
}

// Describe a single-segment FP64 plan of `batch` functions of bandlimit B
// whose device pointers point into the two static arrays.
sgl_status describe(DeviceState& D, int B, int batch) {
  Plan& P = D.plan;
  P = Plan();
  P.prec = SGL_FP64;
  P.samples = SGL_SAMPLES_WEIGHTED;
  P.nfn = batch;
  P.maxB = B;
  P.n_samples = sample_count(B, B) * batch;
  P.n_coeffs = coeff_count(B) * batch;
  SegDesc sg;
  memset(&sg, 0, sizeof(sg));
  sg.B = B;
  sg.R = B;  // the Gauss-Laguerre grid
  sg.NB = batch;
  sg.n1 = fft_n1(2 * B);
  sg.n2 = 2 * B / sg.n1;
  sg.fn0 = 0;
  // offsets of the (only) segment within workspaces 1 and 2; the workspaces
  // themselves sit back to back in the scratch (d_w1, d_w2 below)
  sg.w1_off = 0;
  sg.w2_off = 0;
  int64_t tab = 0;
  sg.tab_misc = tab;
  tab += misc_size(B, B);
  sg.tab_leg_f = tab;
  tab += leg_table_size(B);
  sg.tab_leg_i = tab;
  tab += leg_table_size(B);
  sg.tab_rad_f = tab;
  tab += rad_table_size(B, B);
  sg.tab_rad_i = tab;
  tab += rad_table_size(B, B);
  sg.tab_leg_s = tab;  // packed with the others, unused here
  tab += leg_table_size(B);
  sg.tab_dct = tab;
  tab += 5 * B;
  sg.si_rows = 0;
  P.tab_elems = tab;
  HostTables H;
  std::string msg;
  if (!build_tables(B, SGL_GRID_LAGUERRE, H, msg)) return fail(SGL_ERR_ARG, "table generation: " + msg);
  P.tables.push_back(std::move(H));
  P.segs.push_back(sg);

  std::vector<int64_t> fn_samp(batch), fn_coef(batch), si_rows;
  for (int b = 0; b < batch; ++b) {
    fn_samp[b] = sample_count(B, B) * b;
    fn_coef[b] = coeff_count(B) * b;
  }
  for (int mi = 0; mi < 2 * B - 1; ++mi)
    for (int p = 0; p < 2; ++p) si_rows.push_back(si_rows_before(B, mi, p));
  int TM, TN, TK;
  gemm_tile_dims(TM, TN, TK);
  std::vector<int4> lf, rf, ff;
  for (int g = 0; g < 2 * (2 * B - 1); ++g) {
    const int m = (g >> 1) - (B - 1);
    const int N = n_par(B, m < 0 ? -m : m, g & 1);
    for (int r0 = 0; r0 < batch * 2 * B; r0 += TM)
      for (int c0 = 0; c0 < N; c0 += TN) lf.push_back(make_int4(0, g, r0, c0));
  }
  for (int l = 0; l < B; ++l)
    for (int r0 = 0; r0 < batch * (2 * l + 1) * 2; r0 += TM)
      for (int c0 = 0; c0 < B - l; c0 += TN) rf.push_back(make_int4(0, l, r0, c0));
  const int JP = fft_pairs_per_cta(SGL_FP64, B);
  for (int sh = 0; sh < batch * B; ++sh)
    for (int j0 = 0; j0 < B; j0 += JP) ff.push_back(make_int4(0, sh, j0, 0));

  std::vector<double> t;
  pack_tables<double>(P, t);
  std::vector<unsigned char>& img = D.image;
  img.clear();
  const size_t o_tab = put(img, t);
  const size_t o_seg = put(img, P.segs);
  const size_t o_samp = put(img, fn_samp);
  const size_t o_coef = put(img, fn_coef);
  const size_t o_si = put(img, si_rows);
  const size_t o_lf = put(img, lf);
  const size_t o_rf = put(img, rf);
  const size_t o_ff = put(img, ff);
  if (img.size() > kConstBytes)
    return fail(SGL_ERR_UNSUPPORTED, "tables and schedules exceed the static region of " +
                                         std::to_string(kConstBytes) + " bytes");
  unsigned char* c = D.cst;
  P.d_tab = c + o_tab;
  P.d_segs = (SegDesc*)(c + o_seg);
  P.d_fn_samp = (int64_t*)(c + o_samp);
  P.d_fn_coef = (int64_t*)(c + o_coef);
  P.d_si_rows = (int64_t*)(c + o_si);
  P.leg_fwd.d_tiles[0] = (int4*)(c + o_lf);  // 64 x 64 tiles only
  P.leg_fwd.ntiles[0] = (int)lf.size();
  P.rad_fwd.d_tiles[0] = (int4*)(c + o_rf);
  P.rad_fwd.ntiles[0] = (int)rf.size();
  P.d_fft_fwd = (int4*)(c + o_ff);
  P.n_fft_fwd = (int)ff.size();
  P.d_w1 = D.scratch;
  P.d_w2 = D.scratch + w1_size(B, batch, B);
  return SGL_OK;
}

// True for managed memory and for device memory of device `dev` (the kernels
// run there, with that device's static arrays; a buffer of another GPU would
// be reached across devices, or not at all without peer access).
bool device_pointer(const void* p, int dev) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  if (a.type == cudaMemoryTypeManaged) return true;
  return a.type == cudaMemoryTypeDevice && a.device == dev;
}

}  // namespace

extern "C" sgl_status sgl_forward_noalloc(int B, int batch, const void* samples, void* coeffs,
                                          sgl_stream_t stream) {
  std::lock_guard<std::mutex> lock(g_mu);
  if (B < 1 || B > kMaxB || !bandlimit_supported(B))
    return fail(SGL_ERR_UNSUPPORTED, "sgl_forward_noalloc accepts bandlimits 1.." + std::to_string(kMaxB));
  if (batch < 1) return fail(SGL_ERR_ARG, "batch must be >= 1");
  if (!samples || !coeffs) return fail(SGL_ERR_ARG, "null data pointer");
  const size_t need = (size_t)(w1_size(B, batch, B) + w2_size(B, batch, B));
  if (need > kScratchDoubles)
    return fail(SGL_ERR_UNSUPPORTED, "B=" + std::to_string(B) + " batch=" + std::to_string(batch) + " needs " +
                                         std::to_string(need) + " scratch doubles; the static scratch holds " +
                                         std::to_string(kScratchDoubles));
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return fail(SGL_ERR_CUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
  if (dev < 0 || dev >= kMaxDevices) return fail(SGL_ERR_UNSUPPORTED, "device index too large");
  if (!device_pointer(samples, dev) || !device_pointer(coeffs, dev))
    return fail(SGL_ERR_ARG, "sgl_forward_noalloc takes device pointers of the current device only");
  if ((uintptr_t)samples % 16 || (uintptr_t)coeffs % 16)
    return fail(SGL_ERR_ARG, "data pointers must be aligned to the complex element size (16 bytes)");
  DeviceState& D = g_dev[dev];
  if (!D.ready) {
    // once per device, with that device current
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return fail(SGL_ERR_CUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
    D.scratch = (double*)p;
    e = cudaGetSymbolAddress(&p, g_noalloc_const);
    if (e != cudaSuccess) return fail(SGL_ERR_CUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
    D.cst = (unsigned char*)p;
    D.ready = true;
  }
  cudaStream_t s = (cudaStream_t)stream;
  if (D.B != B || D.batch != batch) {
    D.B = D.batch = 0;
    sgl_status st = describe(D, B, batch);
    if (st != SGL_OK) return st;
    e = cudaMemcpyAsync(D.cst, D.image.data(), D.image.size(), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return fail(SGL_ERR_CUDA, std::string("table upload: ") + cudaGetErrorString(e));
    D.B = B;
    D.batch = batch;
  }
  e = run_forward(D.plan, samples, coeffs, s, true);
  if (e != cudaSuccess) return fail(SGL_ERR_CUDA, std::string("forward launch: ") + cudaGetErrorString(e));
  return SGL_OK;
}
