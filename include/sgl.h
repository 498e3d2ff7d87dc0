/*
 * sgl.h - C ABI of the GB300 spherical Gauss-Laguerre (SGL) transform library.
 *
 * The library computes, for bandlimit B, the forward SGL transform of samples
 * on the SGL grid (the quadrature of the SGL sampling theorem, Thm 3.4), its
 * inverse (reconstruction of the samples from the coefficients, Algorithm 2 /
 * Algorithm 4) and the adjoints of both (matrix form, Sect. 3.4), batched over
 * many functions.  Every step runs in the library's own CUDA kernels for
 * sm_103a; nothing falls back to the CPU.
 *
 * Grid (the sampling theorem with B radial nodes):
 *   r_i      i < B    r_i^2 = t_i, the zeros of the generalized Laguerre
 *                     polynomial L_B^(1/2) (Gauss-Laguerre rule for
 *                     t^(1/2) e^(-t), Thm 3.3 restated in t = r^2);
 *   theta_j  j < 2B   (2j+1) pi / (4B)            (Thm 3.1);
 *   phi_k    k < 2B   k pi / B                    (Thm 3.1).
 * Weights: what_i = (w_i / 2) exp(t_i) (the exp(r^2)-modified radial weight of
 * Sect. 3.2, in the symmetric form), beta_j = (pi/B) b_j with b_j of Thm 3.1.
 *
 * Sample convention: samples are Gaussian-weighted, ftil(x) = exp(-r^2/2) f(x),
 * unless the plan was made with SGL_SAMPLES_PHYSICAL (FP64 plans only), in
 * which case they are the plain values f(x).
 *
 * Layouts (index maps of Sect. 3.4, with i < B):
 *   samples      [batch][i][j][k], complex interleaved (re, im),
 *                psi = 4B^2 i + 2B j + k within one function;
 *   coefficients [batch][omega], complex interleaved,
 *                omega(n,l,m) = n(n-1)(2n-1)/6 + l(l+1) + m, |m| <= l < n <= B,
 *                Omega = B(B+1)(2B+1)/6 per function.
 * Element type: double (complex128) for SGL_FP64 plans, float (complex64)
 * for every other precision.
 *
 * Buffers: every data pointer may point to device memory or to host memory
 * (pinned or pageable); the library asks the CUDA driver which it is.  Host
 * buffers are staged through plan-owned device memory, and the call then
 * synchronizes its stream before it returns; on single-bandlimit plans of
 * 16 or more functions on complex samples such a call runs in chunks of
 * functions that grow from n/16 by a factor of about 1.6 (4, 7, 12, 20, 21
 * for 64 functions; in the reverse order when only the output is on the
 * host), the host-to-device copies of later chunks and the device-to-host
 * copies of earlier ones (on two streams of the plan) overlapping the
 * kernels of the chunk in between (the first such call builds the chunk
 * plans; the results equal those of one device-buffer call).  Device buffers
 * are used in place and the call is asynchronous (stream-ordered); they
 * must be aligned to the complex element (16 bytes for SGL_FP64 plans, 8
 * otherwise: the kernels move whole complex values), else the call returns
 * SGL_ERR_ARG.  Inputs are never modified.  The caller owns all data buffers; the plan owns its
 * tables and workspace.
 *
 * Errors: argument errors are found before any work is queued and returned
 * as SGL_ERR_ARG.  CUDA launch errors are returned as SGL_ERR_CUDA.  A
 * device-side error flag (a bounded wait that gave up) is latched in the plan
 * and returned as SGL_ERR_TIMEOUT by the next call that synchronizes or by
 * sgl_check().  No call aborts the process.  sgl_last_error() returns a
 * message for the most recent failure on a plan (or, when passed NULL, for
 * the most recent failed creation or plan-free call on the calling thread).
 *
 * Concurrency: a plan's workspace is shared by its calls, so calls on one
 * plan must be ordered (one stream, or synchronized); distinct plans are
 * independent.
 */
#ifndef SGL_H_
#define SGL_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct sgl_plan_s* sgl_plan_t;   /* opaque; freed by sgl_destroy */
typedef struct CUstream_st* sgl_stream_t; /* a cudaStream_t; NULL = legacy default stream */

typedef enum {
  SGL_OK = 0,
  SGL_ERR_ARG = 1,          /* invalid argument (size, pointer, enum) */
  SGL_ERR_ALLOC = 2,        /* device or host allocation failed */
  SGL_ERR_CUDA = 3,         /* a CUDA runtime call or launch failed */
  SGL_ERR_TIMEOUT = 4,      /* a bounded device-side wait gave up */
  SGL_ERR_UNSUPPORTED = 5   /* valid but unsupported request (e.g. B too large) */
} sgl_status;

typedef enum {
  SGL_FP64 = 0,    /* every stage in double precision on the CUDA cores */
  SGL_FP32 = 1,    /* every stage in single precision on the CUDA cores */
  SGL_TF32X3 = 2,  /* FP32 FFT; Legendre and radial stages on tcgen05 tensor
                      cores as three TF32 products (hi*hi + hi*lo + lo*hi)
                      with FP32 accumulation; bandlimits divisible by 4 */
  SGL_TF32 = 3,    /* as SGL_TF32X3 with the hi*hi product only (inputs and
                      tables rounded to TF32, 11 significant bits): the fast,
                      low-accuracy variant (normwise error of order 1e-3) */
  SGL_BF16X3 = 4,  /* as SGL_TF32X3 with BF16 hi/lo pairs (8 + 8 significant
                      bits) on the kind::f16 tensor-core path: normwise error
                      of order 1e-5 */
  SGL_FP16X3 = 5   /* the Legendre sums (Eq. DLT) and radial sums (Eq.
                      DRT_matrix) as three products of FP16 hi/lo pairs
                      (11 + 11 significant bits, as TF32x3) on the kind::f16
                      tensor-core path, FP32 accumulation and FFT.  FP16's
                      range is held by power-of-two scales: one per table
                      block (each order m and parity of the Legendre tables,
                      each degree of the radial tables), chosen on the host,
                      and one per function and stage for the data, taken from
                      the largest magnitude of the function's phi-spectra
                      (forward) or coefficients (inverse), measured by the
                      kernels of each call, times a bound on the growth
                      through the table for the second stage.  Normwise
                      error as TF32x3 (of order 1e-7 to 1e-6) for inputs of
                      any magnitude FP32 holds; bandlimits divisible by 4 */
} sgl_precision;

typedef enum {
  SGL_SAMPLES_WEIGHTED = 0, /* samples are exp(-r^2/2) f(x) */
  SGL_SAMPLES_PHYSICAL = 1, /* samples are f(x); SGL_FP64 plans only */
  SGL_SAMPLES_REAL = 2      /* real f: samples exp(-r^2/2) f(x) as reals (see below) */
} sgl_samples;

/*
 * Radial grids.  SGL_GRID_LAGUERRE: B radii, the zeros of the generalized
 * Laguerre polynomial L_B^(1/2) in t = r^2 (the default of sgl_plan; exact
 * for bandlimit B: 4B^3 samples per function).  SGL_GRID_HALF_RANGE_HERMITE:
 * the paper's own grid, 2B radii at the nodes of the half-range Gauss-Hermite
 * rule of order 2B (Thm 3.3, Thm 3.4 / Eq. zwischenstufe_2: 8B^3 samples per
 * function, samples [batch][i < 2B][j][k]).  The coefficients do not depend
 * on the grid.
 */
typedef enum {
  SGL_GRID_LAGUERRE = 0,
  SGL_GRID_HALF_RANGE_HERMITE = 1
} sgl_grid_kind;

/*
 * Real functions (SGL_SAMPLES_REAL, sgl_plan only, every precision).  For a
 * real f the coefficients obey fhat_{n,l,-m} = (-1)^m conj(fhat_{n,l,m})
 * (Def 2.1: Y_l^{-m} = (-1)^m conj(Y_l^m), real radial part), so a real
 * function carries half the information of a complex one.  Such a plan
 * transforms the functions two at a time as the real and imaginary parts of
 * one complex function and separates the two coefficient sets with that
 * symmetry: about half the work and half the sample bytes per function.
 *   samples      [batch][i][j][k] reals (double for SGL_FP64, else float),
 *                weighted as SGL_SAMPLES_WEIGHTED; sgl_sample_count counts
 *                reals, and sample pointers need the real type's alignment;
 *   coefficients the full complex layout above (both signs of m).
 *   sgl_forward  the coefficients of the real functions (obeying the
 *                symmetry up to rounding);
 *   sgl_inverse  the real part of the inverse transform of the given
 *                coefficients (the inverse of their symmetric part), so any
 *                coefficient array is accepted;
 *   sgl_adjoint  the adjoints of these two maps for the real inner product
 *                on samples and Re <u, v> on coefficients: of_inverse == 0
 *                gives the real part of the complex adjoint, of_inverse != 0
 *                the complex adjoint of real samples.
 * Host buffers are staged in one piece (no chunked overlap).
 */

/* Largest supported bandlimit.  2B must factor as 2^a * q with 2^a <= 16
 * (the power of two capped at 16) and q <= 16; every B <= 16 and every
 * multiple of 8 up to 128 qualifies. */
#define SGL_MAX_B 128

/*
 * sgl_plan - create a plan for `batch` functions of bandlimit B.
 *   out      receives the plan (set to NULL on failure).
 *   B        bandlimit, 1 <= B <= SGL_MAX_B (see above for the factor rule).
 *   batch    number of functions per call, >= 1.
 *   prec     an sgl_precision.
 *   samples  an sgl_samples; SGL_SAMPLES_PHYSICAL requires SGL_FP64;
 *            SGL_SAMPLES_REAL makes a plan for `batch` real functions.
 * Builds the FP64 tables on the host (nodes and weights of Thm 3.1 and of the
 * radial Gauss-Laguerre rule; Legendre functions, Def 2.1 and Eq.
 * legendre_recurrence; radial functions, Lemma 3.7), uploads them and
 * allocates the workspace on the current CUDA device.
 */
sgl_status sgl_plan(sgl_plan_t* out, int B, int batch, int prec, int samples);

/*
 * sgl_plan_grid - sgl_plan on the radial grid `grid` (an sgl_grid_kind).
 * SGL_GRID_LAGUERRE is sgl_plan itself.  SGL_GRID_HALF_RANGE_HERMITE takes
 * every precision and sample convention.  Sample counts, offsets, sgl_grid's
 * r and w_r arrays and the host-buffer staging follow the plan's 2B radii.
 * Tensor-core plans run each function's radial sums (Eq. DRT_matrix over the
 * 2B nodes) as two partial sums over the first and the second B nodes, added
 * by one more kernel per forward call (Thm 3.3 and Thm 3.4 are unchanged:
 * the same rule, summed in two parts); with SGL_SAMPLES_REAL the real
 * functions are paired first, as for sgl_plan, and each pair is split into
 * its halves.  Host buffers are staged whole, without sub-batches.
 */
sgl_status sgl_plan_grid(sgl_plan_t* out, int B, int batch, int prec, int samples, int grid);

/*
 * sgl_plan_many - one plan for nfn functions with their own bandlimits
 * B_per_fn[f] (each obeying the rules of sgl_plan), weighted samples.
 * Samples of function f start at element offset sgl_sample_offset(plan, f)
 * of the samples buffer and its coefficients at sgl_coeff_offset(plan, f)
 * (complex elements); functions are packed in order, each in its own
 * single-function layout.  All functions run in the same kernel launches.
 */
sgl_status sgl_plan_many(sgl_plan_t* out, const int* B_per_fn, int nfn, int prec);

/*
 * sgl_forward - SGL coefficients of the samples (Thm 3.4 quadrature, computed
 * as Algorithm 3: phi-FFT of every ring (Eq. SFFT_rearranged), a Legendre sum
 * per order m (Eq. DLT), a radial sum per degree l (Eq. DRT)).
 *   samples  batch sample arrays (layout above), device or host.
 *   coeffs   batch coefficient arrays, device or host; fully overwritten.
 */
sgl_status sgl_forward(sgl_plan_t plan, const void* samples, void* coeffs, sgl_stream_t stream);

/*
 * sgl_inverse - samples on the grid of the function with the given
 * coefficients (Algorithm 4: iDRT per l, Legendre synthesis per m, inverse
 * phi-FFT; no weights).  The phi-frequency m = B (Nyquist) is zero.
 */
sgl_status sgl_inverse(sgl_plan_t plan, const void* coeffs, void* samples, sgl_stream_t stream);

/*
 * sgl_adjoint - the Hermitian adjoint of one of the two maps (Sect. 3.4):
 *   of_inverse == 0: adjoint of sgl_forward, coefficients -> samples,
 *                    out = diag(what_i beta_j) * inverse(in);
 *   of_inverse != 0: adjoint of sgl_inverse, samples -> coefficients,
 *                    out = the forward sum with what_i and beta_j dropped.
 * For SGL_SAMPLES_PHYSICAL plans the adjoint is taken of the physical maps.
 */
sgl_status sgl_adjoint(sgl_plan_t plan, int of_inverse, const void* in, void* out, sgl_stream_t stream);

/*
 * sgl_grid - copy the grid of function `fn` (0 for single-B plans) to host
 * arrays: r[R], theta[2B], phi[2B], w_r[R] (= what_i), w_theta[2B]
 * (= beta_j), with R = sgl_radii(plan, fn) (B, or 2B on the paper's grid).
 * Any pointer may be NULL to skip that array.
 */
sgl_status sgl_grid(sgl_plan_t plan, int fn, double* r, double* theta, double* phi,
                    double* w_r, double* w_theta);

/* Element counts and offsets (complex elements; reals for the samples of
 * SGL_SAMPLES_REAL plans). */
int64_t sgl_sample_count(sgl_plan_t plan);           /* whole batch */
int64_t sgl_coeff_count(sgl_plan_t plan);            /* whole batch */
int64_t sgl_sample_offset(sgl_plan_t plan, int fn);  /* -1 if fn out of range */
int64_t sgl_coeff_offset(sgl_plan_t plan, int fn);
int     sgl_num_functions(sgl_plan_t plan);
int     sgl_bandlimit(sgl_plan_t plan, int fn);      /* -1 if fn out of range */
int     sgl_radii(sgl_plan_t plan, int fn);          /* radial nodes of fn; -1 if out of range */
int64_t sgl_workspace_bytes(sgl_plan_t plan);        /* device bytes the plan holds */

/* Number of kernel launches one sgl_forward / sgl_inverse call makes. */
int sgl_launches_per_call(sgl_plan_t plan);

/* Read the plan's device error flag with a copy on `stream`, synchronize that
 * stream, and return the latched state: SGL_OK, or SGL_ERR_TIMEOUT once any
 * bounded device-side wait of the plan has given up. */
sgl_status sgl_check(sgl_plan_t plan, sgl_stream_t stream);

/*
 * Stage timing (profiling aid).  While enabled, every stage launch of the
 * plan is bracketed by CUDA events recorded on the call's stream; sgl_stage_times
 * synchronizes on the last event and returns, for each of the SGL_NUM_STAGES
 * stages, the summed device milliseconds and the number of launches since
 * profiling was enabled (arrays of SGL_NUM_STAGES entries, either may be NULL).
 * Stage names: sgl_stage_name(i).  Disabling clears the sums.
 */
#define SGL_NUM_STAGES 6
sgl_status  sgl_set_profiling(sgl_plan_t plan, int enable);
sgl_status  sgl_stage_times(sgl_plan_t plan, double* ms, int64_t* launches);
const char* sgl_stage_name(int stage);

/*
 * sgl_autotune - choose the plan's launch configuration by timing it on this
 * GPU (an implementation aid; the paper has no counterpart).  Tuned: the ring
 * pairs per CTA of the forward and of the inverse phi-FFT, and for
 * SGL_TF32X3 plans the tile width policy of the inverse radial stage.  Each
 * candidate is timed with CUDA events over whole forward or inverse calls
 * (one warm-up, best of three) on `stream`; the fastest is kept.  The
 * transforms computed are the same for every candidate (the FFT choices give
 * identical results; the radial tile policy changes only the summation order
 * of the TF32x3 accumulation).
 *   samples, coeffs  device buffers of sgl_sample_count / sgl_coeff_count
 *                    complex elements, used as scratch: both are overwritten.
 *   cache_path       NULL, or a text file of earlier results: a line for this
 *                    GPU model, precision and bandlimit list is applied without
 *                    timing; otherwise the result is appended to the file.
 * Synchronizes `stream`; replaces device schedules, so call it before capturing
 * the plan's calls in a CUDA graph.  Host buffers give SGL_ERR_ARG.
 */
sgl_status sgl_autotune(sgl_plan_t plan, void* samples, void* coeffs, const char* cache_path,
                        sgl_stream_t stream);

/* The plan's launch configuration as text, e.g. "fft_fwd_jp=8 fft_inv_jp=16
 * rad_inv_narrow=65 source=timed"; valid until the next call on the plan. */
const char* sgl_tuning(sgl_plan_t plan);

/*
 * sgl_selftest_wait - check the failure detection of the tensor-core kernels
 * on the current device (an implementation aid; the paper has no
 * counterpart).  Those kernels bound every wait on an mbarrier and, when a
 * wait gives up, set the plan's error flag, wait (bounded) for the copies and
 * MMAs they had already issued, free their tensor memory and end (sgl_check
 * then returns SGL_ERR_TIMEOUT).  This call runs one small kernel that holds
 * tensor memory and has a copy in flight while it waits on a barrier that is
 * never completed, with the bound limit_ns (1 .. 2e9 ns), and stores 1 in
 * *gave_up when the wait gave up, the wind-down finished and the kernel
 * ended as designed (0 otherwise).
 * Synchronous; SGL_ERR_ARG for a bad bound or a NULL pointer.
 */
sgl_status sgl_selftest_wait(int64_t limit_ns, int* gave_up);

/*
 * sgl_set_graphs - run the plan's calls through CUDA graphs of its own (an
 * implementation aid; the paper has no counterpart).  While enabled, every
 * sgl_forward, sgl_inverse and sgl_adjoint call with device buffers replays a
 * graph of that call's launches on the caller's stream: one launch in place
 * of the plan's (up to 34 for uneven bandlimits).  The graph of a call kind
 * (direction, weights) and buffer pair is captured on its first call, on a
 * stream of the plan (nothing runs during the capture; the replay follows on
 * the caller's stream), and kept: at most 8 per plan, the least recently used
 * one dropped first, so callers that reuse their buffers capture once.  Calls
 * with host buffers, calls while stage profiling is on, and calls on a stream
 * that is itself being captured launch directly as before.  sgl_autotune and
 * sgl_set_dlt drop the plan's graphs (their launches change); so does
 * disabling.  Results are those of the direct launches, bit for bit.
 */
sgl_status sgl_set_graphs(sgl_plan_t plan, int enable);

/* Number of graphs the plan holds (0 .. 8); -1 for a NULL plan. */
int sgl_graph_count(sgl_plan_t plan);

/* Message for the last failure on `plan`; with NULL, for the last failed
 * plan creation or plan-free call (sgl_forward_noalloc, sgl_midpoint) on the
 * calling thread.  The string stays valid until the next call on the same
 * plan (with NULL: the next such call on the same thread). */
const char* sgl_last_error(sgl_plan_t plan);

/* Release the plan, its tables and its workspace.  NULL is ignored. */
void sgl_destroy(sgl_plan_t plan);

/*
 * sgl_forward_noalloc - the FP64 forward transform (same result as
 * sgl_forward on an FP64, weighted-samples plan of the same B and batch),
 * for callers that cannot allocate device memory.  The paper has no
 * counterpart; this entry point exists for deployment.
 *
 * Who needs it: code that must not call cudaMalloc once it is running, e.g.
 * a host application whose device memory is owned by its own allocator or a
 * fixed budget, a plugin running inside such an application, or a real-time
 * loop where an allocation could block on the device.  Creating a plan
 * allocates tables and workspace; this call does not: its scratch lives in a
 * static device array compiled into the library (16 MiB of doubles), and its
 * tables and launch schedules in a second static array (8 MiB).  A GPU holds
 * both arrays from the moment the part of the library that defines them is
 * loaded on it until the process exits.  Under CUDA's lazy module loading
 * (the default) that happens at the first call on the device, which also
 * loads the forward kernels' code: the driver reserves that memory then, and
 * the call fails with SGL_ERR_CUDA if the device has no room left.  Make the
 * first call at start-up, before the caller's allocator takes the device's
 * memory, or run with CUDA_MODULE_LOADING=EAGER (everything loaded when the
 * library is).  Later calls reserve nothing.
 *
 *   B        bandlimit, 1 <= B <= 32 (and the factor rule of SGL_MAX_B).
 *   batch    functions, >= 1, with 4 B^2 (2B-1) + 2 B^3 doubles of scratch per
 *            function fitting the 2^21-double scratch: B = 32 allows 6
 *            functions, B = 16 allows 52, B = 8 allows 431.  Larger requests
 *            return SGL_ERR_UNSUPPORTED with a message saying how much
 *            scratch they need.  The tables and launch schedules of the
 *            call must also fit the 8 MiB table array; only at B = 1 does
 *            that bind first (about 170,000 functions), again with
 *            SGL_ERR_UNSUPPORTED and a message.
 *   samples  device pointer, batch x 4B^3 complex doubles (weighted samples).
 *   coeffs   device pointer, batch x Omega complex doubles; overwritten.
 *            Host pointers are rejected (SGL_ERR_ARG): staging them would
 *            need device memory; so are pointers not 16-byte aligned and
 *            device memory of a GPU other than the current one (managed
 *            memory is accepted).
 *   stream   stream the kernels are launched on.
 *
 * Set-up: the first call on a device looks up the device addresses of the
 * two static arrays (cudaGetSymbolAddress, with that device current), and a
 * call whose (B, batch) differs from the previous call on that device copies
 * the new tables into the static array and synchronizes `stream`.  Make such
 * calls before any stream capture.
 *
 * Sharing: every call on a device uses the same scratch and table arrays,
 * which keep the last call's contents.  Calls whose kernels overlap on the GPU
 * (different streams, or different (B, batch) while earlier work still runs)
 * race on them.  Nothing in the scratch has to start at zero: each stage
 * writes every element the next stage reads.  On failure the message is
 * available from sgl_last_error(NULL).
 */
sgl_status sgl_forward_noalloc(int B, int batch, const void* samples, void* coeffs, sgl_stream_t stream);

/*
 * sgl_set_dlt - choose how the forward Legendre sums (Eq. DLT) of an
 * SGL_FP64 or SGL_FP32 plan are taken: seminaive == 0, directly (the
 * default); seminaive != 0, by the paper's seminaive algorithm (Eq. DCT,
 * Eq. dct_trick): a DCT of every order's data over the rings (with the
 * theta-parity fold: a DCT-II of the symmetric and a DCT-IV of the
 * antisymmetric part, each of length B, through an FFT of length 2B), then
 * for each degree l an inner product over the first deg/2 + 1 DCT
 * coefficients with the stored cosine coefficients of Lambda_lm (of
 * Lambda_lm / sin theta for odd m).  Same results up to rounding; applies to
 * sgl_forward and to sgl_adjoint(of_inverse != 0).  Tensor-core plans return
 * SGL_ERR_UNSUPPORTED.  Not safe while calls on the plan are in flight.
 */
sgl_status sgl_set_dlt(sgl_plan_t plan, int seminaive);

/*
 * sgl_midpoint - SGL coefficients by the midpoint rule on a Cartesian grid,
 * the current practice the paper's Discussion describes (built to compare
 * accuracy and cost with the SGL transform; no sampling theorem makes it
 * exact):
 *   fhat_nlm ~= sum_k f(x_k) conj(H_nlm(x_k)) exp(-|x_k|^2) dV,
 * the midpoint rule for the inner product of Eq. (inner_product); x_k are the
 * midpoints of the M^3 cells of the cube [-L, L]^3 and dV = (2L/M)^3.
 *   B       bandlimit, 1..32.
 *   M, L    cells per axis (1..1024) and half-width of the cube (> 0).
 *   batch   functions, 1..65535.
 *   prec    SGL_FP64 (complex double) or SGL_FP32 (complex float).
 *   f       device pointer: batch x M^3 complex PHYSICAL samples f(x_k),
 *           index (ix * M + iy) * M + iz, x = -L + (ix + 1/2) 2L/M (same for
 *           y, z).
 *   coeffs  device pointer: batch x Omega complex in the coefficient layout;
 *           overwritten (cleared, then accumulated with atomic adds, so the
 *           summation order and the last bits vary from run to run).
 *   stream  stream the memset and the kernel are queued on (asynchronous).
 * Errors: SGL_ERR_ARG / SGL_ERR_UNSUPPORTED for arguments (host or misaligned
 * pointers included), SGL_ERR_CUDA for launch errors; sgl_last_error(NULL)
 * has the message.
 */
sgl_status sgl_midpoint(int B, int M, double L, int batch, int prec, const void* f, void* coeffs,
                        sgl_stream_t stream);

/* Library version string. */
const char* sgl_version(void);

#ifdef __cplusplus
}
#endif

#endif /* SGL_H_ */
