/*
 * gfdeconv — guided-filter non-blind image deconvolution on one GB300 GPU.
 *
 * The method (Yang, Zhu, Zhang, Huang, arXiv 1609.01839):
 *   observation model y = h * u_orig + gamma, circular convolution, i.i.d.
 *   Gaussian noise of variance sigma^2 (Sec. 1, Eq. 1; h and sigma known);
 *   Step 0 u_E = 0; then per iteration (Sec. 3.1, Steps 1-3):
 *     lambda by the discrepancy principle (Sec. 3.2, Eq. 10-12),
 *     u_I from Eq. 8 and u_p from Eq. 9 (FFT-domain solves of Eq. 6 and 7),
 *     u = guidfilter(u_I, u_p, w, eps) (Sec. 2, Eq. 3-5), u_E <- u.
 *
 * Conventions for every entry point:
 *   - Images are float32, row-major, M rows by N columns, with M and N powers
 *     of two in [8, 4096] (the canvas; pad other sizes before calling).
 *   - Buffers named "device" are CUDA device pointers on the context's device,
 *     owned by the caller; the library never frees or retains them after the
 *     call's stream work completes.  The library owns only its workspace.
 *     Device image buffers (observations, outputs, u_orig, u_init, spectra)
 *     must start on a 16-byte boundary (cudaMalloc and PyTorch allocations
 *     do); a misaligned one is rejected with GFD_ERR_INVALID_ARG.
 *   - Calls are stream-ordered and asynchronous on `stream` (a cudaStream_t;
 *     NULL = the legacy default stream) unless stated otherwise.  Argument
 *     errors are returned synchronously, before any launch.  Conditions found
 *     on the device (non-convergence, non-finite values, an invalid PSF) are
 *     reported per image by gfdeconv_status() after the stream is synchronised.
 *   - A context is not thread-safe: use one context per host thread / stream.
 *   - Return value: GFD_OK (0) or a negative gfd_status code.
 */
#ifndef GFDECONV_H
#define GFDECONV_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct gfdeconv_ctx gfdeconv_ctx;

typedef enum {
  GFD_OK = 0,
  GFD_ERR_INVALID_ARG = -1,      /* null pointer, bad w/eps/sigma/iters/PSF size */
  GFD_ERR_UNSUPPORTED_SIZE = -2, /* M or N not a power of two in [8, 4096] */
  GFD_ERR_NONFINITE_INPUT = -3,  /* non-finite scalar argument */
  GFD_ERR_ALLOC = -4,            /* workspace allocation failed */
  GFD_ERR_CUDA = -5,             /* a CUDA runtime call failed */
  GFD_ERR_NONCONVERGED = -6,     /* (status) lambda root outside the bracket */
  GFD_ERR_TIMEOUT = -7,          /* reserved: no entry point waits on the device */
  GFD_ERR_SCRATCH_LIMIT = -8     /* gfdeconv_fft2_r2c_noalloc: M*N above its static scratch */
} gfd_status;

/* Per-image status bits returned by gfdeconv_status(). */
#define GFD_STATUS_NONCONVERGED 1 /* Eq. 11 root lies below 1e-14: lambda = 1e-14 returned */
#define GFD_STATUS_NONFINITE 2    /* a non-finite residual or lambda appeared */
#define GFD_STATUS_BAD_PSF 4      /* sum of h <= 0 */
#define GFD_STATUS_BAD_RHO 8      /* Eq. 12 radicand <= 0 */
#define GFD_STATUS_PASSES_EXHAUSTED 16 /* the lambda pass schedule ran out with the
                                          root still bracketed: lambda is the
                                          bracket's geometric midpoint, which may
                                          miss the requested lambda_rtol */
#define GFD_STATUS_COPY_TIMEOUT 32 /* a column pass's bulk copy of a spectrum tile
                                      did not complete within its wait limit
                                      (the kernel went on; this image's results
                                      are not to be trusted) */

/* Arithmetic of the guided filter's window statistics (Sec. 2, Eq. 3-4:
 * mu_k, pbar_k, sigma_k^2 = E[I^2] - mu_k^2 and the covariance are formed from
 * window sums of I, p, I^2 and I p).  Every variant takes the statistics about
 * a per-strip reference value (a_k and b_k do not depend on it). */
#define GFD_VAR_COMPENSATED 0  /* split sums (default): each deviation is split on a
                                  power-of-two grid from a bound on |u_I|, |u_p| into
                                  an integer leading part (window sums exact in int32,
                                  n S_II - S_I^2 exact in int64) and an FP32 remainder
                                  (its sums compensate the leading part's truncation) */
#define GFD_VAR_FP64 1         /* FP64 accumulators (reference point; slow on this part) */
#define GFD_VAR_FP32 2         /* plain FP32 sums about the reference (precision study) */
#define GFD_VAR_FP32_RAW 3     /* plain FP32 sums of the raw values, no reference shift */
#define GFD_VAR_DOUBLE_FLOAT 4 /* double-float (FP32 pairs, error-free two-sum and
                                  two-product) running sums: ~48-bit sums */

/* Window boundary of the guided filter (Sec. 2). */
#define GFD_BOUNDARY_PERIODIC 0  /* windows wrap around the canvas; every window holds
                                    w^2 pixels and Eq. 3 and 5's 1/w^2 is exact (default) */
#define GFD_BOUNDARY_TRUNCATED 1 /* windows are cut at the canvas edge and every mean is
                                    normalised by the number of pixels it covers */

typedef struct {
  /* Window-statistics arithmetic: one of GFD_VAR_* (0 = compensated). */
  int var_precision;
  /* rho of the discrepancy target (Sec. 3.2): <= 0 selects Eq. 12, else a
   * fixed value in (0, 1]. */
  double rho;
  /* 1 (default): capture each solve as a CUDA graph and replay it when the
   * same batch (pointers, sizes, parameters) is solved again. */
  int use_graphs;
  /* Spectral passes of Eq. 11 launched per iteration after the one fused
   * into the forward transform (images whose root is resolved skip them) in
   * iterations 0-2, whose brackets are wide; later iterations, whose bracket
   * is centred on the extrapolated root, launch at most 2.  <= 0 selects 4,
   * at most 16.  If an image's root is still bracketed after the last pass of
   * an iteration, GFD_STATUS_PASSES_EXHAUSTED is set. */
  int lambda_max_passes;
  /* Relative width of the final lambda bracket (the root search stops below
   * it); <= 0 selects 1e-13, else in [1e-14, 1e-2]. */
  double lambda_rtol;
  /* Guided-filter window boundary: one of GFD_BOUNDARY_* (0 = periodic). */
  int boundary;
  /* Path of a tile-shape file written by gfdeconv_autotune (read at create;
   * NULL or "" = built-in shapes).  The string is not retained. */
  const char* tune_cache;
} gfdeconv_opts;

/* One image of a batched solve.  All pointers are device pointers. */
typedef struct {
  const float* y;   /* observation, M*N */
  int M, N;         /* canvas, powers of two in [8, 4096] */
  const float* h;   /* PSF, kh*kw row-major, centre at (kh/2, kw/2) */
  int kh, kw;       /* odd, 1..255; a PSF larger than the canvas wraps around it */
  double sigma;     /* noise std (Eq. 1), > 0 */
  int w;            /* guided-filter window, odd, 1..17 */
  double eps;       /* guided-filter regulariser (Eq. 3), > 0 */
  float* u_out;     /* result u^K, M*N; also holds the iterate during the solve */
  double* lambda_out; /* [iters] lambda_k (+inf: u_E in K, Sec. 3.2) or NULL */
  double* isnr_out; /* [iters] ISNR of u^{k+1} in dB, needs u_orig, or NULL */
  double* res_out;  /* [iters] ||h*u_E^k - y||^2 or NULL */
  const float* u_orig; /* clean image for ISNR, M*N, or NULL */
  const float* u_init; /* starting u_E (resume), M*N, or NULL for Step 0's 0 */
  float* uI_out;    /* last iteration's u_I (Eq. 8), M*N, or NULL */
  float* up_out;    /* last iteration's u_p (Eq. 9), M*N, or NULL */
  float* u_iters;   /* [iters][M*N] checkpoints: the iterate u_E^k entering each
                       iteration k (u_E^0 = 0 or u_init), for gfdeconv_backward_batched;
                       or NULL */
} gfdeconv_image;

/* Gradients of one image for gfdeconv_backward_batched (device pointers). */
typedef struct {
  const float* g_u; /* in: dL/du^K, M*N (u^K = the solve's u_out) */
  float* g_y;       /* out: dL/dy, M*N */
  float* g_h;       /* out: dL/dh, kh*kw */
  double* g_eps;    /* out: dL/deps, one double */
} gfdeconv_grad;

/* Create a context on `cuda_device` (opts NULL = defaults).  Allocates the
 * twiddle and gradient-weight tables; workspaces grow on first use. */
int gfdeconv_create(gfdeconv_ctx** out, int cuda_device, const gfdeconv_opts* opts);

/* Destroy a context and free its workspace (synchronises the device). */
void gfdeconv_destroy(gfdeconv_ctx* ctx);

/* The whole method on one image (Sec. 3.1 Steps 0-3 with Sec. 3.2's lambda):
 * `iters` iterations from u_E = 0 (or u_init), writing u^iters to u_out and
 * the per-iteration lambda_k / ISNR_k when the arrays are given. */
int gfdeconv_solve(gfdeconv_ctx* ctx, const float* y, int M, int N, const float* h,
                   int kh, int kw, double sigma, int w, double eps, int iters,
                   float* u_out, double* lambda_out, double* isnr_out,
                   const float* u_orig, const float* u_init, void* stream);

/* The same method on n independent images of possibly different sizes, run
 * together: every phase of an iteration is one launch per distinct canvas
 * size covering all images of that size.  `imgs` is a HOST array of n
 * descriptors whose pointers are device pointers. */
int gfdeconv_solve_batched(gfdeconv_ctx* ctx, int n, const gfdeconv_image* imgs,
                           int iters, void* stream);

/* As gfdeconv_solve_batched, but every pointer in `imgs` is HOST memory
 * (pinned memory recommended): inputs are copied to the device, the batch is
 * solved, outputs are copied back, and the call returns after the stream has
 * been synchronised. */
int gfdeconv_solve_batched_host(gfdeconv_ctx* ctx, int n, const gfdeconv_image* imgs,
                                int iters, void* stream);

/* u = guidfilter(I, p, w, eps) (Sec. 2, Eq. 3-5) with periodic windows:
 * I guidance, p filtering input, all M*N device buffers. */
int gfdeconv_guidfilter(gfdeconv_ctx* ctx, const float* I, const float* p, int M, int N,
                        int w, double eps, float* u_out, void* stream);

/* Observations whose size is not a power of two (the paper's images are
 * square powers of two; reading: pad only the observation).  y (m x n,
 * device) is extended to y_canvas (M x N, device, M >= m, N >= n powers of
 * two in [8, 4096]) by symmetric reflection at its bottom and right edges
 * (the edge sample repeated, period 2m and 2n); solve on the canvas, then
 * gfdeconv_crop takes the top-left m x n part of a canvas result.  Both
 * return GFD_ERR_INVALID_ARG when m > M or n > N. */
int gfdeconv_pad_symmetric(gfdeconv_ctx* ctx, const float* y, int m, int n, float* y_canvas,
                           int M, int N, void* stream);
int gfdeconv_crop(gfdeconv_ctx* ctx, const float* u_canvas, int M, int N, float* u, int m, int n,
                  void* stream);

/* Guided filter with a colour guidance image (the guided filter applies to
 * colour as well as grey-scale images, Sec. 3.1): I is 3 device planes
 * [3][M][N] (channel-major), p and u_out M*N device planes.  Per window,
 * a_k = (Sigma_k + eps U)^-1 (mean(I p) - mu_k pbar_k) with Sigma_k the
 * window covariance of the 3 channels (Eq. 3 with a 3-vector slope),
 * b_k = pbar_k - a_k . mu_k (Eq. 4), u = abar . I + bbar (Eq. 5).  Window
 * statistics and the 3 x 3 solves in FP64; periodic or truncated windows as
 * gfdeconv_opts.boundary selects (var_precision does not apply). */
int gfdeconv_guidfilter_color(gfdeconv_ctx* ctx, const float* I, const float* p, int M, int N,
                              int w, double eps, float* u_out, void* stream);

/* 2-D real DFT of x (M*N device) into the packed half spectrum X (device,
 * M*(N/2) complex64 = M*N floats): X[m][l] = F(x)(m, l) for 1 <= l < N/2 and
 * X[m][0] = F(x)(m, 0) + i F(x)(m, N/2).  The DFT diagonalises the circular
 * operators of Sec. 3.1. */
int gfdeconv_fft2_r2c(gfdeconv_ctx* ctx, const float* x, int M, int N, float* X, void* stream);

/* gfdeconv_fft2_r2c without any allocation.  The paper has no counterpart:
 * this is an interface variant, not a step of the method.
 *
 * Same arguments, result and layout as gfdeconv_fft2_r2c, but the call makes
 * no cudaMalloc / cudaFree and calls no allocating library: its intermediate
 * row-pass plane and its kernel descriptor live in one file-scope
 * `static __device__ __align__(256)` array of GFD_NOALLOC_SCRATCH_BYTES,
 * allocated when the library's device code is loaded.  It serves callers that
 * must not allocate on the device: code running under a memory budget that a
 * caching allocator has already claimed in full (a cudaMalloc can fail there
 * although the caller has room in its own pool), and latency-bound loops for
 * which the workspace growth of gfdeconv_fft2_r2c (cudaFree synchronises the
 * whole device) is not acceptable.
 *
 * Limit: M*N <= GFD_NOALLOC_MAX_PIXELS (1024 x 1024); larger sizes return
 * GFD_ERR_SCRATCH_LIMIT before any work.  The first call on each device looks
 * up the scratch address with cudaGetSymbolAddress and caches it for the
 * process (host threads may race on that first call safely): make that first
 * call outside any stream capture.  The cached address belongs to the
 * device's current context; after cudaDeviceReset on that device, create a
 * new gfdeconv context and do not use this entry point again in the process.  Nothing in the scratch has to start
 * at zero: every call writes the descriptor and the whole intermediate plane
 * before reading them.  The scratch is shared by every call on a device, so
 * calls whose stream work overlaps (different streams, or different host
 * threads without ordering between them) race on it: order them on one stream
 * or synchronise between them.  ctx must be a live context (its twiddle table
 * is used; the context allocates nothing here either). */
#define GFD_NOALLOC_MAX_PIXELS (1024 * 1024)
#define GFD_NOALLOC_SCRATCH_BYTES (256 + 4 * GFD_NOALLOC_MAX_PIXELS)
int gfdeconv_fft2_r2c_noalloc(gfdeconv_ctx* ctx, const float* x, int M, int N, float* X,
                              void* stream);

/* Inverse of gfdeconv_fft2_r2c: x = (1/(M N)) * inverse DFT of the packed
 * half spectrum X (a Hermitian spectrum is assumed). */
int gfdeconv_fft2_c2r(gfdeconv_ctx* ctx, const float* X, int M, int N, float* x, void* stream);

/* Per-image status bits (GFD_STATUS_*) of the last solve on this context.
 * Synchronises the last solve's stream.  `n` entries are written. */
int gfdeconv_status(gfdeconv_ctx* ctx, int* per_image_status, int n);

/* Phases of a solve, for gfdeconv_solve_batched_timed. */
#define GFD_NUM_PHASES 8
#define GFD_PHASE_SETUP 0          /* statistics, rho, H = F(h), Y = F(y) (once) */
#define GFD_PHASE_ROW_FWD 1        /* row pass of F(u_E) */
#define GFD_PHASE_COL_FWD_LAMBDA 2 /* column pass of F(u_E) + first Eq. 11 pass */
#define GFD_PHASE_LAMBDA_PASS 3    /* further Eq. 11 passes (skip when resolved) */
#define GFD_PHASE_COL_SOLVE_INV 4  /* Eq. 8, 9 + inverse column passes */
#define GFD_PHASE_ROW_INV 5        /* inverse row passes -> u_I, u_p */
#define GFD_PHASE_GUIDED_FILTER 6  /* Eq. 3-5 (+ ISNR sums) */
#define GFD_PHASE_COPY 7           /* memsets / device copies */

/* Instrumentation: the same solve as gfdeconv_solve_batched, launched
 * directly (no graph) with a CUDA event pair on `stream` around every launch.
 * Adds each phase's summed device time in milliseconds to phase_ms[p] and its
 * launch count to phase_launches[p] (host arrays of GFD_NUM_PHASES entries).
 * Synchronises `stream` before returning. */
int gfdeconv_solve_batched_timed(gfdeconv_ctx* ctx, int n, const gfdeconv_image* imgs,
                                 int iters, void* stream, double* phase_ms,
                                 long long* phase_launches);

/* Autotuner of the batched solve (Sec. 3.1's per-iteration steps, scheduled
 * for this GPU; the paper has no counterpart).  Times the solve of `imgs`
 * (device buffers, as for gfdeconv_solve_batched; their outputs are
 * overwritten) on `stream` with event pairs around every launch, for each
 * candidate of one tile shape at a time:
 *   col_threads in {64, 128, 256}: threads per column-pass block, which fixes
 *     the tile width of the spectra (4096-row canvases always use 512);
 *   row_threads in {64, 128, 256}: threads per row-pass block (rows per item);
 *   gf_rows in {16, 32, 64}: output rows per guided-filter item;
 * keeping per canvas size the fastest over the phases the shape affects, then
 * times graph replays of the solve with 1 to 4 concurrent chains.  The
 * result applies to the context's later solves and, if `path` is not NULL
 * or "", is merged into that tile-shape file (other canvas sizes kept), which
 * gfdeconv_opts.tune_cache reads at create.  Synchronises `stream`.  Returns
 * GFD_ERR_INVALID_ARG for a malformed existing file or one that cannot be
 * written. */
int gfdeconv_autotune(gfdeconv_ctx* ctx, int n, const gfdeconv_image* imgs, int iters,
                      const char* path, void* stream);

/* Read a tile-shape file without a GPU (host only): *chains receives its
 * chain count (4 if it names none), *n_classes the number of canvas sizes it
 * holds, and the first max_classes of them go to shapes[5 * i + 0..4] as
 * (M, N, col_threads, row_threads, gf_rows).  A missing file is an empty
 * table.  Returns GFD_ERR_INVALID_ARG for a malformed file or a value outside
 * the ranges gfdeconv_autotune searches. */
int gfdeconv_tune_read(const char* path, int* chains, int* n_classes, int* shapes,
                       int max_classes);

/* Tile shapes the context uses for an M x N canvas (tuned or built-in) and
 * its chain count; any output pointer may be NULL. */
int gfdeconv_tune_get(gfdeconv_ctx* ctx, int M, int N, int* col_threads, int* row_threads,
                      int* gf_rows, int* chains);

/* Reverse mode of the unrolled method: given dL/du^K for each image, the
 * gradients dL/dy, dL/dh and dL/deps of a loss L of the result u^K of
 * `iters` iterations (Sec. 3.1 Steps 0-3 with Sec. 3.2's lambda).  `imgs`
 * are the descriptors of a completed gfdeconv_solve_batched call with u_iters
 * and lambda_out set (the checkpoints u_E^k and the lambda_k it wrote are
 * read, nothing else of its outputs); all images share one canvas size,
 * windows are periodic (gfdeconv_opts.boundary = 0).  Each iteration is
 * recomputed from its checkpoint with its lambda_k (U_E, Eq. 8-9, u_I and
 * u_p) and undone in reverse: the guided filter (Eq. 3-5), the spectral
 * solves (Eq. 8-9), lambda through the implicit derivative of Eq. 11 (where
 * lambda = inf, u_E in K, lambda is a constant and u_I = u_p = u_E), the
 * DFTs; H, Y and T = rho P sigma^2 (Eq. 12) collect their gradients over the
 * iterations.  FP32 spectra and planes, compensated (double-float) window
 * sums, FP64 sums over bins and pixels.  Returns GFD_ERR_INVALID_ARG for
 * missing checkpoints or lambdas, or mixed canvas sizes. */
int gfdeconv_backward_batched(gfdeconv_ctx* ctx, int n, const gfdeconv_image* imgs,
                              const gfdeconv_grad* grads, int iters, void* stream);

/* Number of kernel launches the last solve issued (for instrumentation). */
long long gfdeconv_last_launch_count(gfdeconv_ctx* ctx);

/* Text of the last CUDA runtime error behind a GFD_ERR_CUDA / GFD_ERR_ALLOC
 * return on this host thread ("no error" if none; static storage). */
const char* gfdeconv_last_cuda_error(void);

/* Architecture check: *binary_version receives the compute capability the
 * library's device code was compiled for, as the CUDA runtime reports it for
 * one library kernel loaded on `cuda_device` (cudaFuncAttributes::binaryVersion,
 * major * 10 + minor: 103 for sm_103a), and *device_cc the device's own
 * compute capability in the same form.  Either pointer may be NULL.  Needs a
 * CUDA device: without one it returns GFD_ERR_CUDA and writes nothing. */
int gfdeconv_device_arch(int cuda_device, int* binary_version, int* device_cc);

/* Human-readable text for a gfd_status code (static storage). */
const char* gfdeconv_strerror(int code);

#ifdef __cplusplus
}
#endif

#endif /* GFDECONV_H */
