// Host-side launchers of the device kernels (internal to the library).
#pragma once
#include <cuda_runtime.h>

#include "common.cuh"

namespace gfd {

enum PlaneSel : int {
  SEL_Y = 0,   // observation (real)
  SEL_U = 1,   // iterate / output (real)
  SEL_S = 2,   // spectrum scratch
  SEL_QI = 3,  // U_I then u_I
  SEL_QP = 4,  // U_p then u_p
  SEL_H = 5,   // PSF spectrum
  SEL_YS = 6,  // observation spectrum
  SEL_UI = 7,  // u_I (real)
  SEL_UP = 8,  // u_p (real)
};

// Tile shapes of one size class (threads per block of the row passes, which
// fixes rows per row item; of the column passes, which fixes the spectra's
// tile width; rows per guided-filter item), chosen by gfdeconv_autotune.
constexpr int DEF_ROW_THREADS = 256;
constexpr int DEF_COL_THREADS = 256;
constexpr int DEF_GF_ROWS = 64;

struct Tables {
  const float2* tw;    // W_L^m for every L = 2..4096, size L at offset tab_off(L)
  const float* d2;     // 4 sin^2(pi m / L), same layout
  const float4* twdf;  // W_L^m in double-float (re hi, re lo, im hi, im lo), same layout
};

// Images of a class sharing one guided-filter radius (contiguous range).
struct RadGroup {
  int img0, n_img, rad;
};

// Everything a launch needs about one size class.
struct ClassLaunch {
  ClassDesc cd;
  const ImgDesc* imgs;  // device array (whole batch)
  ImgState* st;         // device array (whole batch)
  int max_rad;          // largest guided-filter radius in the class
  int n_rad_groups;
  RadGroup rad_groups[9];
  int grid_div;         // persistent grids use 1/grid_div of the resident slots (0 = 1)
  int row_threads;      // threads per row-pass block (0 = DEF_ROW_THREADS)
  int gf_rows;          // largest rows per guided-filter item (0 = DEF_GF_ROWS)
  int class_id;         // index of the class in its plan (instrumentation)
};

// Row pass of the 2-D real DFT: real plane src -> packed rows dst.
// do_sum: accumulate the FP64 sum of src into st.sum_u.
cudaError_t launch_row_r2c(const ClassLaunch& c, const Tables& t, int src, int dst,
                           bool do_sum, cudaStream_t s);
// Inverse row pass: spectrum sel0 -> real plane dsel0 (and sel1 -> dsel1
// unless sel1 < 0), outputs scaled by `scale`.
cudaError_t launch_row_c2r(const ClassLaunch& c, const Tables& t, int sel0, int sel1, int dsel0,
                           int dsel1, float scale, cudaStream_t s);
// Tile width (columns per tile) of the spectra of an M x N class whose
// column passes run col_threads threads per block (0 = default).
int class_tile_width(int M, int N, int col_threads);
// Rows per item of a row pass of length-L transforms on an M-row class.
int rows_per_item(int L, int M, int row_threads);
// Plain column FFT src -> dst (in place allowed), forward or inverse.
cudaError_t launch_col_plain(const ClassLaunch& c, const Tables& t, int src, int dst,
                             bool inverse, cudaStream_t s);
// Forward column FFT of S in place fused with the first lambda pass.
cudaError_t launch_col_fwd_lambda(const ClassLaunch& c, const Tables& t, int iter,
                                  cudaStream_t s);
// Fallback lambda pass over the stored spectrum (exits early where resolved).
cudaError_t launch_lambda_pass(const ClassLaunch& c, int iter, bool last_chance,
                               cudaStream_t s);
// Spectral solves (Eq. 8, 9) fused with the inverse column FFTs: S -> QI, Qp.
cudaError_t launch_col_solve_inv(const ClassLaunch& c, const Tables& t, cudaStream_t s);
// Guided filter (Eq. 3-5): real planes (uI, up) -> u.  iter < 0: no ISNR.
// var_mode: GFD_VAR_*; boundary: GFD_BOUNDARY_*.
cudaError_t launch_guided_filter(const ClassLaunch& c, int iter, int var_mode, int boundary,
                                 cudaStream_t s);
// Colour guided filter: guidance I planar [3][M][N], p, window w; ab is a
// 4 * M * N workspace (a_r, a_g, a_b, b); u the output.
cudaError_t launch_guided_filter_color(const float* I, const float* p, int M, int N, int w,
                                       double eps, int boundary, float* ab, float* u,
                                       cudaStream_t s);
// Largest |u_I|, |u_p| of every image into ImgState::absmax (which must be
// zero before), for guided-filter calls outside a solve.
cudaError_t launch_plane_absmax(const ClassLaunch& c, cudaStream_t s);
// Double-float 2-D real DFT of real plane src into spectrum plane dst
// (SEL_H or SEL_YS); uses the S and Q_I planes as scratch.
cudaError_t launch_fft2_r2c_df(const ClassLaunch& c, const float4* twdf, int src, int dst,
                               cudaStream_t s);
// Setup kernels.
cudaError_t launch_setup_stats(const ClassLaunch& c, cudaStream_t s);
cudaError_t launch_init_u(const ClassLaunch& c, cudaStream_t s);
cudaError_t launch_setup_init(const ClassLaunch& c, double rho_fixed, cudaStream_t s);
cudaError_t launch_embed_psf(const ClassLaunch& c, int dst, cudaStream_t s);
cudaError_t launch_unpack_dc(const ClassLaunch& c, cudaStream_t s);

// Symmetric padding of an m x n plane to M x N, and the top-left crop back.
cudaError_t launch_pad_symmetric(const float* y, int m, int n, float* dst, int M, int N,
                                 cudaStream_t s);
cudaError_t launch_crop(const float* src, int N, float* dst, int m, int n, cudaStream_t s);

// Copy every image's iterate u_E into its checkpoint slot u_iters[k] (images
// without u_iters are skipped).
cudaError_t launch_save_iterate(const ClassLaunch& c, int k, cudaStream_t s);

// Per-image state of a backward solve (k_adjoint.cu).  Real planes are M*N
// floats, spectra packed row-major half spectra (M*N/2 float2).
struct AdjDesc {
  const float* y;
  const float* h;
  int kh, kw;
  double sigma, eps, rho_fixed;
  const float* uI;    // u_I, u_p of the recomputed forward step
  const float* up;
  float* gu;          // g_u of the step's output; then of its input
  float *A, *MU, *PB, *VE;                    // a, mu, pbar, sigma^2 + eps
  float *GI0, *GCOV, *GVAR, *GMU, *GPB;       // pointwise adjoints of Eq. 3-5
  float *guI, *gup;                           // g_uI, g_up
  float *gtmp, *gtmp2;                        // adjoint DFT results
  float2 *H, *Y, *UE, *UI, *Up, *GUI, *GUp;   // spectra of the step
  float2 *gUE, *gH, *gY;                      // their gradients
  const double* lam_hist;  // lambda_k of the forward solve, k = 0..iters-1
  double* lam;        // lambda of the step (+inf: u_E in K)
  double* acc;        // g_lam, P f', c, g_T, sum y, sum y^2, sum |h|, g_num, g_den
  double* g_eps;      // accumulated dL/deps
  double* g_eps_out;  // caller outputs
  float* gy_out;
  float* gh_out;
};
constexpr int ADJ_ACC = 9;
cudaError_t launch_adj_guided_filter(const AdjDesc* descs, int n, int M, int N, int rad,
                                     cudaStream_t s);
// Start of backward step k: lambda_k into every image's state, and the
// spectra U_I, U_p (Eq. 8-9) of the step from U_E, H, Y into UI, Up.
cudaError_t launch_adj_recompute(const AdjDesc* descs, int n, int M, int N, int k,
                                 const float* d2tab, cudaStream_t s);
cudaError_t launch_adj_spectral(const AdjDesc* descs, int n, int M, int N, const float* d2tab,
                                cudaStream_t s);
cudaError_t launch_adj_next(const AdjDesc* descs, int n, int M, int N, cudaStream_t s);
cudaError_t launch_adj_stats(const AdjDesc* descs, int n, int M, int N, cudaStream_t s);
cudaError_t launch_adj_final(const AdjDesc* descs, int n, int M, int N, int max_psf,
                             cudaStream_t s);

// Opt every kernel into large dynamic shared memory (once per process/device).
cudaError_t configure_kernels();

}  // namespace gfd
