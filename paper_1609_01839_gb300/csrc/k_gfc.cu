// Guided filter with a colour guidance image (the paper notes the guided
// filter serves colour as well as grey-scale images, Sec. 3.1): guidance I
// with 3 channels (planar [3][M][N]), filtering input p.  Per window k,
//   a_k = (Sigma_k + eps U)^-1 (mean_k(I p) - mu_k pbar_k)   (3-vector, Eq. 3)
//   b_k = pbar_k - a_k . mu_k                                 (Eq. 4)
//   u   = abar . I + bbar                                     (Eq. 5)
// with mu_k, Sigma_k the window mean and covariance of I.
//
// Two tiled passes, each a TILE x TILE block of output pixels whose input
// tile plus an r-pixel halo is staged in shared memory:
//   1. the 13 window sums (I_c, p, I_c I_d, I_c p) by separable sums (along
//      rows into a shared [rows][TILE][13] array, then down its columns) in
//      FP64 (inputs are FP32; products and sums of up to 289 terms are exact
//      to ~1e-16), the 3 x 3 solve by Cramer's rule in FP64 -> a, b planes;
//   2. the window sums of a and b (FP64) -> u.
// Windows are periodic or truncated at the canvas edge (means over the
// pixels inside).  The FP64 work is a few hundred operations per pixel,
// well below this part's FP64 rate for the sizes served.
#include "common.cuh"
#include "launch.h"

namespace gfd {

constexpr int CGF_TILE = 16;
constexpr int CGF_RMAX = 8;

// Shared layout of pass 1 (rad r): input tile [4][T+2r][T+2r] floats, row
// sums [T+2r][T][13] doubles.
GFD_HD size_t cgf_smem1(int rad) {
  const int E = CGF_TILE + 2 * rad;
  return (size_t)E * CGF_TILE * 13 * sizeof(double) + (size_t)4 * E * E * sizeof(float);
}
// pass 2: input tile [4][T+2r][T+2r] floats (a_r, a_g, a_b, b), row sums
// [T+2r][T][4] doubles.
GFD_HD size_t cgf_smem2(int rad) {
  const int E = CGF_TILE + 2 * rad;
  return (size_t)E * CGF_TILE * 4 * sizeof(double) + (size_t)4 * E * E * sizeof(float);
}

// Canvas index of tile coordinate v (may lie outside [0, L)); -1 when the
// window is truncated there.
GFD_D int cgf_wrap(int v, int L, bool trunc) {
  if (trunc) return (v >= 0 && v < L) ? v : -1;
  return v & (L - 1);
}

GFD_D int cgf_count(int x, int L, int rad) {
  const int a = x - rad < 0 ? 0 : x - rad;
  const int b = x + rad > L - 1 ? L - 1 : x + rad;
  return b - a + 1;
}

// Stage an E x E tile of 4 planes (origin (y0 - rad, x0 - rad)) into s[4][E][E];
// out-of-canvas pixels of truncated windows are zero.
GFD_D void cgf_stage(float* s, const float* const* planes, int M, int N, int y0, int x0, int rad,
                     bool trunc) {
  const int E = CGF_TILE + 2 * rad;
  for (int e = threadIdx.x; e < E * E; e += blockDim.x) {
    const int ty = e / E, tx = e - ty * E;
    const int gy = cgf_wrap(y0 - rad + ty, M, trunc), gx = cgf_wrap(x0 - rad + tx, N, trunc);
    const bool in = gy >= 0 && gx >= 0;
    const size_t off = in ? (size_t)gy * N + gx : 0;
#pragma unroll
    for (int c = 0; c < 4; ++c) s[c * E * E + e] = in ? __ldg(&planes[c][off]) : 0.0f;
  }
}

// Pass 1: window statistics and the 3 x 3 solve of Eq. 3; a (3 planes) and b.
__global__ void __launch_bounds__(CGF_TILE * CGF_TILE)
k_cgf_ab(const float* __restrict__ I, const float* __restrict__ p, int M, int N, int rad,
         double eps, int trunc_i, float* __restrict__ ab) {
  extern __shared__ __align__(16) unsigned char cgf_sm[];
  const bool trunc = trunc_i != 0;
  const int E = CGF_TILE + 2 * rad;
  double* rows = reinterpret_cast<double*>(cgf_sm);                        // [E][T][13]
  float* tile = reinterpret_cast<float*>(rows + (size_t)E * CGF_TILE * 13);  // [4][E][E]
  const size_t P = (size_t)M * N;
  const int x0 = blockIdx.x * CGF_TILE, y0 = blockIdx.y * CGF_TILE;
  const float* planes[4] = {I, I + P, I + 2 * P, p};
  cgf_stage(tile, planes, M, N, y0, x0, rad, trunc);
  __syncthreads();
  // row sums: every tile row e and output column tx, 13 quantities
  for (int e = threadIdx.x; e < E * CGF_TILE; e += blockDim.x) {
    const int ty = e / CGF_TILE, tx = e - ty * CGF_TILE;
    double s[13];
#pragma unroll
    for (int q = 0; q < 13; ++q) s[q] = 0.0;
    for (int dx = 0; dx <= 2 * rad; ++dx) {
      const int o = ty * E + tx + dx;
      const double r = tile[o], g = tile[E * E + o], b = tile[2 * E * E + o];
      const double v = tile[3 * E * E + o];
      s[0] += r; s[1] += g; s[2] += b; s[3] += v;
      s[4] += r * r; s[5] += r * g; s[6] += r * b; s[7] += g * g; s[8] += g * b; s[9] += b * b;
      s[10] += r * v; s[11] += g * v; s[12] += b * v;
    }
#pragma unroll
    for (int q = 0; q < 13; ++q) rows[(size_t)e * 13 + q] = s[q];
  }
  __syncthreads();
  const int tx = threadIdx.x % CGF_TILE, ty = threadIdx.x / CGF_TILE;
  const int gy = y0 + ty, gx = x0 + tx;
  double S[13];
#pragma unroll
  for (int q = 0; q < 13; ++q) S[q] = 0.0;
  for (int dy = 0; dy <= 2 * rad; ++dy) {
    const double* rr = rows + ((size_t)(ty + dy) * CGF_TILE + tx) * 13;
#pragma unroll
    for (int q = 0; q < 13; ++q) S[q] += rr[q];
  }
  const double n = trunc ? (double)cgf_count(gy, M, rad) * cgf_count(gx, N, rad)
                         : (double)((2 * rad + 1) * (2 * rad + 1));
  const double in = 1.0 / n;
  const double mr = S[0] * in, mg = S[1] * in, mb = S[2] * in, mp = S[3] * in;
  // Sigma + eps U (symmetric) and the covariance of I with p
  const double c00 = S[4] * in - mr * mr + eps, c01 = S[5] * in - mr * mg, c02 = S[6] * in - mr * mb;
  const double c11 = S[7] * in - mg * mg + eps, c12 = S[8] * in - mg * mb;
  const double c22 = S[9] * in - mb * mb + eps;
  const double vr = S[10] * in - mr * mp, vg = S[11] * in - mg * mp, vb = S[12] * in - mb * mp;
  // Cramer's rule on the positive-definite 3 x 3 system
  const double m00 = c11 * c22 - c12 * c12, m01 = c02 * c12 - c01 * c22, m02 = c01 * c12 - c02 * c11;
  const double det = c00 * m00 + c01 * m01 + c02 * m02;
  const double m11 = c00 * c22 - c02 * c02, m12 = c01 * c02 - c00 * c12;
  const double m22 = c00 * c11 - c01 * c01;
  const double id = 1.0 / det;
  const double ar = (m00 * vr + m01 * vg + m02 * vb) * id;
  const double ag = (m01 * vr + m11 * vg + m12 * vb) * id;
  const double ab_ = (m02 * vr + m12 * vg + m22 * vb) * id;
  const double bb = mp - (ar * mr + ag * mg + ab_ * mb);
  if (gy < M && gx < N) {
    const size_t o = (size_t)gy * N + gx;
    ab[o] = (float)ar;
    ab[P + o] = (float)ag;
    ab[2 * P + o] = (float)ab_;
    ab[3 * P + o] = (float)bb;
  }
}

// Pass 2: window means of a and b, u = abar . I + bbar (Eq. 5).
__global__ void __launch_bounds__(CGF_TILE * CGF_TILE)
k_cgf_out(const float* __restrict__ I, const float* __restrict__ ab, int M, int N, int rad,
          int trunc_i, float* __restrict__ u) {
  extern __shared__ __align__(16) unsigned char cgf_sm[];
  const bool trunc = trunc_i != 0;
  const int E = CGF_TILE + 2 * rad;
  double* rows = reinterpret_cast<double*>(cgf_sm);                       // [E][T][4]
  float* tile = reinterpret_cast<float*>(rows + (size_t)E * CGF_TILE * 4);  // [4][E][E]
  const size_t P = (size_t)M * N;
  const int x0 = blockIdx.x * CGF_TILE, y0 = blockIdx.y * CGF_TILE;
  const float* planes[4] = {ab, ab + P, ab + 2 * P, ab + 3 * P};
  cgf_stage(tile, planes, M, N, y0, x0, rad, trunc);
  __syncthreads();
  for (int e = threadIdx.x; e < E * CGF_TILE; e += blockDim.x) {
    const int ty = e / CGF_TILE, tx = e - ty * CGF_TILE;
    double s[4] = {0.0, 0.0, 0.0, 0.0};
    for (int dx = 0; dx <= 2 * rad; ++dx) {
      const int o = ty * E + tx + dx;
#pragma unroll
      for (int c = 0; c < 4; ++c) s[c] += tile[c * E * E + o];
    }
#pragma unroll
    for (int c = 0; c < 4; ++c) rows[(size_t)e * 4 + c] = s[c];
  }
  __syncthreads();
  const int tx = threadIdx.x % CGF_TILE, ty = threadIdx.x / CGF_TILE;
  const int gy = y0 + ty, gx = x0 + tx;
  if (gy >= M || gx >= N) return;
  double S[4] = {0.0, 0.0, 0.0, 0.0};
  for (int dy = 0; dy <= 2 * rad; ++dy) {
    const double* rr = rows + ((size_t)(ty + dy) * CGF_TILE + tx) * 4;
#pragma unroll
    for (int c = 0; c < 4; ++c) S[c] += rr[c];
  }
  const double n = trunc ? (double)cgf_count(gy, M, rad) * cgf_count(gx, N, rad)
                         : (double)((2 * rad + 1) * (2 * rad + 1));
  const size_t o = (size_t)gy * N + gx;
  const double v = S[0] * __ldg(&I[o]) + S[1] * __ldg(&I[P + o]) + S[2] * __ldg(&I[2 * P + o]) + S[3];
  u[o] = (float)(v / n);
}

cudaError_t launch_guided_filter_color(const float* I, const float* p, int M, int N, int w,
                                       double eps, int boundary, float* ab, float* u,
                                       cudaStream_t s) {
  const int rad = (w - 1) / 2;
  const dim3 grid((N + CGF_TILE - 1) / CGF_TILE, (M + CGF_TILE - 1) / CGF_TILE);
  const int trunc = boundary == GFD_BOUNDARY_TRUNCATED ? 1 : 0;
  k_cgf_ab<<<grid, CGF_TILE * CGF_TILE, cgf_smem1(rad), s>>>(I, p, M, N, rad, eps, trunc, ab);
  k_cgf_out<<<grid, CGF_TILE * CGF_TILE, cgf_smem2(rad), s>>>(I, ab, M, N, rad, trunc, u);
  return cudaGetLastError();
}

cudaError_t configure_gfc_kernels() {
  cudaError_t e = cudaFuncSetAttribute(k_cgf_ab, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)cgf_smem1(CGF_RMAX));
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(k_cgf_out, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)cgf_smem2(CGF_RMAX));
}

}  // namespace gfd
