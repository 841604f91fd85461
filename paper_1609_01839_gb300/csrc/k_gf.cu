// Guided filter u = guidfilter(u_I, u_p, w, eps) (Sec. 2, Eq. 3-5), periodic
// windows, one 32 x 32 output tile per block.
//
// With r = (w-1)/2 the block loads the (32+4r)^2 input tile (periodic wrap),
// forms the window sums of I, p, I*I and I*p over the (32+2r)^2 pixels whose
// coefficients the tile needs (separable: column sums, then row sums, each a
// sliding window), computes a_k (Eq. 3) and b_k (Eq. 4) there, and then the
// window means of a and b over the tile to give u = abar I + bbar (Eq. 5).
// The cost per pixel does not depend on w (the O(N^2) exact box filter the
// paper relies on).
//
// Window statistics are taken about a per-tile reference value (the guidance
// and input at the tile centre): sigma_k^2 = E[(I-c)^2] - (E[I]-c)^2 is the
// same number as E[I^2] - mu^2 but without its cancellation where the window
// mean is close to c.
#include "common.cuh"
#include "launch.h"

namespace gfd {

constexpr int GF_T = 32;        // tile edge
constexpr int GF_THREADS = 256;
constexpr int GF_SEG = 8;       // sliding run length
constexpr int GF_RMAX = 8;      // w <= 17

GFD_HD int gf_pitch(int w) { return w | 1; }
GFD_HD size_t gf_smem_floats(int rad) {
  const int H0 = GF_T + 4 * rad, W0 = H0, H1 = GF_T + 2 * rad, W1 = H1;
  const int P0 = gf_pitch(W0), P1 = gf_pitch(W1);
  return (size_t)2 * H0 * P0 + (size_t)4 * H1 * P0 + (size_t)2 * H1 * P1;
}

template <int RAD>
GFD_D void gf_tile(const float* __restrict__ I, const float* __restrict__ p, float* __restrict__ u,
                   const float* __restrict__ uo, int M, int N, int y0, int x0, float eps,
                   bool shifted, float* sm, float& err) {
  constexpr int WIN = 2 * RAD + 1;
  constexpr int H0 = GF_T + 4 * RAD, W0 = H0, H1 = GF_T + 2 * RAD, W1 = H1;
  constexpr int P0 = W0 | 1, P1 = W1 | 1;
  float* sI = sm;
  float* sP = sI + H0 * P0;
  float* vJ = sP + H0 * P0;
  float* vQ = vJ + H1 * P0;
  float* vJJ = vQ + H1 * P0;
  float* vJQ = vJJ + H1 * P0;
  float* sA = vJQ + H1 * P0;
  float* sB = sA + H1 * P1;
  float* va = vJJ;  // stage-2 column sums reuse dead stage-1 storage
  float* vb = vJQ;
  float* so = sA;   // output tile reuses sA after stage 2's column sums
  const int tid = threadIdx.x;
  const float inv_n = 1.0f / (float)(WIN * WIN);

  float cI = 0.0f, cP = 0.0f;
  if (shifted) {
    const size_t c = (size_t)((y0 + GF_T / 2) & (M - 1)) * N + ((x0 + GF_T / 2) & (N - 1));
    cI = __ldg(&I[c]);
    cP = __ldg(&p[c]);
  }
  for (int idx = tid; idx < H0 * W0; idx += GF_THREADS) {
    const int ty = idx / W0, tx = idx - ty * W0;
    const size_t g = (size_t)((y0 - 2 * RAD + ty) & (M - 1)) * N + ((x0 - 2 * RAD + tx) & (N - 1));
    sI[ty * P0 + tx] = __ldg(&I[g]);
    sP[ty * P0 + tx] = __ldg(&p[g]);
  }
  __syncthreads();

  // stage 1, column sums of J = I - cI, Q = p - cP, J*J, J*Q over WIN rows
  constexpr int NS1 = (H1 + GF_SEG - 1) / GF_SEG;
  for (int item = tid; item < W0 * NS1; item += GF_THREADS) {
    const int x = item % W0, sg = item / W0;
    const int oy0 = sg * GF_SEG;
    const int oy1 = min(oy0 + GF_SEG, H1);
    float sj = 0.f, sq = 0.f, sjj = 0.f, sjq = 0.f;
#pragma unroll
    for (int dd = 0; dd < WIN; ++dd) {
      const float J = sI[(oy0 + dd) * P0 + x] - cI, Q = sP[(oy0 + dd) * P0 + x] - cP;
      sj += J;
      sq += Q;
      sjj = fmaf(J, J, sjj);
      sjq = fmaf(J, Q, sjq);
    }
    vJ[oy0 * P0 + x] = sj;
    vQ[oy0 * P0 + x] = sq;
    vJJ[oy0 * P0 + x] = sjj;
    vJQ[oy0 * P0 + x] = sjq;
    for (int oy = oy0 + 1; oy < oy1; ++oy) {
      const float Jn = sI[(oy + 2 * RAD) * P0 + x] - cI, Qn = sP[(oy + 2 * RAD) * P0 + x] - cP;
      const float Jo = sI[(oy - 1) * P0 + x] - cI, Qo = sP[(oy - 1) * P0 + x] - cP;
      sj += Jn - Jo;
      sq += Qn - Qo;
      sjj += fmaf(Jn, Jn, -Jo * Jo);
      sjq += fmaf(Jn, Qn, -Jo * Qo);
      vJ[oy * P0 + x] = sj;
      vQ[oy * P0 + x] = sq;
      vJJ[oy * P0 + x] = sjj;
      vJQ[oy * P0 + x] = sjq;
    }
  }
  __syncthreads();

  // stage 1, row sums -> a_k (Eq. 3), b_k (Eq. 4)
  constexpr int NSW1 = (W1 + GF_SEG - 1) / GF_SEG;
  for (int item = tid; item < H1 * NSW1; item += GF_THREADS) {
    const int oy = item % H1, sg = item / H1;
    const int ox0 = sg * GF_SEG;
    const int ox1 = min(ox0 + GF_SEG, W1);
    const float* rJ = vJ + oy * P0;
    const float* rQ = vQ + oy * P0;
    const float* rJJ = vJJ + oy * P0;
    const float* rJQ = vJQ + oy * P0;
    float sj = 0.f, sq = 0.f, sjj = 0.f, sjq = 0.f;
#pragma unroll
    for (int dd = 0; dd < WIN; ++dd) {
      sj += rJ[ox0 + dd];
      sq += rQ[ox0 + dd];
      sjj += rJJ[ox0 + dd];
      sjq += rJQ[ox0 + dd];
    }
    for (int ox = ox0; ox < ox1; ++ox) {
      if (ox > ox0) {
        sj += rJ[ox + 2 * RAD] - rJ[ox - 1];
        sq += rQ[ox + 2 * RAD] - rQ[ox - 1];
        sjj += rJJ[ox + 2 * RAD] - rJJ[ox - 1];
        sjq += rJQ[ox + 2 * RAD] - rJQ[ox - 1];
      }
      const float mJ = sj * inv_n, mQ = sq * inv_n;
      const float var = fmaf(-mJ, mJ, sjj * inv_n);   // sigma_k^2
      const float cov = fmaf(-mJ, mQ, sjq * inv_n);   // mean(I p) - mu pbar
      const float a = cov / (var + eps);
      const float b = (mQ + cP) - a * (mJ + cI);
      sA[oy * P1 + ox] = a;
      sB[oy * P1 + ox] = b;
    }
  }
  __syncthreads();

  // stage 2, column sums of a and b over WIN rows
  constexpr int NS2 = (GF_T + GF_SEG - 1) / GF_SEG;
  for (int item = tid; item < W1 * NS2; item += GF_THREADS) {
    const int x = item % W1, sg = item / W1;
    const int oy0 = sg * GF_SEG;
    const int oy1 = min(oy0 + GF_SEG, GF_T);
    float s_a = 0.f, s_b = 0.f;
#pragma unroll
    for (int dd = 0; dd < WIN; ++dd) {
      s_a += sA[(oy0 + dd) * P1 + x];
      s_b += sB[(oy0 + dd) * P1 + x];
    }
    va[oy0 * P1 + x] = s_a;
    vb[oy0 * P1 + x] = s_b;
    for (int oy = oy0 + 1; oy < oy1; ++oy) {
      s_a += sA[(oy + 2 * RAD) * P1 + x] - sA[(oy - 1) * P1 + x];
      s_b += sB[(oy + 2 * RAD) * P1 + x] - sB[(oy - 1) * P1 + x];
      va[oy * P1 + x] = s_a;
      vb[oy * P1 + x] = s_b;
    }
  }
  __syncthreads();

  // stage 2, row sums -> u = abar I + bbar (Eq. 5)
  constexpr int NSW2 = (GF_T + GF_SEG - 1) / GF_SEG;
  for (int item = tid; item < GF_T * NSW2; item += GF_THREADS) {
    const int ty = item % GF_T, sg = item / GF_T;
    const int tx0 = sg * GF_SEG;
    const float* ra = va + ty * P1;
    const float* rb = vb + ty * P1;
    float s_a = 0.f, s_b = 0.f;
#pragma unroll
    for (int dd = 0; dd < WIN; ++dd) {
      s_a += ra[tx0 + dd];
      s_b += rb[tx0 + dd];
    }
    for (int tx = tx0; tx < tx0 + GF_SEG; ++tx) {
      if (tx > tx0) {
        s_a += ra[tx + 2 * RAD] - ra[tx - 1];
        s_b += rb[tx + 2 * RAD] - rb[tx - 1];
      }
      const float Iv = sI[(ty + 2 * RAD) * P0 + tx + 2 * RAD];
      so[ty * GF_T + tx] = fmaf(s_a * inv_n, Iv, s_b * inv_n);
    }
  }
  __syncthreads();
  for (int idx = tid; idx < GF_T * GF_T; idx += GF_THREADS) {
    const int ty = idx / GF_T, tx = idx - ty * GF_T;
    const int gy = y0 + ty, gx = x0 + tx;
    if (gy < M && gx < N) {
      const float v = so[idx];
      u[(size_t)gy * N + gx] = v;
      if (uo) {
        const float e = v - __ldg(&uo[(size_t)gy * N + gx]);
        err = fmaf(e, e, err);
      }
    }
  }
}

__global__ void __launch_bounds__(GF_THREADS)
k_guided_filter(ClassDesc cd, const ImgDesc* __restrict__ imgs, ImgState* st, int iter,
                int plain_var) {
  extern __shared__ float gsm[];
  __shared__ double red[GF_THREADS / 32];
  __shared__ int s_flag;
  const int gi = cd.img0 + blockIdx.z;
  const ImgDesc& d = imgs[gi];
  const int M = cd.M, N = cd.N;
  const int y0 = blockIdx.y * GF_T, x0 = blockIdx.x * GF_T;
  const float* I = d.uI;
  const float* p = d.up;
  const float* uo = (iter >= 0 && d.isnr_out) ? d.uo : nullptr;
  const float eps = (float)d.eps;
  const bool shifted = plain_var == 0;
  float err = 0.0f;
  switch ((d.w - 1) / 2) {
    case 0: gf_tile<0>(I, p, d.u, uo, M, N, y0, x0, eps, shifted, gsm, err); break;
    case 1: gf_tile<1>(I, p, d.u, uo, M, N, y0, x0, eps, shifted, gsm, err); break;
    case 2: gf_tile<2>(I, p, d.u, uo, M, N, y0, x0, eps, shifted, gsm, err); break;
    case 3: gf_tile<3>(I, p, d.u, uo, M, N, y0, x0, eps, shifted, gsm, err); break;
    case 4: gf_tile<4>(I, p, d.u, uo, M, N, y0, x0, eps, shifted, gsm, err); break;
    case 5: gf_tile<5>(I, p, d.u, uo, M, N, y0, x0, eps, shifted, gsm, err); break;
    case 6: gf_tile<6>(I, p, d.u, uo, M, N, y0, x0, eps, shifted, gsm, err); break;
    case 7: gf_tile<7>(I, p, d.u, uo, M, N, y0, x0, eps, shifted, gsm, err); break;
    default: gf_tile<8>(I, p, d.u, uo, M, N, y0, x0, eps, shifted, gsm, err); break;
  }
  if (uo == nullptr) return;
  // ||u - u_orig||^2 for the ISNR of this iteration (FP32 in a warp, FP64 across)
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) err += __shfl_xor_sync(0xffffffffu, err, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = (double)err;
  __syncthreads();
  ImgState* S = st + gi;
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int w = 0; w < GF_THREADS / 32; ++w) s += red[w];
    atomicAdd(&S->err2, s);
    __threadfence();
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    const unsigned int nb = gridDim.x * gridDim.y;
    const unsigned int prev = atomicAdd(&S->gf_done, 1u);
    s_flag = (prev == nb - 1);
  }
  __syncthreads();
  if (s_flag && threadIdx.x == 0) {
    __threadfence();
    const double e2 = __ldcg(&S->err2);
    d.isnr_out[iter] = 10.0 * log10(S->den_isnr / e2);
    S->err2 = 0.0;
    S->gf_done = 0;
    __threadfence();
  }
}

cudaError_t launch_guided_filter(const ClassLaunch& c, int iter, int plain_var, cudaStream_t s) {
  const int tx = (c.cd.N + GF_T - 1) / GF_T, ty = (c.cd.M + GF_T - 1) / GF_T;
  const size_t smem = gf_smem_floats(c.max_rad) * sizeof(float);
  k_guided_filter<<<dim3(tx, ty, c.cd.n_img), GF_THREADS, smem, s>>>(c.cd, c.imgs, c.st, iter,
                                                                      plain_var);
  return cudaGetLastError();
}

cudaError_t configure_gf_kernel() {
  return cudaFuncSetAttribute(k_guided_filter, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)(gf_smem_floats(GF_RMAX) * sizeof(float)));
}

}  // namespace gfd
