// Guided filter u = guidfilter(u_I, u_p, w, eps) (Sec. 2, Eq. 3-5) with
// periodic windows, streamed down column strips.
//
// A work item is a strip of W output columns and H output rows of one image.
// With r = (w-1)/2 the block streams the H + 4r input rows of the strip's
// W + 4r input columns (periodic wrap) through a ring buffer in shared
// memory, GF_RB rows per batch, the next batch being copied asynchronously
// while the current one is processed:
//   1. window sums down each column of I-c_I, p-c_p, their squares and
//      product (running sums, Kahan-compensated);
//   2. window sums along each row of those -> mu_k, pbar_k, sigma_k^2 and
//      the covariance -> a_k (Eq. 3), b_k (Eq. 4), into a ring of (a, b) rows;
//   3. running window sums of a and b down each column (compensated);
//   4. window sums along each row -> abar, bbar -> u = abar I + bbar (Eq. 5).
// Every sum costs O(1) per pixel, independent of w (the O(N^2) exact box
// filter the paper relies on).  Window statistics are taken about reference
// values (c_I, c_p: the item's centre pixel), which removes the cancellation
// in sigma_k^2 = E[I^2] - mu^2 where the window mean is close to c_I.
#include "common.cuh"
#include "launch.h"

namespace gfd {

constexpr int GF_W = 128;      // output columns per item (at most N)
constexpr int GF_H = 128;      // output rows per item (at most M)
constexpr int GF_RB = 8;       // input rows per batch
constexpr int GF_C = 8;        // columns per thread in the row sums
constexpr int GF_THREADS = 256;
constexpr int GF_RMAX = 8;     // w <= 17

// Row pitches are 1 (mod 32) so that rows fall on consecutive banks.
GFD_HD int gf_pitch(int w) { return ((w + 30) / 32) * 32 + 1; }
GFD_HD int gf_rin(int rad) { return 2 * GF_RB + 2 * rad + 1; }
GFD_HD int gf_rab(int rad) { return GF_RB + 2 * rad + 1; }
GFD_HD size_t gf_smem_floats(int rad) {
  const int Wp = gf_pitch(GF_W + 4 * rad), W1p = gf_pitch(GF_W + 2 * rad);
  return (size_t)2 * gf_rin(rad) * Wp + (size_t)4 * GF_RB * Wp + (size_t)2 * gf_rab(rad) * W1p +
         (size_t)2 * GF_RB * W1p;
}

struct Kahan {
  float s, c;
};
GFD_D void kadd(Kahan& k, float x) {
  const float y = x - k.c;
  const float t = k.s + y;
  k.c = (t - k.s) - y;
  k.s = t;
}
GFD_D float kval(const Kahan& k) { return k.s - k.c; }

GFD_D void cp_async4(void* smem_dst, const void* gsrc) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(smem_u32(smem_dst)), "l"(gsrc)
               : "memory");
}

// Shared-memory arrays, plane-major, rows of pitch Wp (input columns) or
// W1p (columns of a, b).  The row-sum stages give lane l the batch row
// l % GF_RB and a run of GF_C columns, so a warp touches 8 rows x 4 runs at
// distinct banks.
template <int RAD>
struct GfLayout {
  static constexpr int WIN = 2 * RAD + 1;
  static constexpr int Wp = ((GF_W + 4 * RAD + 30) / 32) * 32 + 1;
  static constexpr int W1p = ((GF_W + 2 * RAD + 30) / 32) * 32 + 1;
  static constexpr int Rin = 2 * GF_RB + 2 * RAD + 1;
  static constexpr int Rab = GF_RB + 2 * RAD + 1;
  float* in;   // [2][Rin][Wp]   input rows (I, p), ring
  float* vs;   // [4][RB][Wp]    column window sums of the batch rows
  float* ab;   // [2][Rab][W1p]  a, b rows, ring
  float* vs2;  // [2][RB][W1p]   column window sums of a, b
  GFD_D explicit GfLayout(float* sm) {
    in = sm;
    vs = in + 2 * Rin * Wp;
    ab = vs + 4 * GF_RB * Wp;
    vs2 = ab + 2 * Rab * W1p;
  }
};

template <int RAD>
GFD_D void gf_items(const ClassDesc& cd, const ImgDesc* __restrict__ imgs, ImgState* st, int iter,
                    bool shifted, int W, int H, float* sm, double* red, int* s_flag) {
  using Lay = GfLayout<RAD>;
  constexpr int WIN = Lay::WIN, Wp = Lay::Wp, W1p = Lay::W1p, Rin = Lay::Rin, Rab = Lay::Rab;
  const Lay L(sm);
  const int M = cd.M, N = cd.N;
  const int tid = threadIdx.x;
  const int strips = N / W, blocks = M / H;
  const int per_img = strips * blocks;
  const int n_items = cd.n_img * per_img;
  const int nrows = H + 4 * RAD;  // input rows of an item
  const int nq = (nrows + GF_RB - 1) / GF_RB;
  const int win_used = W + 4 * RAD, w1_used = W + 2 * RAD;
  const float inv_n = 1.0f / (float)(WIN * WIN);

  // Input row y of an item whose row 0 has stream index `base` lives in ring
  // slot (base + y) % Rin; consecutive items continue the stream, so the next
  // item's first batch can be fetched during the current item's last one.
  auto prefetch = [&](int item, int q, int base) {
    if (item < n_items) {
      const int li = item / per_img, rem = item - li * per_img;
      const int y0 = (rem / strips) * H, x0 = (rem % strips) * W;
      const ImgDesc& d = imgs[cd.img0 + li];
      const int r0 = q * GF_RB;
      const int rows = min(GF_RB, nrows - r0);
      for (int e = tid; e < 2 * rows * win_used; e += blockDim.x) {
        const int plane = e / (rows * win_used);
        const int rr = e - plane * rows * win_used;
        const int row = rr / win_used, c = rr - row * win_used;
        const int gy = (y0 - 2 * RAD + r0 + row) & (M - 1);
        const int gx = (x0 - 2 * RAD + c) & (N - 1);
        const float* src = (plane == 0 ? d.uI : d.up) + (size_t)gy * N + gx;
        cp_async4(L.in + (plane * Rin + (base + r0 + row) % Rin) * Wp + c, src);
      }
    }
    cp_async_commit();
  };

  int item = blockIdx.x;
  int base = 0;  // stream index of the current item's input row 0
  prefetch(item, 0, base);
  while (item < n_items) {
    const int li = item / per_img, rem = item - li * per_img;
    const int y0 = (rem / strips) * H, x0 = (rem % strips) * W;
    const int gi = cd.img0 + li;
    const ImgDesc& d = imgs[gi];
    const float* uo = (iter >= 0 && d.isnr_out) ? d.uo : nullptr;
    float cI = 0.0f, cP = 0.0f;
    if (shifted) {
      const size_t c = (size_t)((y0 + H / 2) & (M - 1)) * N + ((x0 + W / 2) & (N - 1));
      cI = __ldg(&d.uI[c]);
      cP = __ldg(&d.up[c]);
    }
    const float eps = (float)d.eps;
    Kahan sJ{0, 0}, sQ{0, 0}, sJJ{0, 0}, sJQ{0, 0}, sa{0, 0}, sb{0, 0};
    float err = 0.0f;
    const int next_base = base + nq * GF_RB;
    for (int q = 0; q < nq; ++q) {
      cp_async_wait<0>();
      __syncthreads();
      if (q + 1 < nq)
        prefetch(item, q + 1, base);
      else
        prefetch(item + gridDim.x, 0, next_base);
      const int r0 = q * GF_RB;
      const int rows = min(GF_RB, nrows - r0);
      // 1. column window sums of the four statistics (input column tid)
      if (tid < win_used) {
        for (int rho = 0; rho < rows; ++rho) {
          const int y = r0 + rho;
          const float* rn = L.in + ((base + y) % Rin) * Wp;
          const float J = rn[tid] - cI, Q = rn[Rin * Wp + tid] - cP;
          kadd(sJ, J);
          kadd(sQ, Q);
          kadd(sJJ, J * J);
          kadd(sJQ, J * Q);
          if (y >= WIN) {
            const float* ro = L.in + ((base + y - WIN) % Rin) * Wp;
            const float Jo = ro[tid] - cI, Qo = ro[Rin * Wp + tid] - cP;
            kadd(sJ, -Jo);
            kadd(sQ, -Qo);
            kadd(sJJ, -(Jo * Jo));
            kadd(sJQ, -(Jo * Qo));
          }
          if (y >= 2 * RAD) {
            float* v = L.vs + rho * Wp;
            constexpr int PS = GF_RB * Wp;  // plane stride
            v[tid] = kval(sJ);
            v[PS + tid] = kval(sQ);
            v[2 * PS + tid] = kval(sJJ);
            v[3 * PS + tid] = kval(sJQ);
          }
        }
      }
      __syncthreads();
      // 2. row window sums -> a_k (Eq. 3), b_k (Eq. 4) for stage-1 row y - r
      {
        const int runs = (w1_used + GF_C - 1) / GF_C;
        constexpr int PS = GF_RB * Wp;
        for (int u = tid; u < GF_RB * runs; u += blockDim.x) {
          const int rho = u % GF_RB, run = u / GF_RB;
          const int y = r0 + rho;
          if (rho >= rows || y < 2 * RAD) continue;
          const float* v = L.vs + rho * Wp;
          const int c0 = run * GF_C, c1 = min(c0 + GF_C, w1_used);
          float s0 = 0.f, s1 = 0.f, s2 = 0.f, s3 = 0.f;
#pragma unroll
          for (int dd = 0; dd < WIN; ++dd) {
            s0 += v[c0 + dd];
            s1 += v[PS + c0 + dd];
            s2 += v[2 * PS + c0 + dd];
            s3 += v[3 * PS + c0 + dd];
          }
          float* abr = L.ab + ((base + y) % Rab) * W1p;
          for (int c = c0; c < c1; ++c) {
            if (c > c0) {
              s0 += v[c + 2 * RAD] - v[c - 1];
              s1 += v[PS + c + 2 * RAD] - v[PS + c - 1];
              s2 += v[2 * PS + c + 2 * RAD] - v[2 * PS + c - 1];
              s3 += v[3 * PS + c + 2 * RAD] - v[3 * PS + c - 1];
            }
            const float mJ = s0 * inv_n, mQ = s1 * inv_n;
            const float var = fmaf(-mJ, mJ, s2 * inv_n);  // sigma_k^2
            const float cov = fmaf(-mJ, mQ, s3 * inv_n);  // mean(I p) - mu pbar
            const float a = cov / (var + eps);
            abr[c] = a;
            abr[Rab * W1p + c] = (mQ + cP) - a * (mJ + cI);
          }
        }
      }
      __syncthreads();
      // 3. column window sums of a and b (column tid of the a, b rows)
      if (tid < w1_used) {
        for (int rho = 0; rho < rows; ++rho) {
          const int y = r0 + rho;
          if (y < 2 * RAD) continue;
          const float* an = L.ab + ((base + y) % Rab) * W1p;
          kadd(sa, an[tid]);
          kadd(sb, an[Rab * W1p + tid]);
          if (y >= 2 * RAD + WIN) {
            const float* ao = L.ab + ((base + y - WIN) % Rab) * W1p;
            kadd(sa, -ao[tid]);
            kadd(sb, -ao[Rab * W1p + tid]);
          }
          if (y >= 4 * RAD) {
            float* v2 = L.vs2 + rho * W1p;
            v2[tid] = kval(sa);
            v2[GF_RB * W1p + tid] = kval(sb);
          }
        }
      }
      __syncthreads();
      // 4. row window sums -> u = abar I + bbar (Eq. 5) for output row y - 4r
      {
        const int runs = W / GF_C;
        constexpr int PS2 = GF_RB * W1p;
        for (int u = tid; u < GF_RB * runs; u += blockDim.x) {
          const int rho = u % GF_RB, run = u / GF_RB;
          const int y = r0 + rho;
          if (rho >= rows || y < 4 * RAD) continue;
          const float* v2 = L.vs2 + rho * W1p;
          const float* ri = L.in + ((base + y - 2 * RAD) % Rin) * Wp;
          const int x0r = run * GF_C;
          float sa_ = 0.f, sb_ = 0.f;
#pragma unroll
          for (int dd = 0; dd < WIN; ++dd) {
            sa_ += v2[x0r + dd];
            sb_ += v2[PS2 + x0r + dd];
          }
          const int gy = (y0 + y - 4 * RAD) & (M - 1);
          float* urow = d.u + (size_t)gy * N;
          const float* orow = uo ? uo + (size_t)gy * N : nullptr;
#pragma unroll
          for (int c = 0; c < GF_C; ++c) {
            const int x = x0r + c;
            if (c > 0) {
              sa_ += v2[x + 2 * RAD] - v2[x - 1];
              sb_ += v2[PS2 + x + 2 * RAD] - v2[PS2 + x - 1];
            }
            const float val = fmaf(sa_ * inv_n, ri[x + 2 * RAD], sb_ * inv_n);
            const int gx = (x0 + x) & (N - 1);
            urow[gx] = val;
            if (orow) {
              const float e = val - __ldg(&orow[gx]);
              err = fmaf(e, e, err);
            }
          }
        }
      }
    }
    if (uo) {
      // ||u - u_orig||^2 of this item (FP32 in a warp, FP64 across warps)
      err = warp_sum(err);
      if ((tid & 31) == 0) red[tid >> 5] = (double)err;
      __syncthreads();
      ImgState* S = st + gi;
      if (tid == 0) {
        double s = 0.0;
        for (int w = 0; w < num_warps(); ++w) s += red[w];
        atomicAdd(&S->err2, s);
        __threadfence();
        const unsigned int prev = atomicAdd(&S->gf_done, 1u);
        *s_flag = (prev == (unsigned)per_img - 1);
      }
      __syncthreads();
      if (*s_flag && tid == 0) {
        __threadfence();
        const double e2 = __ldcg(&S->err2);
        d.isnr_out[iter] = 10.0 * log10(S->den_isnr / e2);
        S->err2 = 0.0;
        S->gf_done = 0;
        __threadfence();
      }
    }
    base = next_base;
    item += gridDim.x;
  }
  cp_async_wait<0>();
}

__global__ void __launch_bounds__(GF_THREADS)
k_guided_filter(ClassDesc cd, const ImgDesc* __restrict__ imgs, ImgState* st, int iter,
                int plain_var, int rad, int W, int H) {
  extern __shared__ __align__(16) float gsm[];
  __shared__ double red[GF_THREADS / 32];
  __shared__ int s_flag;
  const bool shifted = plain_var == 0;
  switch (rad) {
    case 0: gf_items<0>(cd, imgs, st, iter, shifted, W, H, gsm, red, &s_flag); break;
    case 1: gf_items<1>(cd, imgs, st, iter, shifted, W, H, gsm, red, &s_flag); break;
    case 2: gf_items<2>(cd, imgs, st, iter, shifted, W, H, gsm, red, &s_flag); break;
    case 3: gf_items<3>(cd, imgs, st, iter, shifted, W, H, gsm, red, &s_flag); break;
    case 4: gf_items<4>(cd, imgs, st, iter, shifted, W, H, gsm, red, &s_flag); break;
    case 5: gf_items<5>(cd, imgs, st, iter, shifted, W, H, gsm, red, &s_flag); break;
    case 6: gf_items<6>(cd, imgs, st, iter, shifted, W, H, gsm, red, &s_flag); break;
    case 7: gf_items<7>(cd, imgs, st, iter, shifted, W, H, gsm, red, &s_flag); break;
    default: gf_items<8>(cd, imgs, st, iter, shifted, W, H, gsm, red, &s_flag); break;
  }
}

static int gf_sm_count() {
  static int n = 0;
  if (n == 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n <= 0) n = 1;
  }
  return n;
}

// One launch per window radius present in the class (the images of a class
// are ordered by radius, so each group is a contiguous range).
cudaError_t launch_guided_filter(const ClassLaunch& c, int iter, int plain_var, cudaStream_t s) {
  const int W = c.cd.N < GF_W ? c.cd.N : GF_W;
  const int H = c.cd.M < GF_H ? c.cd.M : GF_H;
  for (int g = 0; g < c.n_rad_groups; ++g) {
    const RadGroup& rg = c.rad_groups[g];
    ClassDesc cd = c.cd;
    cd.img0 = rg.img0;
    cd.n_img = rg.n_img;
    const size_t smem = gf_smem_floats(rg.rad) * sizeof(float);
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_guided_filter, GF_THREADS, smem) !=
            cudaSuccess || per_sm < 1)
      per_sm = 1;
    const int n_items = cd.n_img * (cd.N / W) * (cd.M / H);
    int grid = per_sm * gf_sm_count();
    if (grid > n_items) grid = n_items;
    k_guided_filter<<<grid, GF_THREADS, smem, s>>>(cd, c.imgs, c.st, iter, plain_var, rg.rad, W, H);
  }
  return cudaGetLastError();
}

cudaError_t configure_gf_kernel() {
  return cudaFuncSetAttribute(k_guided_filter, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)(gf_smem_floats(GF_RMAX) * sizeof(float)));
}

}  // namespace gfd
