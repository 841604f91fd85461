// Guided filter u = guidfilter(u_I, u_p, w, eps) (Sec. 2, Eq. 3-5) with
// periodic windows, streamed down column strips.
//
// A work item is a strip of GF_W output columns and H output rows of one
// image.  With r = (w-1)/2 the block streams the H + 4r input rows of the
// strip's input columns (periodic wrap; 16-byte copies of a window that
// starts on a 4-column boundary) through a ring buffer in shared memory,
// GF_RB rows per batch, the next batch being copied asynchronously while the
// current one is processed:
//   1. window sums down each column of J = I - c_I, Q = p - c_p, J^2, J Q;
//   2. window sums along each row of those -> mu_k, pbar_k, sigma_k^2 and
//      the covariance -> a_k (Eq. 3), b_k (Eq. 4), into a ring of (a, b) rows;
//   3. window sums of a and b down each column;
//   4. window sums along each row -> abar, bbar -> u = abar I + bbar (Eq. 5).
// Column sums are formed directly for the first row of each GF_SB-row
// sub-block and slid over the rest (so every stage keeps all threads busy
// and no sum is carried over more than GF_SB - 1 slides); row sums slide over
// runs of GF_C columns.  Window statistics are taken about reference values
// (c_I, c_p: the item's centre pixel), which removes the cancellation in
// sigma_k^2 = E[I^2] - mu^2 where the window mean is close to c_I.  Images
// narrower than GF_W are covered by one strip whose columns wrap; only the
// first N outputs are stored.
#include "common.cuh"
#include "launch.h"

namespace gfd {

constexpr int GF_W = 64;       // output columns per item
constexpr int GF_H = 128;      // output rows per item (at most M)
constexpr int GF_RB = 16;      // input rows per batch
constexpr int GF_SB = 4;       // rows per column-sum sub-block
constexpr int GF_C = 4;        // columns per thread in the row sums
constexpr int GF_THREADS = 256;
constexpr int GF_RMAX = 8;     // w <= 17

// Shared-memory geometry for window radius RAD.  Input rows hold the
// 4-aligned column window [x0 - 4Q, x0 + GF_W + 4Q) (pitch a multiple of 4
// for the 16-byte copies); logical column c (window start x0 - 2r) sits at
// c + OFF.  Rows of the sums have odd pitches.
template <int RAD>
struct GfGeom {
  static constexpr int WIN = 2 * RAD + 1;
  static constexpr int Q = (2 * RAD + 3) / 4;
  static constexpr int OFF = 4 * Q - 2 * RAD;
  static constexpr int WW = GF_W + 8 * Q;          // copied input columns
  static constexpr int CW = WW / 4;                // 16-byte chunks per row
  static constexpr int IP = WW + 4;                // input pitch
  static constexpr int WU = GF_W + 4 * RAD;        // columns of the statistics
  static constexpr int W1 = GF_W + 2 * RAD;        // columns of a, b
  static constexpr int VP = WU | 1;                // pitch of the column sums
  static constexpr int AP = W1 | 1;                // pitch of a, b and their sums
  static constexpr int Rin = 2 * GF_RB + 2 * RAD;  // input ring rows
  static constexpr int Rab = GF_RB + 2 * RAD;      // a, b ring rows
  static constexpr int floats = 2 * Rin * IP + 4 * GF_RB * VP + 2 * Rab * AP + 2 * GF_RB * AP;
};

static size_t gf_smem_bytes(int rad) {
  switch (rad) {
    case 0: return GfGeom<0>::floats * sizeof(float);
    case 1: return GfGeom<1>::floats * sizeof(float);
    case 2: return GfGeom<2>::floats * sizeof(float);
    case 3: return GfGeom<3>::floats * sizeof(float);
    case 4: return GfGeom<4>::floats * sizeof(float);
    case 5: return GfGeom<5>::floats * sizeof(float);
    case 6: return GfGeom<6>::floats * sizeof(float);
    case 7: return GfGeom<7>::floats * sizeof(float);
    default: return GfGeom<8>::floats * sizeof(float);
  }
}

GFD_D int wrap_dec(int s, int R) { return s == 0 ? R - 1 : s - 1; }
GFD_D int wrap_inc(int s, int R) { return s == R - 1 ? 0 : s + 1; }
GFD_D int wrap_sub(int s, int k, int R) {  // (s - k) mod R for 0 <= k <= R
  const int t = s - k;
  return t < 0 ? t + R : t;
}

template <int RAD>
GFD_D void gf_items(const ClassDesc& cd, const ImgDesc* __restrict__ imgs, ImgState* st, int iter,
                    bool shifted, int H, float* sm, double* red, int* s_flag) {
  using G = GfGeom<RAD>;
  constexpr int WIN = G::WIN, OFF = G::OFF, IP = G::IP, VP = G::VP, AP = G::AP;
  constexpr int WU = G::WU, W1 = G::W1, Rin = G::Rin, Rab = G::Rab;
  constexpr int NSB = GF_RB / GF_SB;
  float* const inI = sm;                      // [Rin][IP]
  float* const inP = inI + Rin * IP;          // [Rin][IP]
  float* const vs = inP + Rin * IP;           // [4][GF_RB][VP]
  float* const abA = vs + 4 * GF_RB * VP;     // [Rab][AP]
  float* const abB = abA + Rab * AP;          // [Rab][AP]
  float* const vsA = abB + Rab * AP;          // [GF_RB][AP]
  float* const vsB = vsA + GF_RB * AP;        // [GF_RB][AP]
  constexpr int PS = GF_RB * VP;

  const int M = cd.M, N = cd.N;
  const int tid = threadIdx.x;
  const int strips = N >= GF_W ? N / GF_W : 1;
  const int blocks = M / H;
  const int per_img = strips * blocks;
  const int n_items = cd.n_img * per_img;
  const int nrows = H + 4 * RAD;  // input rows of an item
  const int nq = (nrows + GF_RB - 1) / GF_RB;
  const float inv_n = 1.0f / (float)(WIN * WIN);

  // Input row y of an item whose first row has ring slot `bslot` lives in
  // slot (bslot + y) % Rin; consecutive items continue the ring, so the next
  // item's first batch is fetched during the current item's last one.
  // One warp copies one (plane, row) at a time, a lane per 16-byte chunk.
  auto prefetch = [&](int item, int q, int bslot) {
    if (item < n_items) {
      const int li = item / per_img, rem = item - li * per_img;
      const int y0 = (rem / strips) * H, x0 = (rem % strips) * GF_W;
      const ImgDesc& d = imgs[cd.img0 + li];
      const float* planes[2] = {d.uI, d.up};
      const int r0 = q * GF_RB;
      const int rows = min(GF_RB, nrows - r0);
      const int lane = tid & 31;
      if (lane < G::CW) {
        const int gx = (x0 - 4 * G::Q + 4 * lane) & (N - 1);
        for (int pr = tid >> 5; pr < 2 * rows; pr += GF_THREADS / 32) {
          const int plane = pr & 1, row = pr >> 1;
          const int gy = (y0 - 2 * RAD + r0 + row) & (M - 1);
          const int slot = (bslot + r0 + row) % Rin;
          cp_async16((plane ? inP : inI) + slot * IP + 4 * lane, planes[plane] + (size_t)gy * N + gx);
        }
      }
    }
    cp_async_commit();
  };

  int item = blockIdx.x;
  int bslot = 0;
  prefetch(item, 0, bslot);
  while (item < n_items) {
    const int li = item / per_img, rem = item - li * per_img;
    const int y0 = (rem / strips) * H, x0 = (rem % strips) * GF_W;
    const int gi = cd.img0 + li;
    const ImgDesc& d = imgs[gi];
    float* const u_out = d.u;
    const float* uo = (iter >= 0 && d.isnr_out) ? d.uo : nullptr;
    float cI = 0.0f, cP = 0.0f;
    if (shifted) {
      const size_t c = (size_t)((y0 + H / 2) & (M - 1)) * N + ((x0 + GF_W / 2) & (N - 1));
      cI = __ldg(&d.uI[c]);
      cP = __ldg(&d.up[c]);
    }
    const float eps = (float)d.eps;
    float err = 0.0f;
    const int next_bslot = (bslot + nq * GF_RB) % Rin;
    for (int q = 0; q < nq; ++q) {
      cp_async_wait<0>();
      __syncthreads();
      if (q + 1 < nq)
        prefetch(item, q + 1, bslot);
      else
        prefetch(item + gridDim.x, 0, next_bslot);
      const int r0 = q * GF_RB;
      const int rows = min(GF_RB, nrows - r0);
      const int s_r0 = (bslot + r0) % Rin;  // ring slot of input row r0
      // 1. column window sums of J, Q, J^2, J Q for rows y >= 2r of the batch
      //    (window rows y-2r .. y)
      for (int u = tid; u < WU * NSB; u += GF_THREADS) {
        const int c = u % WU, sb = u / WU;
        const int lo = max(sb * GF_SB, 2 * RAD - r0);
        const int hi = min(sb * GF_SB + GF_SB, rows);
        if (lo >= hi) continue;
        const float* cI_col = inI + c + OFF;
        const float* cP_col = inP + c + OFF;
        float s0 = 0.f, s1 = 0.f, s2 = 0.f, s3 = 0.f;
        int sl = s_r0 + lo;
        if (sl >= Rin) sl -= Rin;
        {
          int t = sl;
#pragma unroll
          for (int dd = 0; dd < WIN; ++dd) {
            const float J = cI_col[t * IP] - cI, Qv = cP_col[t * IP] - cP;
            s0 += J;
            s1 += Qv;
            s2 = fmaf(J, J, s2);
            s3 = fmaf(J, Qv, s3);
            t = wrap_dec(t, Rin);
          }
        }
        float* v = vs + lo * VP + c;
        v[0] = s0;
        v[PS] = s1;
        v[2 * PS] = s2;
        v[3 * PS] = s3;
        for (int rho = lo + 1; rho < hi; ++rho) {
          sl = wrap_inc(sl, Rin);
          const int so = wrap_sub(sl, WIN, Rin);
          const float Jn = cI_col[sl * IP] - cI, Qn = cP_col[sl * IP] - cP;
          const float Jo = cI_col[so * IP] - cI, Qo = cP_col[so * IP] - cP;
          s0 += Jn - Jo;
          s1 += Qn - Qo;
          s2 += fmaf(Jn, Jn, -Jo * Jo);
          s3 += fmaf(Jn, Qn, -Jo * Qo);
          v += VP;
          v[0] = s0;
          v[PS] = s1;
          v[2 * PS] = s2;
          v[3 * PS] = s3;
        }
      }
      __syncthreads();
      // 2. row window sums -> a_k (Eq. 3), b_k (Eq. 4); the (a, b) row of
      //    input row y goes to ring slot y % Rab
      {
        constexpr int RUNS = (W1 + GF_C - 1) / GF_C;
        for (int u = tid; u < GF_RB * RUNS; u += GF_THREADS) {
          const int rho = u % GF_RB, run = u / GF_RB;
          const int y = r0 + rho;
          if (rho >= rows || y < 2 * RAD) continue;
          const float* v = vs + rho * VP + run * GF_C;
          float s0 = 0.f, s1 = 0.f, s2 = 0.f, s3 = 0.f;
#pragma unroll
          for (int dd = 0; dd < WIN; ++dd) {
            s0 += v[dd];
            s1 += v[PS + dd];
            s2 += v[2 * PS + dd];
            s3 += v[3 * PS + dd];
          }
          const int slot = y % Rab;
          float* ar = abA + slot * AP + run * GF_C;
          float* br = abB + slot * AP + run * GF_C;
#pragma unroll
          for (int c = 0; c < GF_C; ++c) {
            if (run * GF_C + c >= W1) break;
            if (c > 0) {
              s0 += v[c + 2 * RAD] - v[c - 1];
              s1 += v[PS + c + 2 * RAD] - v[PS + c - 1];
              s2 += v[2 * PS + c + 2 * RAD] - v[2 * PS + c - 1];
              s3 += v[3 * PS + c + 2 * RAD] - v[3 * PS + c - 1];
            }
            const float mJ = s0 * inv_n, mQ = s1 * inv_n;
            const float var = fmaf(-mJ, mJ, s2 * inv_n);  // sigma_k^2
            const float cov = fmaf(-mJ, mQ, s3 * inv_n);  // mean(I p) - mu pbar
            const float a = cov / (var + eps);
            ar[c] = a;
            br[c] = (mQ + cP) - a * (mJ + cI);
          }
        }
      }
      __syncthreads();
      // 3. column window sums of a and b for rows y >= 4r (a, b rows y-2r .. y)
      for (int u = tid; u < W1 * NSB; u += GF_THREADS) {
        const int c = u % W1, sb = u / W1;
        const int lo = max(sb * GF_SB, 4 * RAD - r0);
        const int hi = min(sb * GF_SB + GF_SB, rows);
        if (lo >= hi) continue;
        const float* a_col = abA + c;
        const float* b_col = abB + c;
        int sl = (r0 + lo) % Rab;
        float sa = 0.f, sb_ = 0.f;
        {
          int t = sl;
#pragma unroll
          for (int dd = 0; dd < WIN; ++dd) {
            sa += a_col[t * AP];
            sb_ += b_col[t * AP];
            t = wrap_dec(t, Rab);
          }
        }
        vsA[lo * AP + c] = sa;
        vsB[lo * AP + c] = sb_;
        for (int rho = lo + 1; rho < hi; ++rho) {
          sl = wrap_inc(sl, Rab);
          const int so = wrap_sub(sl, WIN, Rab);
          sa += a_col[sl * AP] - a_col[so * AP];
          sb_ += b_col[sl * AP] - b_col[so * AP];
          vsA[rho * AP + c] = sa;
          vsB[rho * AP + c] = sb_;
        }
      }
      __syncthreads();
      // 4. row window sums -> u = abar I + bbar (Eq. 5) for output row y - 4r,
      //    GF_C consecutive outputs per thread, one 16-byte store
      {
        static_assert(GF_W / GF_C * GF_RB == GF_THREADS, "one unit per thread");
        const int rho = tid % GF_RB, run = tid / GF_RB;
        const int y = r0 + rho;
        const int x = run * GF_C;
        if (rho < rows && y >= 4 * RAD && (N >= GF_W || x < N)) {
          const float* va = vsA + rho * AP + x;
          const float* vb = vsB + rho * AP + x;
          int si = s_r0 + rho - 2 * RAD;  // input row y - 2r
          if (si < 0) si += Rin;
          if (si >= Rin) si -= Rin;
          const float* ri = inI + si * IP + x + 2 * RAD + OFF;
          float sa = 0.f, sb_ = 0.f;
#pragma unroll
          for (int dd = 0; dd < WIN; ++dd) {
            sa += va[dd];
            sb_ += vb[dd];
          }
          float o[GF_C];
#pragma unroll
          for (int c = 0; c < GF_C; ++c) {
            if (c > 0) {
              sa += va[c + 2 * RAD] - va[c - 1];
              sb_ += vb[c + 2 * RAD] - vb[c - 1];
            }
            o[c] = fmaf(sa * inv_n, ri[c], sb_ * inv_n);
          }
          const int gy = (y0 + y - 4 * RAD) & (M - 1);
          const size_t off = (size_t)gy * N + x0 + x;
          *reinterpret_cast<float4*>(u_out + off) = make_float4(o[0], o[1], o[2], o[3]);
          if (uo) {
            const float4 t = __ldg(reinterpret_cast<const float4*>(uo + off));
            const float e0 = o[0] - t.x, e1 = o[1] - t.y, e2 = o[2] - t.z, e3 = o[3] - t.w;
            err = fmaf(e0, e0, fmaf(e1, e1, fmaf(e2, e2, fmaf(e3, e3, err))));
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
        for (int w = 0; w < GF_THREADS / 32; ++w) s += red[w];
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
    bslot = next_bslot;
    item += gridDim.x;
  }
  cp_async_wait<0>();
}

__global__ void __launch_bounds__(GF_THREADS, 3)
k_guided_filter(ClassDesc cd, const ImgDesc* __restrict__ imgs, ImgState* st, int iter,
                int plain_var, int rad, int H) {
  extern __shared__ __align__(16) float gsm[];
  __shared__ double red[GF_THREADS / 32];
  __shared__ int s_flag;
  const bool shifted = plain_var == 0;
  switch (rad) {
    case 0: gf_items<0>(cd, imgs, st, iter, shifted, H, gsm, red, &s_flag); break;
    case 1: gf_items<1>(cd, imgs, st, iter, shifted, H, gsm, red, &s_flag); break;
    case 2: gf_items<2>(cd, imgs, st, iter, shifted, H, gsm, red, &s_flag); break;
    case 3: gf_items<3>(cd, imgs, st, iter, shifted, H, gsm, red, &s_flag); break;
    case 4: gf_items<4>(cd, imgs, st, iter, shifted, H, gsm, red, &s_flag); break;
    case 5: gf_items<5>(cd, imgs, st, iter, shifted, H, gsm, red, &s_flag); break;
    case 6: gf_items<6>(cd, imgs, st, iter, shifted, H, gsm, red, &s_flag); break;
    case 7: gf_items<7>(cd, imgs, st, iter, shifted, H, gsm, red, &s_flag); break;
    default: gf_items<8>(cd, imgs, st, iter, shifted, H, gsm, red, &s_flag); break;
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
  const int H = c.cd.M < GF_H ? c.cd.M : GF_H;
  const int strips = c.cd.N >= GF_W ? c.cd.N / GF_W : 1;
  for (int g = 0; g < c.n_rad_groups; ++g) {
    const RadGroup& rg = c.rad_groups[g];
    ClassDesc cd = c.cd;
    cd.img0 = rg.img0;
    cd.n_img = rg.n_img;
    const size_t smem = gf_smem_bytes(rg.rad);
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_guided_filter, GF_THREADS, smem) !=
            cudaSuccess || per_sm < 1)
      per_sm = 1;
    const int n_items = cd.n_img * strips * (cd.M / H);
    int grid = per_sm * gf_sm_count();
    if (grid > n_items) grid = n_items;
    k_guided_filter<<<grid, GF_THREADS, smem, s>>>(cd, c.imgs, c.st, iter, plain_var, rg.rad, H);
  }
  return cudaGetLastError();
}

cudaError_t configure_gf_kernel() {
  return cudaFuncSetAttribute(k_guided_filter, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)gf_smem_bytes(GF_RMAX));
}

}  // namespace gfd
