// Guided filter u = guidfilter(u_I, u_p, w, eps) (Sec. 2, Eq. 3-5) with
// periodic windows, r = (w-1)/2.
//
// Every warp works alone, down a strip of GFW_COLS input columns (4 per
// lane): no block barriers.  Input rows enter a per-warp ring in shared
// memory by 16-byte asynchronous copies GFW_AHEAD rows ahead of use; each lane
// copies and reads only its own 4 columns.  For the item's rows the warp
// forms, row by row,
//   1. window sums down its columns of J = I - c_I, Q = p - c_p, J^2, J Q
//      (in registers; re-formed directly every GFW_SUB rows and slid in
//      between, so no sum is carried over more than GFW_SUB - 1 slides),
//   2. window sums along the row by warp shuffles (the 2r neighbouring
//      columns come from the adjacent lanes) -> mu_k, pbar_k, sigma_k^2 and
//      the covariance -> a_k (Eq. 3), b_k (Eq. 4) for each column,
//   3. window sums of a and b down the columns (a per-warp ring of the last
//      2r+1 rows of a, b in shared memory, each lane touching only its own
//      columns), re-formed / slid like 1.,
//   4. window sums along the row by shuffles -> abar, bbar ->
//      u = abar I + bbar (Eq. 5), stored as 16-byte vectors.
// The strip's outer 4*ceil(r/2) columns on each side are halo (their sums
// are incomplete); the columns in between are the item's output, so
// neighbouring strips overlap by the halo.  Input rows and columns wrap
// periodically.  Window statistics are taken about reference values (c_I,
// c_p: the item's centre pixel), which removes the cancellation in
// sigma_k^2 = E[I^2] - mu^2 where the window mean is close to c_I.
#include "common.cuh"
#include "launch.h"

namespace gfd {

constexpr int GFW_COLS = 128;   // input columns per strip (4 per lane)
constexpr int GFW_SUB = 4;      // rows between direct re-formations of the column sums
constexpr int GFW_WARPS = 4;    // warps per block
constexpr int GFW_AHEAD = 2;    // input rows requested ahead of use
constexpr int GF_RMAX = 8;      // w <= 17
constexpr unsigned FULL = 0xffffffffu;

template <int RAD>
struct GfwGeom {
  static constexpr int WIN = 2 * RAD + 1;
  static constexpr int RI = WIN + 1 + GFW_AHEAD;  // input ring rows: window, the row leaving, ahead
  static constexpr int HALO = 4 * ((RAD + 1) / 2);  // >= 2r, multiple of 4
  static constexpr int WOUT = GFW_COLS - 2 * HALO;  // output columns per strip
};

// per-warp shared memory: (a, b) ring of 2r+1 rows, (I, p) ring of 2r+2+GFW_AHEAD rows
GFD_HD int gfw_ring_floats(int rad) {
  return (2 * (2 * rad + 1) + 2 * (2 * rad + 2 + GFW_AHEAD)) * GFW_COLS;
}
static int gfw_wout(int rad) { return GFW_COLS - 8 * ((rad + 1) / 2); }

// Window sums of radius RAD along the strip: v[k] is column 4*lane + k;
// s[k] = sum of columns 4*lane + k - RAD .. 4*lane + k + RAD.  Columns beyond
// the warp's edges are not available: the lanes within RAD columns of an
// edge get incomplete sums (those columns are halo).
template <int RAD>
GFD_D void hsum4(const float (&v)[4], float (&s)[4]) {
  constexpr int E = 2 * RAD + 4;
  float e[E];  // columns 4*lane - RAD .. 4*lane + 3 + RAD
#pragma unroll
  for (int q = 0; q < E; ++q) {
    const int c = q - RAD;                           // column offset from 4*lane
    const int lo = c >= 0 ? c / 4 : -((3 - c) / 4);  // floor(c / 4): source lane offset
    const int idx = c - 4 * lo;                      // column within the source lane
    if (lo == 0)
      e[q] = v[idx];
    else if (lo > 0)
      e[q] = __shfl_down_sync(FULL, v[idx], lo);
    else
      e[q] = __shfl_up_sync(FULL, v[idx], -lo);
  }
  float acc = 0.0f;
#pragma unroll
  for (int q = 0; q <= 2 * RAD; ++q) acc += e[q];
  s[0] = acc;
#pragma unroll
  for (int k = 1; k < 4; ++k) {
    acc += e[k + 2 * RAD] - e[k - 1];
    s[k] = acc;
  }
}

template <int RAD>
GFD_D void gfw_items(const ClassDesc& cd, const ImgDesc* __restrict__ imgs, ImgState* st,
                     int iter, bool shifted, int H, float* ring, int gwarp, int nwarps) {
  using G = GfwGeom<RAD>;
  constexpr int WIN = G::WIN, HALO = G::HALO, WOUT = G::WOUT, RI = G::RI;
  const int lane = threadIdx.x & 31;
  const int M = cd.M, N = cd.N;
  const int strips = (N + WOUT - 1) / WOUT;
  const int per_img = strips * (M / H);
  const int n_items = cd.n_img * per_img;
  const float inv_n = 1.0f / (float)(WIN * WIN);
  float* const ra = ring;                   // [WIN][GFW_COLS] a
  float* const rb = ra + WIN * GFW_COLS;    // [WIN][GFW_COLS] b
  float* const rI = rb + WIN * GFW_COLS;    // [RI][GFW_COLS] I
  float* const rP = rI + RI * GFW_COLS;     // [RI][GFW_COLS] p
  // this lane's columns lie in the strip's output part
  const bool out_lane = 4 * lane >= HALO && 4 * lane < HALO + WOUT;

  for (int item = gwarp; item < n_items; item += nwarps) {
    const int li = item / per_img, rem = item - li * per_img;
    const int y0 = (rem / strips) * H, x0 = (rem % strips) * WOUT;
    const int gi = cd.img0 + li;
    const ImgDesc& d = imgs[gi];
    const float* __restrict__ I = d.uI;
    const float* __restrict__ P = d.up;
    const float* uo = (iter >= 0 && d.isnr_out) ? d.uo : nullptr;
    // this lane's 4 columns (16-byte aligned: x0 and HALO are multiples of 4)
    const int gx = (x0 - HALO + 4 * lane) & (N - 1);
    const bool store = out_lane && x0 + 4 * lane - HALO < N;
    float cI = 0.0f, cP = 0.0f;
    if (shifted) {
      const size_t c = (size_t)((y0 + H / 2) & (M - 1)) * N + ((x0 + WOUT / 2) & (N - 1));
      cI = __ldg(&I[c]);
      cP = __ldg(&P[c]);
    }
    const float eps = (float)d.eps;
    // input row j of the item is image row y0 - 2r + j, ring slot j % RI
    const int nin = H + 4 * RAD;
    auto fetch = [&](int j) {
      if (j < nin) {
        const size_t off = (size_t)((y0 - 2 * RAD + j) & (M - 1)) * N + gx;
        cp_async16(rI + (j % RI) * GFW_COLS + 4 * lane, I + off);
        cp_async16(rP + (j % RI) * GFW_COLS + 4 * lane, P + off);
      }
    };
    auto ring4 = [&](const float* r, int j) {
      return reinterpret_cast<const float4*>(r + (j % RI) * GFW_COLS)[lane];
    };
    for (int j = 0; j <= 2 * RAD; ++j) fetch(j);
    cp_async_commit();
#pragma unroll
    for (int a = 1; a < GFW_AHEAD; ++a) {
      fetch(2 * RAD + a);
      cp_async_commit();
    }
    float V[4][4];   // [J, Q, J^2, J Q][column]: window sums down the columns
    float VA[2][4];  // [a, b][column]
    float err = 0.0f;
    // stats row s (image row y0 - r + s) has its column window on input rows
    // j = s .. s + 2r; output row t = s - 2r needs stats rows t .. t + 2r
    for (int s = 0; s < H + 2 * RAD; ++s) {
      fetch(s + 2 * RAD + GFW_AHEAD);  // its slot held row s - 2, no longer needed
      cp_async_commit();
      cp_async_wait<GFW_AHEAD>();      // rows up to s + 2r have landed
      const int t = s - 2 * RAD;  // output row (if >= 0)
      // the reference row of the ISNR sums is requested early (used last)
      float4 g = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
      if (uo && store && t >= 0)
        g = __ldg(reinterpret_cast<const float4*>(uo + (size_t)((y0 + t) & (M - 1)) * N + gx));
      if (s % GFW_SUB == 0) {
#pragma unroll
        for (int q = 0; q < 4; ++q)
#pragma unroll
          for (int k = 0; k < 4; ++k) V[q][k] = 0.0f;
#pragma unroll
        for (int dd = 0; dd < WIN; ++dd) {
          const float4 iv = ring4(rI, s + dd), pv = ring4(rP, s + dd);
          const float J[4] = {iv.x - cI, iv.y - cI, iv.z - cI, iv.w - cI};
          const float Q[4] = {pv.x - cP, pv.y - cP, pv.z - cP, pv.w - cP};
#pragma unroll
          for (int k = 0; k < 4; ++k) {
            V[0][k] += J[k];
            V[1][k] += Q[k];
            V[2][k] = fmaf(J[k], J[k], V[2][k]);
            V[3][k] = fmaf(J[k], Q[k], V[3][k]);
          }
        }
      } else {
        const float4 in = ring4(rI, s + 2 * RAD), pn = ring4(rP, s + 2 * RAD);
        const float4 io = ring4(rI, s - 1), po = ring4(rP, s - 1);
        const float Jn[4] = {in.x - cI, in.y - cI, in.z - cI, in.w - cI};
        const float Qn[4] = {pn.x - cP, pn.y - cP, pn.z - cP, pn.w - cP};
        const float Jo[4] = {io.x - cI, io.y - cI, io.z - cI, io.w - cI};
        const float Qo[4] = {po.x - cP, po.y - cP, po.z - cP, po.w - cP};
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          V[0][k] += Jn[k] - Jo[k];
          V[1][k] += Qn[k] - Qo[k];
          V[2][k] += fmaf(Jn[k], Jn[k], -Jo[k] * Jo[k]);
          V[3][k] += fmaf(Jn[k], Qn[k], -Jo[k] * Qo[k]);
        }
      }
      // 2. row window sums -> a_k (Eq. 3), b_k (Eq. 4)
      float S0[4], S1[4], S2[4], S3[4];
      hsum4<RAD>(V[0], S0);
      hsum4<RAD>(V[1], S1);
      hsum4<RAD>(V[2], S2);
      hsum4<RAD>(V[3], S3);
      float A[4], B[4];
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const float mJ = S0[k] * inv_n, mQ = S1[k] * inv_n;
        const float var = fmaf(-mJ, mJ, S2[k] * inv_n);  // sigma_k^2
        const float cov = fmaf(-mJ, mQ, S3[k] * inv_n);  // mean(I p) - mu pbar
        A[k] = __fdividef(cov, var + eps);  // var + eps >= eps > 0
        B[k] = (mQ + cP) - A[k] * (mJ + cI);
      }
      // 3. ring slot s % WIN holds stats row s - WIN until overwritten here
      float4* const sa = reinterpret_cast<float4*>(ra + (s % WIN) * GFW_COLS) + lane;
      float4* const sb = reinterpret_cast<float4*>(rb + (s % WIN) * GFW_COLS) + lane;
      const bool slide = t > 0 && t % GFW_SUB != 0;
      if (slide) {
        const float4 oa = *sa, ob = *sb;
        VA[0][0] += A[0] - oa.x;
        VA[0][1] += A[1] - oa.y;
        VA[0][2] += A[2] - oa.z;
        VA[0][3] += A[3] - oa.w;
        VA[1][0] += B[0] - ob.x;
        VA[1][1] += B[1] - ob.y;
        VA[1][2] += B[2] - ob.z;
        VA[1][3] += B[3] - ob.w;
      }
      *sa = make_float4(A[0], A[1], A[2], A[3]);
      *sb = make_float4(B[0], B[1], B[2], B[3]);
      if (t < 0) continue;
      if (!slide) {  // direct: the ring holds stats rows t .. t + 2r
#pragma unroll
        for (int k = 0; k < 4; ++k) VA[0][k] = VA[1][k] = 0.0f;
#pragma unroll
        for (int q = 0; q < WIN; ++q) {
          const float4 a4 = reinterpret_cast<const float4*>(ra + q * GFW_COLS)[lane];
          const float4 b4 = reinterpret_cast<const float4*>(rb + q * GFW_COLS)[lane];
          VA[0][0] += a4.x;
          VA[0][1] += a4.y;
          VA[0][2] += a4.z;
          VA[0][3] += a4.w;
          VA[1][0] += b4.x;
          VA[1][1] += b4.y;
          VA[1][2] += b4.z;
          VA[1][3] += b4.w;
        }
      }
      // 4. row window sums of a, b -> u = abar I + bbar (Eq. 5); the guidance
      //    at output row t is input row j = t + 2r = s
      float SA[4], SB[4];
      hsum4<RAD>(VA[0], SA);
      hsum4<RAD>(VA[1], SB);
      const float4 iv = ring4(rI, s);
      const float ic[4] = {iv.x, iv.y, iv.z, iv.w};
      float o[4];
#pragma unroll
      for (int k = 0; k < 4; ++k) o[k] = fmaf(SA[k] * inv_n, ic[k], SB[k] * inv_n);
      if (store) {
        const size_t off = (size_t)((y0 + t) & (M - 1)) * N + gx;
        *reinterpret_cast<float4*>(d.u + off) = make_float4(o[0], o[1], o[2], o[3]);
        if (uo) {
          const float e0 = o[0] - g.x, e1 = o[1] - g.y, e2 = o[2] - g.z, e3 = o[3] - g.w;
          err = fmaf(e0, e0, fmaf(e1, e1, fmaf(e2, e2, fmaf(e3, e3, err))));
        }
      }
    }
    cp_async_wait<0>();  // the ring is reused by the next item
    if (uo) {
      // ||u - u_orig||^2 of this item: FP32 in the warp, FP64 across items
      err = warp_sum(err);
      if (lane == 0) {
        ImgState* S = st + gi;
        atomicAdd(&S->err2, (double)err);
        __threadfence();
        const unsigned int prev = atomicAdd(&S->gf_done, 1u);
        if (prev == (unsigned)per_img - 1) {
          __threadfence();
          const double e2 = __ldcg(&S->err2);
          d.isnr_out[iter] = 10.0 * log10(S->den_isnr / e2);
          S->err2 = 0.0;
          S->gf_done = 0;
          __threadfence();
        }
      }
    }
    __syncwarp();
  }
}

__global__ void __launch_bounds__(GFW_WARPS * 32)
k_guided_filter(ClassDesc cd, const ImgDesc* __restrict__ imgs, ImgState* st, int iter,
                int plain_var, int rad, int H) {
  extern __shared__ __align__(16) float gsm[];
  const int warp = threadIdx.x >> 5;
  const int gwarp = blockIdx.x * GFW_WARPS + warp;
  const int nwarps = gridDim.x * GFW_WARPS;
  float* ring = gsm + (size_t)warp * gfw_ring_floats(rad);
  const bool shifted = plain_var == 0;
  switch (rad) {
    case 0: gfw_items<0>(cd, imgs, st, iter, shifted, H, ring, gwarp, nwarps); break;
    case 1: gfw_items<1>(cd, imgs, st, iter, shifted, H, ring, gwarp, nwarps); break;
    case 2: gfw_items<2>(cd, imgs, st, iter, shifted, H, ring, gwarp, nwarps); break;
    case 3: gfw_items<3>(cd, imgs, st, iter, shifted, H, ring, gwarp, nwarps); break;
    case 4: gfw_items<4>(cd, imgs, st, iter, shifted, H, ring, gwarp, nwarps); break;
    case 5: gfw_items<5>(cd, imgs, st, iter, shifted, H, ring, gwarp, nwarps); break;
    case 6: gfw_items<6>(cd, imgs, st, iter, shifted, H, ring, gwarp, nwarps); break;
    case 7: gfw_items<7>(cd, imgs, st, iter, shifted, H, ring, gwarp, nwarps); break;
    default: gfw_items<8>(cd, imgs, st, iter, shifted, H, ring, gwarp, nwarps); break;
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
// are ordered by radius, so each group is a contiguous range).  Items are
// (image, strip, block of H rows); H is halved (down to 16) while there are
// fewer items than resident warps.
cudaError_t launch_guided_filter(const ClassLaunch& c, int iter, int plain_var, cudaStream_t s) {
  for (int g = 0; g < c.n_rad_groups; ++g) {
    const RadGroup& rg = c.rad_groups[g];
    ClassDesc cd = c.cd;
    cd.img0 = rg.img0;
    cd.n_img = rg.n_img;
    const size_t smem = (size_t)GFW_WARPS * gfw_ring_floats(rg.rad) * sizeof(float);
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_guided_filter, GFW_WARPS * 32,
                                                      smem) != cudaSuccess ||
        per_sm < 1)
      per_sm = 1;
    const int div = c.grid_div > 1 ? c.grid_div : 1;
    const int warps = (per_sm * gf_sm_count() + div - 1) / div * GFW_WARPS;
    const int strips = (cd.N + gfw_wout(rg.rad) - 1) / gfw_wout(rg.rad);
    int H = cd.M < 64 ? cd.M : 64;
    while (H > 16 && cd.n_img * strips * (cd.M / H) < warps) H /= 2;
    const int n_items = cd.n_img * strips * (cd.M / H);
    int grid = (per_sm * gf_sm_count() + div - 1) / div;
    const int need = (n_items + GFW_WARPS - 1) / GFW_WARPS;
    if (grid > need) grid = need;
    k_guided_filter<<<grid, GFW_WARPS * 32, smem, s>>>(cd, c.imgs, c.st, iter, plain_var, rg.rad, H);
  }
  return cudaGetLastError();
}

cudaError_t configure_gf_kernel() {
  return cudaFuncSetAttribute(k_guided_filter, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)(GFW_WARPS * gfw_ring_floats(GF_RMAX) * sizeof(float)));
}

}  // namespace gfd
