// Once-per-solve kernels: PSF embedding, observation statistics, the
// discrepancy target (Sec. 3.2, Eq. 12) and the unpacked DC / Nyquist columns.
#include "df.cuh"
#include "lambda.cuh"
#include "launch.h"

namespace gfd {

GFD_D df warp_sum_df(df v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1)
    v = df_add(v, df{__shfl_xor_sync(0xffffffffu, v.hi, o), __shfl_xor_sync(0xffffffffu, v.lo, o)});
  return v;
}

// Sum y, y^2, (y - u_orig)^2 over each image, and sum h, sum |h|.  Each
// thread keeps compensated sums (an FP32 running sum plus the exact rounding
// errors of its additions, summed apart; each square formed exactly by a
// two-product, each difference by a two-sum) over float4 groups, so no FP64
// instruction runs per pixel; warps and blocks add double-float values, and
// the per-block results are added in FP64.  grid (chunks, n_img).
struct CAcc {
  float hi = 0.0f, lo = 0.0f;
  GFD_D void add(float v) {
    const df t = two_sum(hi, v);
    hi = t.hi;
    lo += t.lo;
  }
  GFD_D void add(df v) {
    const df t = two_sum(hi, v.hi);
    hi = t.hi;
    lo += t.lo + v.lo;
  }
  GFD_D df get() const { return two_sum(hi, lo); }
};

__global__ void k_setup_stats(ClassDesc cd, const ImgDesc* __restrict__ imgs, ImgState* st) {
  __shared__ df red[3][32];
  const int gi = cd.img0 + blockIdx.y;
  const ImgDesc& d = imgs[gi];
  const size_t P4 = (size_t)cd.M * cd.N / 4;
  const float4* y4 = reinterpret_cast<const float4*>(d.y);
  const float4* o4 = reinterpret_cast<const float4*>(d.uo);
  CAcc ay, ayy, ae;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < P4;
       i += (size_t)gridDim.x * blockDim.x) {
    const float4 v4 = __ldg(&y4[i]);
    const float v[4] = {v4.x, v4.y, v4.z, v4.w};
    float o[4] = {0.0f, 0.0f, 0.0f, 0.0f};
    if (o4) {
      const float4 q = __ldg(&o4[i]);
      o[0] = q.x; o[1] = q.y; o[2] = q.z; o[3] = q.w;
    }
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      ay.add(v[k]);
      ayy.add(two_prod(v[k], v[k]));
      if (o4) {
        const df e = two_sum(v[k], -o[k]);  // exact difference
        df e2 = two_prod(e.hi, e.hi);
        e2.lo = fmaf(2.0f * e.hi, e.lo, e2.lo);
        ae.add(e2);
      }
    }
  }
  df sy = ay.get(), syy = ayy.get(), se = ae.get();
  sy = warp_sum_df(sy);
  syy = warp_sum_df(syy);
  se = warp_sum_df(se);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane == 0) {
    red[0][warp] = sy;
    red[1][warp] = syy;
    red[2][warp] = se;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    df a = red[0][0], b = red[1][0], c = red[2][0];
    for (int w = 1; w < (int)(blockDim.x >> 5); ++w) {
      a = df_add(a, red[0][w]);
      b = df_add(b, red[1][w]);
      c = df_add(c, red[2][w]);
    }
    atomicAdd(&st[gi].sum_y, df_to_double(a));
    atomicAdd(&st[gi].sum_yy, df_to_double(b));
    if (d.uo) atomicAdd(&st[gi].den_isnr, df_to_double(c));
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    double sh = 0.0, sa = 0.0;
    for (int i = 0; i < d.kh * d.kw; ++i) {
      const double v = (double)d.h[i];
      sh += v;
      sa += fabs(v);
    }
    st[gi].sum_h = sh;
    st[gi].amax = sa;  // squared in k_setup_init
  }
}

// Starting iterate of every image of a class: u_E = u_init, or 0 (Step 0).
// Images are M*N floats, 16-byte aligned, M*N a multiple of 4 for every
// supported canvas; grid-stride over float4 groups of all images.
__global__ void k_init_u(ClassDesc cd, const ImgDesc* __restrict__ imgs) {
  const size_t P4 = (size_t)cd.M * cd.N / 4;
  const size_t total = P4 * cd.n_img;
  for (size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
       idx += (size_t)gridDim.x * blockDim.x) {
    const size_t li = idx / P4, i = idx - li * P4;
    const ImgDesc& d = imgs[cd.img0 + li];
    const float4 v = d.u0 ? __ldg(reinterpret_cast<const float4*>(d.u0) + i)
                          : make_float4(0.0f, 0.0f, 0.0f, 0.0f);
    reinterpret_cast<float4*>(d.u)[i] = v;
  }
}

// rho (Eq. 12), the target T = rho P sigma^2 (Sec. 3.2), the first bracket.
__global__ void k_setup_init(ClassDesc cd, const ImgDesc* __restrict__ imgs, ImgState* st,
                             double rho_fixed) {
  const int li = blockIdx.x * blockDim.x + threadIdx.x;
  if (li >= cd.n_img) return;
  const int gi = cd.img0 + li;
  const ImgDesc& d = imgs[gi];
  ImgState* S = st + gi;
  const double P = (double)cd.M * cd.N;
  const double sig2 = d.sigma * d.sigma;
  const double h1 = S->amax;
  S->amax = h1 * h1;
  if (!(S->sum_h > 0.0)) S->status |= ST_BAD_PSF;
  double rho;
  if (rho_fixed > 0.0) {
    rho = rho_fixed;
  } else {
    // ||y - mu(y)||^2 = sum y^2 - (sum y)^2 / P
    const double num = (S->sum_yy - S->sum_y * S->sum_y / P) - P * sig2;
    const double den = h1 * h1 * S->sum_yy;
    const double rad = 1.0 - num / den;
    if (rad > 0.0) {
      rho = fmin(1.0, sqrt(rad));
    } else {
      S->status |= ST_BAD_RHO;
      rho = 1.0;
    }
  }
  S->rho = rho;
  S->T = rho * P * sig2;
  S->invT = 1.0 / S->T;
  S->lam = NAN;
  S->need = 0;
  S->rtol = d.lam_rtol;
  set_bracket(S, INITIAL_LO, INITIAL_HI);
}

// Zero the per-item partial slots of the spectral passes (each pass leaves
// them zeroed again after reducing them).
__global__ void k_zero_parts(ClassDesc cd, const ImgDesc* __restrict__ imgs, int n_slots) {
  const ImgDesc& d = imgs[cd.img0 + blockIdx.y];
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n_slots; i += gridDim.x * blockDim.x)
    d.part[i] = 0.0;
}

// Circular PSF embedding: offset (a - kh/2, b - kw/2) -> canvas index mod (M, N).
__global__ void k_embed_psf(ClassDesc cd, const ImgDesc* __restrict__ imgs, int dst_sel) {
  const size_t P = (size_t)cd.M * cd.N;
  const size_t total = P * cd.n_img;
  for (size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
       idx += (size_t)gridDim.x * blockDim.x) {
    const int li = (int)(idx / P);
    const int rem = (int)(idx - (size_t)li * P);
    const int i = rem / cd.N, j = rem - i * cd.N;
    const ImgDesc& d = imgs[cd.img0 + li];
    const int rh = d.kh / 2, rw = d.kw / 2;
    float s = 0.0f;
    for (int a = (i + rh) % cd.M; a < d.kh; a += cd.M)
      for (int b = (j + rw) % cd.N; b < d.kw; b += cd.N) s += d.h[a * d.kw + b];
    float* dst = dst_sel == SEL_UI ? d.uI : d.up;
    dst[rem] = s;
  }
}

// Unpack column 0 of the packed H and Y into the bins (k, 0) and (k, N/2);
// the DC bins take the FP64 sums (rounded once).
__global__ void k_unpack_dc(ClassDesc cd, const ImgDesc* __restrict__ imgs, const ImgState* st) {
  const int gi = cd.img0 + blockIdx.y;
  const ImgDesc& d = imgs[gi];
  const int M = cd.M, TB = cd.TB;  // column 0 is column 0 of tile 0
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= M) return;
  const int km = (M - k) & (M - 1);
  const float2 hk = d.H[(size_t)k * TB], hm = d.H[(size_t)km * TB];
  const float2 yk = d.Y[(size_t)k * TB], ym = d.Y[(size_t)km * TB];
  float2 A, B;
  {
    const float2 c = cconj(hm);
    A = cscale(cadd(hk, c), 0.5f);
    const float2 D = csub(hk, c);
    B = make_float2(0.5f * D.y, -0.5f * D.x);
  }
  if (k == 0) A = make_float2((float)st[gi].sum_h, 0.0f);
  d.H0[k] = A;
  d.HN[k] = B;
  {
    const float2 c = cconj(ym);
    A = cscale(cadd(yk, c), 0.5f);
    const float2 D = csub(yk, c);
    B = make_float2(0.5f * D.y, -0.5f * D.x);
  }
  if (k == 0) A = make_float2((float)st[gi].sum_y, 0.0f);
  d.Y0[k] = A;
  d.YN[k] = B;
  if (k == 0) {
    d.H[0].x = (float)st[gi].sum_h;
    d.Y[0].x = (float)st[gi].sum_y;
  }
}

// y (m x n) -> canvas (M x N): symmetric reflection at the bottom and right
// edges with period 2m (2n), the edge sample repeated.
__global__ void k_pad_symmetric(const float* __restrict__ y, int m, int n, float* __restrict__ dst,
                                int M, int N) {
  const size_t total = (size_t)M * N;
  for (size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
       idx += (size_t)gridDim.x * blockDim.x) {
    const int i = (int)(idx / N), j = (int)(idx - (size_t)i * N);
    const int ti = i % (2 * m), tj = j % (2 * n);
    const int si = ti < m ? ti : 2 * m - 1 - ti, sj = tj < n ? tj : 2 * n - 1 - tj;
    dst[idx] = __ldg(&y[(size_t)si * n + sj]);
  }
}

// canvas (M x N) -> its top-left m x n part.
__global__ void k_crop(const float* __restrict__ src, int N, float* __restrict__ dst, int m, int n) {
  const size_t total = (size_t)m * n;
  for (size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
       idx += (size_t)gridDim.x * blockDim.x) {
    const int i = (int)(idx / n), j = (int)(idx - (size_t)i * n);
    dst[idx] = __ldg(&src[(size_t)i * N + j]);
  }
}

static unsigned plane_blocks(size_t total) {
  size_t nb = (total + 255) / 256;
  if (nb > 152 * 16) nb = 152 * 16;
  return (unsigned)(nb < 1 ? 1 : nb);
}

cudaError_t launch_pad_symmetric(const float* y, int m, int n, float* dst, int M, int N,
                                 cudaStream_t s) {
  k_pad_symmetric<<<plane_blocks((size_t)M * N), 256, 0, s>>>(y, m, n, dst, M, N);
  return cudaGetLastError();
}

cudaError_t launch_crop(const float* src, int N, float* dst, int m, int n, cudaStream_t s) {
  k_crop<<<plane_blocks((size_t)m * n), 256, 0, s>>>(src, N, dst, m, n);
  return cudaGetLastError();
}

// u_iters[k] <- u for every image of the class that keeps checkpoints.
__global__ void k_save_iterate(ClassDesc cd, const ImgDesc* __restrict__ imgs, int k) {
  const size_t P4 = (size_t)cd.M * cd.N / 4;
  const size_t total = P4 * cd.n_img;
  for (size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
       idx += (size_t)gridDim.x * blockDim.x) {
    const size_t li = idx / P4, i = idx - li * P4;
    const ImgDesc& d = imgs[cd.img0 + li];
    if (!d.u_iters) continue;
    reinterpret_cast<float4*>(d.u_iters + (size_t)k * cd.M * cd.N)[i] =
        __ldcg(reinterpret_cast<const float4*>(d.u) + i);
  }
}

cudaError_t launch_save_iterate(const ClassLaunch& c, int k, cudaStream_t s) {
  const size_t total = (size_t)c.cd.M * c.cd.N / 4 * c.cd.n_img;
  k_save_iterate<<<plane_blocks(total), 256, 0, s>>>(c.cd, c.imgs, k);
  return cudaGetLastError();
}

cudaError_t launch_setup_stats(const ClassLaunch& c, cudaStream_t s) {
  const size_t P = (size_t)c.cd.M * c.cd.N;
  int chunks = (int)((P + 256 * 16 - 1) / (256 * 16));  // 4 float4 groups per thread
  if (chunks > 1024) chunks = 1024;
  k_setup_stats<<<dim3(chunks, c.cd.n_img), 256, 0, s>>>(c.cd, c.imgs, c.st);
  return cudaGetLastError();
}

cudaError_t launch_init_u(const ClassLaunch& c, cudaStream_t s) {
  const size_t total = (size_t)c.cd.M * c.cd.N / 4 * c.cd.n_img;
  size_t nb = (total + 255) / 256;
  if (nb > 152 * 16) nb = 152 * 16;
  if (nb < 1) nb = 1;
  k_init_u<<<(unsigned)nb, 256, 0, s>>>(c.cd, c.imgs);
  return cudaGetLastError();
}

cudaError_t launch_setup_init(const ClassLaunch& c, double rho_fixed, cudaStream_t s) {
  k_setup_init<<<(c.cd.n_img + 127) / 128, 128, 0, s>>>(c.cd, c.imgs, c.st, rho_fixed);
  const size_t Lc = c.cd.N / 2;
  const size_t col_items = Lc / 2, pass_items = (size_t)c.cd.M * Lc / 4096 + 1;
  const int n_slots = (int)((KNODES + 1) * (col_items > pass_items ? col_items : pass_items));
  k_zero_parts<<<dim3((n_slots + 255) / 256, c.cd.n_img), 256, 0, s>>>(c.cd, c.imgs, n_slots);
  return cudaGetLastError();
}

cudaError_t launch_embed_psf(const ClassLaunch& c, int dst, cudaStream_t s) {
  const size_t total = (size_t)c.cd.M * c.cd.N * c.cd.n_img;
  size_t nb = (total + 255) / 256;
  if (nb > 152 * 64) nb = 152 * 64;
  k_embed_psf<<<(unsigned)nb, 256, 0, s>>>(c.cd, c.imgs, dst);
  return cudaGetLastError();
}

cudaError_t launch_unpack_dc(const ClassLaunch& c, cudaStream_t s) {
  k_unpack_dc<<<dim3((c.cd.M + 127) / 128, c.cd.n_img), 128, 0, s>>>(c.cd, c.imgs, c.st);
  return cudaGetLastError();
}

cudaError_t configure_fft_kernels();
cudaError_t configure_gf_kernel();
cudaError_t configure_gfc_kernels();
cudaError_t configure_adj_kernels();
cudaError_t configure_df_kernels();

cudaError_t configure_kernels() {
  cudaError_t e = configure_fft_kernels();
  if (e != cudaSuccess) return e;
  if ((e = configure_df_kernels()) != cudaSuccess) return e;
  if ((e = configure_gfc_kernels()) != cudaSuccess) return e;
  if ((e = configure_adj_kernels()) != cudaSuccess) return e;
  return configure_gf_kernel();
}

}  // namespace gfd
