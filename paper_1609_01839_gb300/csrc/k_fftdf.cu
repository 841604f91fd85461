// Double-float 2-D real DFT for the once-per-solve spectra H = F(h) and
// Y = F(y) (Sec. 3.1: the solves of Eq. 8-9 and the residual of Eq. 10-11
// are formed in the DFT domain).
//
// Why not the FP32 transform: its error is about 1e-7 of the spectrum's
// norm in every bin, and the norm of Y is dominated by the image's mean and
// low frequencies.  The bins that decide lambda (|H|^2 <~ lambda: high
// frequencies, where |Y| is at the noise level) then carry errors of
// ~1e-7 * ||y|| / sigma relative to their own size, and the root of Eq. 11
// moves by that times its condition number.  Computing H and Y in
// double-float arithmetic (about 48 bits, FP32 instructions only) and
// rounding once to FP32 removes this term; the per-iteration transforms of
// u_E stay in FP32 (their errors enter Eq. 11 multiplied by |H|).
//
// Same layout as the FP32 path: rows of N reals are transformed as N/2
// complex points z[n] = x[2n] + i x[2n+1] and post-processed into the packed
// half spectrum (X[0] + i X[N/2] in column 0), stored column-tiled; the
// column pass transforms each packed column (length M).  Radix-2
// decimation in time from bit-reversed order, in shared memory.
#include "df.cuh"
#include "launch.h"

namespace gfd {

struct cdf {
  df re, im;
};

// Double-float sum with one two-sum: error within ~2^-44 (|a| + |b|).  A
// transform needs errors small against the norm of its data, not relative
// accuracy under cancellation, so the cheaper form suffices here.
GFD_D df dfs_add(df a, df b) {
  const df s = two_sum(a.hi, b.hi);
  return quick_two_sum(s.hi, s.lo + (a.lo + b.lo));
}
GFD_D df dfs_sub(df a, df b) { return dfs_add(a, df_neg(b)); }

GFD_D cdf cdf_add(cdf a, cdf b) { return cdf{dfs_add(a.re, b.re), dfs_add(a.im, b.im)}; }
GFD_D cdf cdf_sub(cdf a, cdf b) { return cdf{dfs_sub(a.re, b.re), dfs_sub(a.im, b.im)}; }
// x1 * y1 + s * x2 * y2 (s = +1 or -1) in double-float: the two leading
// products exactly (FMA), one two-sum, the cross terms into the low part.
GFD_D df df_dot2(df x1, df y1, df x2, df y2, float sg) {
  const float p1 = x1.hi * y1.hi, e1 = fmaf(x1.hi, y1.hi, -p1);
  const float p2 = sg * (x2.hi * y2.hi), e2 = sg * fmaf(x2.hi, y2.hi, -sg * p2);
  const df s = two_sum(p1, p2);
  float lo = s.lo + (e1 + e2);
  lo = fmaf(x1.hi, y1.lo, fmaf(x1.lo, y1.hi, lo));
  lo = fmaf(sg * x2.hi, y2.lo, fmaf(sg * x2.lo, y2.hi, lo));
  return quick_two_sum(s.hi, lo);
}
GFD_D cdf cdf_mul(cdf a, cdf b) {
  return cdf{df_dot2(a.re, b.re, a.im, b.im, -1.0f), df_dot2(a.re, b.im, a.im, b.re, 1.0f)};
}
GFD_D cdf cdf_half(cdf a) {  // exact
  return cdf{df{0.5f * a.re.hi, 0.5f * a.re.lo}, df{0.5f * a.im.hi, 0.5f * a.im.lo}};
}

// W_L^m from the per-length table (float4: re hi, re lo, im hi, im lo)
GFD_D cdf tw_df(const float4* __restrict__ tab, int L, int m) {
  const float4 v = __ldg(&tab[tab_off(L) + m]);
  return cdf{df{v.x, v.y}, df{v.z, v.w}};
}

// Shared buffer of one transform: hi and lo planes of re and im, each of
// padded length df_plane(L).  Element i sits at i + i/32, so the bit-reversed
// scatter (consecutive i land L/2 apart) and the small-stride butterfly
// steps spread over the banks.
GFD_HD int df_plane(int L) { return L + (L >> 5); }
struct CdfBuf {
  float* rh;
  float* rl;
  float* ih;
  float* il;
  GFD_D static CdfBuf at(float* base, int L) {
    const int p = df_plane(L);
    return CdfBuf{base, base + p, base + 2 * p, base + 3 * p};
  }
  GFD_D cdf get(int i) const {
    i += i >> 5;
    return cdf{df{rh[i], rl[i]}, df{ih[i], il[i]}};
  }
  GFD_D void put(int i, cdf v) const {
    i += i >> 5;
    rh[i] = v.re.hi;
    rl[i] = v.re.lo;
    ih[i] = v.im.hi;
    il[i] = v.im.lo;
  }
};

GFD_D cdf cdf_mul_negi(cdf a) { return cdf{a.im, df_neg(a.re)}; }  // -i a, exact

// Two consecutive radix-2 DIT stages (half sizes h and 2h) on the four
// points k, k+h, k+2h, k+3h, k = 4 (q - j) + j with j = q mod h.  The
// second stage's twiddle for the odd pair is W_4h^(j+h) = -i W_4h^j, so one
// twiddle product is replaced by an exact multiplication by -i; for h = 1
// every twiddle is 1 and no product is formed.
GFD_D void df_radix4(const CdfBuf& x, int L, int h, const float4* __restrict__ tab, int q) {
  const int j = q & (h - 1);
  const int k = ((q - j) << 2) + j;
  const cdf a0 = x.get(k), a1 = x.get(k + h), a2 = x.get(k + 2 * h), a3 = x.get(k + 3 * h);
  cdf b0, b1, b2, b3;
  if (h == 1) {
    b0 = cdf_add(a0, a1);
    b1 = cdf_sub(a0, a1);
    b2 = cdf_add(a2, a3);
    b3 = cdf_sub(a2, a3);
  } else {
    const cdf w1 = tw_df(tab, L, j * (L / (2 * h)));  // W_2h^j
    const cdf v1 = cdf_mul(w1, a1), v3 = cdf_mul(w1, a3);
    b0 = cdf_add(a0, v1);
    b1 = cdf_sub(a0, v1);
    b2 = cdf_add(a2, v3);
    b3 = cdf_sub(a2, v3);
  }
  cdf v2 = b2, v4 = cdf_mul_negi(b3);
  if (h > 1) {
    const cdf w2 = tw_df(tab, L, j * (L / (4 * h)));  // W_4h^j
    v2 = cdf_mul(w2, b2);
    v4 = cdf_mul_negi(cdf_mul(w2, b3));
  }
  x.put(k, cdf_add(b0, v2));
  x.put(k + 2 * h, cdf_sub(b0, v2));
  x.put(k + h, cdf_add(b1, v4));
  x.put(k + 3 * h, cdf_sub(b1, v4));
}

GFD_D void df_radix2(const CdfBuf& x, int L, int h, const float4* __restrict__ tab, int q) {
  const int j = q & (h - 1);
  const int k = ((q - j) << 1) + j;
  const cdf u = x.get(k);
  const cdf v = cdf_mul(tw_df(tab, L, j * (L / (2 * h))), x.get(k + h));
  x.put(k, cdf_add(u, v));
  x.put(k + h, cdf_sub(u, v));
}

// In-place DIT transform of length L (input already bit-reversed) by `nt`
// threads with index t: radix-4 steps, one radix-2 stage last when log2 L is
// odd; synchronises the block after every step.  `active` threads take part
// in the arithmetic, all of them in the barriers.
GFD_D void fft_df(const CdfBuf& x, int L, const float4* __restrict__ tab, int t, int nt,
                  bool active = true) {
  int h = 1;
  for (; 4 * h <= L; h *= 4) {
    if (active)
      for (int q = t; q < L / 4; q += nt) df_radix4(x, L, h, tab, q);
    __syncthreads();
  }
  if (h < L) {
    if (active)
      for (int q = t; q < L / 2; q += nt) df_radix2(x, L, h, tab, q);
    __syncthreads();
  }
}

GFD_D int bitrev(int i, int lg) { return (int)(__brev((unsigned)i) >> (32 - lg)); }

// Row pass: real plane src -> packed row spectra, hi to plane dhi, lo to
// plane dlo (tiled layout).  One block per row.
__global__ void __launch_bounds__(256)
k_row_r2c_df(ClassDesc cd, const ImgDesc* __restrict__ imgs, const float4* __restrict__ tab,
             int src_sel, int dhi_sel, int dlo_sel) {
  extern __shared__ float sm[];
  const int M = cd.M, N = cd.N, L = N / 2, TB = cd.TB;
  const int li = blockIdx.x / M, row = blockIdx.x - li * M;
  const ImgDesc& d = imgs[cd.img0 + li];
  const CdfBuf x = CdfBuf::at(sm, L);
  const int lg = __ffs(L) - 1;
  const float* src = (src_sel == SEL_Y ? d.y : (src_sel == SEL_UI ? d.uI : d.u)) + (size_t)row * N;
  __shared__ int s_nonzero;
  if (threadIdx.x == 0) s_nonzero = 0;
  __syncthreads();
  bool nz = false;
  for (int n = threadIdx.x; n < L; n += blockDim.x) {
    const float2 v = *reinterpret_cast<const float2*>(src + 2 * n);
    nz |= (v.x != 0.0f) || (v.y != 0.0f);
    x.put(L == 1 ? 0 : bitrev(n, lg), cdf{df{v.x, 0.0f}, df{v.y, 0.0f}});
  }
  if (nz) s_nonzero = 1;
  __syncthreads();
  float2* dhi = reinterpret_cast<float2*>(dhi_sel == SEL_S ? d.S : d.QI);
  float2* dlo = reinterpret_cast<float2*>(dlo_sel == SEL_S ? d.S : d.QI);
  if (!s_nonzero) {  // a zero row (most rows of an embedded PSF) transforms to zero
    for (int k = threadIdx.x; k < L; k += blockDim.x) {
      const size_t o = (size_t)(k / TB) * M * TB + (size_t)row * TB + (k % TB);
      dhi[o] = make_float2(0.0f, 0.0f);
      dlo[o] = make_float2(0.0f, 0.0f);
    }
    return;
  }
  fft_df(x, L, tab, threadIdx.x, blockDim.x);
  for (int k = threadIdx.x; k < L; k += blockDim.x) {
    const cdf Zk = x.get(k);
    cdf X;
    if (k == 0) {
      X = cdf{dfs_add(Zk.re, Zk.im), dfs_sub(Zk.re, Zk.im)};  // X[0] + i X[N/2]
    } else {
      const cdf Zm0 = x.get(L - k);
      const cdf Zm = cdf{Zm0.re, df_neg(Zm0.im)};  // conj Z[L-k]
      const cdf E = cdf_half(cdf_add(Zk, Zm));
      const cdf D = cdf_half(cdf_sub(Zk, Zm));
      const cdf O = cdf{D.im, df_neg(D.re)};  // (Zk - Zm) / (2i)
      X = cdf_add(E, cdf_mul(tw_df(tab, N, k), O));
    }
    const size_t o = (size_t)(k / TB) * M * TB + (size_t)row * TB + (k % TB);
    dhi[o] = make_float2(X.re.hi, X.im.hi);
    dlo[o] = make_float2(X.re.lo, X.im.lo);
  }
}

// Floats per column buffer of the column pass: four padded planes and one
// word of skew, so that the columns of a tile start in different banks.
GFD_HD int df_col_stride(int M) { return 4 * df_plane(M) + 1; }

// Column pass: packed rows (hi in plane shi, lo in plane slo) -> complex
// column transforms rounded once into plane dst.  One block per tile of TB
// columns; threads split over the tile's columns.
__global__ void __launch_bounds__(512)
k_col_df(ClassDesc cd, const ImgDesc* __restrict__ imgs, const float4* __restrict__ tab,
         int shi_sel, int slo_sel, int dst_sel) {
  extern __shared__ float sm[];
  const int M = cd.M, L = cd.N / 2, TB = cd.TB;
  const int tiles = L / TB;
  const int li = blockIdx.x / tiles, t = blockIdx.x - li * tiles;
  const ImgDesc& d = imgs[cd.img0 + li];
  const int lg = __ffs(M) - 1;
  const int cstride = df_col_stride(M);
  const size_t off = (size_t)t * M * TB;
  const float2* shi = reinterpret_cast<const float2*>(shi_sel == SEL_S ? d.S : d.QI) + off;
  const float2* slo = reinterpret_cast<const float2*>(slo_sel == SEL_S ? d.S : d.QI) + off;
  float2* dst = reinterpret_cast<float2*>(dst_sel == SEL_H ? d.H : d.Y) + off;
  for (int e = threadIdx.x; e < M * TB; e += blockDim.x) {
    const int m = e / TB, b = e - m * TB;
    const float2 h = shi[e], l = slo[e];
    const CdfBuf x = CdfBuf::at(sm + b * cstride, M);
    x.put(M == 1 ? 0 : bitrev(m, lg), cdf{df{h.x, l.x}, df{h.y, l.y}});
  }
  __syncthreads();
  // threads per column: the block's threads split evenly over the TB columns
  const int per = blockDim.x / TB;
  const int b = threadIdx.x / per, tt = threadIdx.x - b * per;
  const CdfBuf x = CdfBuf::at(sm + b * cstride, M);
  fft_df(x, M, tab, tt, per, b < TB);
  for (int e = threadIdx.x; e < M * TB; e += blockDim.x) {
    const int m = e / TB, bb = e - m * TB;
    const CdfBuf y = CdfBuf::at(sm + bb * cstride, M);
    const cdf v = y.get(m);
    dst[e] = make_float2(v.re.hi + v.re.lo, v.im.hi + v.im.lo);
  }
}

static int df_sm_count() {
  static int n = 0;
  if (n == 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n <= 0) n = 1;
  }
  return n;
}

// Precise 2-D real DFT of real plane src into spectrum plane dst (SEL_H or
// SEL_YS), using the S and Q_I planes as the double-float intermediate.
cudaError_t launch_fft2_r2c_df(const ClassLaunch& c, const float4* tab, int src, int dst,
                               cudaStream_t s) {
  (void)df_sm_count;
  const int M = c.cd.M, L = c.cd.N / 2, TB = c.cd.TB;
  const int rthreads = L / 4 < 256 ? (L / 4 < 32 ? 32 : L / 4) : 256;
  k_row_r2c_df<<<c.cd.n_img * M, rthreads, (size_t)4 * df_plane(L) * sizeof(float), s>>>(
      c.cd, c.imgs, tab, src, SEL_S, SEL_QI);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  int per = M / 4 < 64 ? M / 4 : 64;
  if (per < 1) per = 1;
  int cthreads = per * TB;
  if (cthreads > 512) cthreads = 512 - 512 % TB;
  if (cthreads < TB) cthreads = TB;
  const size_t smem = (size_t)TB * df_col_stride(M) * sizeof(float);
  k_col_df<<<c.cd.n_img * (L / TB), cthreads, smem, s>>>(c.cd, c.imgs, tab, SEL_S, SEL_QI,
                                                        dst == SEL_H ? SEL_H : SEL_YS);
  return cudaGetLastError();
}

cudaError_t configure_df_kernels() {
  cudaError_t e = cudaFuncSetAttribute(k_col_df, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       160 * 1024);
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(k_row_r2c_df, cudaFuncAttributeMaxDynamicSharedMemorySize, 64 * 1024);
}

}  // namespace gfd
