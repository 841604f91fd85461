// 2-D real DFT passes and the spectral steps of the deblurring solve.
//
// Packed half-spectrum layout (M rows x N/2 complex): S[m][l] = X(m, l) for
// 1 <= l < N/2 and S[m][0] = X(m, 0) + i X(m, N/2), X the full 2-D DFT.  A
// row pass maps each real row to its packed row DFT; a column pass is a plain
// complex FFT down every packed column (column 0 included, since its two real
// row spectra pack into one complex signal).  Bins (m, 0) and (m, N/2) are
// unpacked where a spectral formula needs them.
#include "fft.cuh"
#include "lambda.cuh"
#include "launch.h"

namespace gfd {

GFD_D float* real_plane(const ImgDesc& d, int sel) {
  switch (sel) {
    case SEL_Y: return const_cast<float*>(d.y);
    case SEL_U: return d.u;
    case SEL_S: return reinterpret_cast<float*>(d.S);
    case SEL_QI: return reinterpret_cast<float*>(d.QI);
    case SEL_QP: return reinterpret_cast<float*>(d.Qp);
    case SEL_H: return reinterpret_cast<float*>(d.H);
    default: return reinterpret_cast<float*>(d.Y);
  }
}
GFD_D float2* cplx_plane(const ImgDesc& d, int sel) {
  return reinterpret_cast<float2*>(real_plane(d, sel));
}

constexpr int threads_per_team(int L) { return L / radix_for(L); }

// ---------------------------------------------------------------------------
// Row pass, forward: real rows -> packed row spectra.
// Each row of N reals is read as N/2 complex z[n] = x[2n] + i x[2n+1];
// Z = FFT_{N/2}(z); then X[k] = (Z[k] + conj Z[-k])/2 + W_N^k (Z[k] - conj Z[-k])/(2i)
// and X[0], X[N/2] = Re Z[0] +- Im Z[0] (packed as X[0] + i X[N/2]).
// ---------------------------------------------------------------------------
template <int L>
__global__ void k_row_r2c(ClassDesc cd, const ImgDesc* __restrict__ imgs, ImgState* st,
                          const float2* __restrict__ tw, int rpc, int src_sel, int dst_sel,
                          int do_sum) {
  extern __shared__ float2 smem[];
  constexpr int R = radix_for(L), T = threads_per_team(L);
  constexpr int N = 2 * L;
  const int team = threadIdx.x / T, j = threadIdx.x % T;
  const int row_c = blockIdx.x * rpc + team;  // row within the class
  const int li = row_c / cd.M, row = row_c % cd.M;
  const ImgDesc& d = imgs[cd.img0 + li];
  float2* buf = smem + team * team_stride(L);
  const float2* src = reinterpret_cast<const float2*>(real_plane(d, src_sel)) + (size_t)row * L;
  float part = 0.0f;
#pragma unroll
  for (int i = 0; i < R; ++i) {
    const int n = j + i * T;
    const float2 v = src[n];
    buf[phys(n)] = v;
    part += v.x + v.y;
  }
  if (do_sum) {
    // FP32 within a warp, FP64 across warps
    double* red = reinterpret_cast<double*>(smem + rpc * team_stride(L));
    part = warp_sum(part);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = (double)part;
    __syncthreads();
    if (threadIdx.x == 0) {
      double s = 0.0;
      for (int w = 0; w < num_warps(); ++w) s += red[w];
      atomicAdd(&st[cd.img0 + li].sum_u, s);
    }
  }
  __syncthreads();
  fft_team<L, false>(buf, j, tw);
  float2* dst = cplx_plane(d, dst_sel) + (size_t)row * L;
#pragma unroll
  for (int i = 0; i < R; ++i) {
    const int k = j + i * T;
    const float2 Zk = buf[phys(out_pos<L>(k))];
    float2 out;
    if (k == 0) {
      out = make_float2(Zk.x + Zk.y, Zk.x - Zk.y);
    } else {
      const float2 Zm = cconj(buf[phys(out_pos<L>(L - k))]);
      const float2 E = cscale(cadd(Zk, Zm), 0.5f);
      const float2 D = csub(Zk, Zm);
      const float2 O = make_float2(0.5f * D.y, -0.5f * D.x);  // D / (2i)
      out = cadd(E, cmul(__ldg(&tw[k * (TW_N / N)]), O));
    }
    dst[k] = out;
  }
}

// ---------------------------------------------------------------------------
// Row pass, inverse, in place: packed row spectra -> real rows (scaled).
// Z[k] = (R[k] + conj R[L-k]) + i (R[k] - conj R[L-k]) W_N^{-k}, with
// R[0], R[N/2] the real and imaginary parts of the packed entry 0; the
// unnormalised inverse FFT of Z gives x[2n] + i x[2n+1] times N.
// ---------------------------------------------------------------------------
template <int L>
__global__ void k_row_c2r(ClassDesc cd, const ImgDesc* __restrict__ imgs,
                          const float2* __restrict__ tw, int rpc, int sel0, int sel1,
                          float scale) {
  extern __shared__ float2 smem[];
  constexpr int R = radix_for(L), T = threads_per_team(L);
  constexpr int N = 2 * L;
  const int team = threadIdx.x / T, j = threadIdx.x % T;
  int blk = blockIdx.x;
  int sel = sel0;
  const int nblk_plane = cd.n_img * cd.M / rpc;
  if (blk >= nblk_plane) {
    blk -= nblk_plane;
    sel = sel1;
  }
  const int row_c = blk * rpc + team;
  const int li = row_c / cd.M, row = row_c % cd.M;
  const ImgDesc& d = imgs[cd.img0 + li];
  float2* buf = smem + team * team_stride(L);
  float2* rowp = cplx_plane(d, sel) + (size_t)row * L;
#pragma unroll
  for (int i = 0; i < R; ++i) {
    const int n = j + i * T;
    buf[phys(n)] = rowp[n];
  }
  __syncthreads();
  for (int k = j; k <= L / 2; k += T) {
    if (k == 0) {
      const float2 t0 = buf[phys(0)];
      buf[phys(0)] = make_float2(t0.x + t0.y, t0.x - t0.y);
    } else {
      const int km = L - k;
      const float2 Rk = buf[phys(k)], Rm = buf[phys(km)];
      {
        const float2 E = cadd(Rk, cconj(Rm));
        const float2 O = cmul(csub(Rk, cconj(Rm)), cconj(__ldg(&tw[k * (TW_N / N)])));
        buf[phys(k)] = make_float2(E.x - O.y, E.y + O.x);
      }
      if (km != k) {
        const float2 E = cadd(Rm, cconj(Rk));
        const float2 O = cmul(csub(Rm, cconj(Rk)), cconj(__ldg(&tw[km * (TW_N / N)])));
        buf[phys(km)] = make_float2(E.x - O.y, E.y + O.x);
      }
    }
  }
  __syncthreads();
  fft_team<L, true>(buf, j, tw);
#pragma unroll
  for (int i = 0; i < R; ++i) {
    const int n = j + i * T;
    rowp[n] = cscale(buf[phys(out_pos<L>(n))], scale);
  }
}

// ---------------------------------------------------------------------------
// Column passes.  A block owns B adjacent packed columns of one image; team b
// (threads b, b+B, ...) transforms column c0+b, so that a warp's global
// accesses cover B consecutive complex values of a row.
// ---------------------------------------------------------------------------
template <int M, bool INV>
__global__ void k_col_plain(ClassDesc cd, const ImgDesc* __restrict__ imgs,
                            const float2* __restrict__ tw, int B, int src_sel, int dst_sel) {
  extern __shared__ float2 smem[];
  constexpr int R = radix_for(M), T = threads_per_team(M);
  const int Lc = cd.N / 2;
  const int cpi = Lc / B;
  const ImgDesc& d = imgs[cd.img0 + blockIdx.x / cpi];
  const int c0 = (blockIdx.x % cpi) * B;
  const int b = threadIdx.x & (B - 1), j = threadIdx.x / B;
  float2* buf = smem + b * team_stride(M);
  const float2* src = cplx_plane(d, src_sel) + c0 + b;
  float2* dst = cplx_plane(d, dst_sel) + c0 + b;
#pragma unroll
  for (int i = 0; i < R; ++i) {
    const int a = j + i * T;
    buf[phys(a)] = src[(size_t)a * Lc];
  }
  __syncthreads();
  fft_team<M, INV>(buf, j, tw);
#pragma unroll
  for (int i = 0; i < R; ++i) {
    const int k = j + i * T;
    dst[(size_t)k * Lc] = buf[phys(out_pos<M>(k))];
  }
}

// unpack bins (k, 0) and (k, N/2) from packed column values S[k], S[-k]
GFD_D void unpack_pair(float2 Sk, float2 Smk, float2& A, float2& Bv) {
  const float2 c = cconj(Smk);
  A = cscale(cadd(Sk, c), 0.5f);
  const float2 D = csub(Sk, c);
  Bv = make_float2(0.5f * D.y, -0.5f * D.x);  // D / (2i)
}

// Forward column FFT of the iterate's row spectra (in place on S), fused with
// the first evaluation of Eq. 11 at the nodes of the image's bracket.
template <int M>
__global__ void __launch_bounds__(256) k_col_fwd_lambda(ClassDesc cd, const ImgDesc* __restrict__ imgs,
                                 ImgState* st, const float2* __restrict__ tw, int B,
                                 int iter) {
  extern __shared__ float2 smem[];
  constexpr int R = radix_for(M), T = threads_per_team(M);
  __shared__ float s_nodes[KNODES];
  __shared__ int s_flag;
  const int Lc = cd.N / 2;
  const int cpi = Lc / B;
  const int gi = cd.img0 + blockIdx.x / cpi;
  const ImgDesc& d = imgs[gi];
  ImgState* S = st + gi;
  const int c0 = (blockIdx.x % cpi) * B;
  const int b = threadIdx.x & (B - 1), j = threadIdx.x / B;
  const int col = c0 + b;
  float2* buf = smem + b * team_stride(M);
  float2* spec = d.S + col;
  for (int q = threadIdx.x; q < KNODES; q += blockDim.x) s_nodes[q] = __ldcg(&S->node[q]);
#pragma unroll
  for (int i = 0; i < R; ++i) {
    const int a = j + i * T;
    buf[phys(a)] = spec[(size_t)a * Lc];
  }
  __syncthreads();
  fft_team<M, false>(buf, j, tw);
  float nodes[KNODES];
#pragma unroll
  for (int q = 0; q < KNODES; ++q) nodes[q] = s_nodes[q];
  float acc[KNODES + 1];
#pragma unroll
  for (int q = 0; q <= KNODES; ++q) acc[q] = 0.0f;
  if (col != 0) {
    const float2* Hc = d.H + col;
    const float2* Yc = d.Y + col;
#pragma unroll 4
    for (int i = 0; i < R; ++i) {
      const int k = j + i * T;
      const float2 U = buf[phys(out_pos<M>(k))];
      spec[(size_t)k * Lc] = U;
      const float2 H = __ldg(&Hc[(size_t)k * Lc]);
      const float2 Y = __ldg(&Yc[(size_t)k * Lc]);
      const float2 r = csub(cmul(H, U), Y);
      const float rr = fmaf(r.x, r.x, r.y * r.y);
      const float a = fmaf(H.x, H.x, H.y * H.y);
      accum_bin(2.0f * rr, a, nodes, acc);  // bins l and N-l
    }
  } else {
    for (int i = 0; i < R; ++i) {
      const int k = j + i * T;
      float2 U = buf[phys(out_pos<M>(k))];
      const float2 Um = buf[phys(out_pos<M>((M - k) & (M - 1)))];
      float2 UA, UB;
      unpack_pair(U, Um, UA, UB);
      const float2 HA = d.H0[k], HB = d.HN[k], YA = d.Y0[k], YB = d.YN[k];
      float rA;
      if (k == 0) {
        // DC bin in FP64 from exact sums: d00 = sum(h) sum(u_E) - sum(y)
        const double su = __ldcg(&S->sum_u);
        const double d00 = S->sum_h * su - S->sum_y;
        S->d00 = d00;
        rA = (float)(d00 * d00);
        U.x = (float)su;
      } else {
        const float2 r = csub(cmul(HA, UA), YA);
        rA = fmaf(r.x, r.x, r.y * r.y);
      }
      const float2 rb = csub(cmul(HB, UB), YB);
      accum_bin(rA, fmaf(HA.x, HA.x, HA.y * HA.y), nodes, acc);
      accum_bin(fmaf(rb.x, rb.x, rb.y * rb.y), fmaf(HB.x, HB.x, HB.y * HB.y), nodes, acc);
      spec[(size_t)k * Lc] = U;
    }
  }
  double* red = reinterpret_cast<double*>(smem + B * team_stride(M));
  __syncthreads();
  block_accumulate(acc, red, S);
  if (last_block(&S->cta_done, cpi, &s_flag)) {
    if (threadIdx.x == 0) {
      lambda_update(S, (double)cd.M * cd.N, true, false, iter, d.lam_out, d.res_out);
      S->cta_done = 0;
      __threadfence();
    }
  }
}

// Fallback evaluation of Eq. 11 over the stored spectrum U_E for images whose
// root is still open; a block covers `chunk` packed elements of one image.
__global__ void __launch_bounds__(256) k_lambda_pass(ClassDesc cd, const ImgDesc* __restrict__ imgs, ImgState* st,
                              int chunk, int iter, int last_chance) {
  __shared__ float s_nodes[KNODES];
  __shared__ double red[32 * (KNODES + 1)];
  __shared__ int s_flag;
  const int Lc = cd.N / 2;
  const int per_img = cd.M * Lc;
  const int cpi = per_img / chunk;
  const int gi = cd.img0 + blockIdx.x / cpi;
  ImgState* S = st + gi;
  if (__ldcg(&S->need) == 0) return;
  const ImgDesc& d = imgs[gi];
  for (int q = threadIdx.x; q < KNODES; q += blockDim.x) s_nodes[q] = __ldcg(&S->node[q]);
  __syncthreads();
  float nodes[KNODES];
#pragma unroll
  for (int q = 0; q < KNODES; ++q) nodes[q] = s_nodes[q];
  float acc[KNODES + 1];
#pragma unroll
  for (int q = 0; q <= KNODES; ++q) acc[q] = 0.0f;
  const int e0 = (blockIdx.x % cpi) * chunk;
  const int M = cd.M;
  for (int e = e0 + threadIdx.x; e < e0 + chunk; e += blockDim.x) {
    const int k = e / Lc, col = e - k * Lc;
    const float2 U = d.S[e];
    if (col != 0) {
      const float2 H = __ldg(&d.H[e]), Y = __ldg(&d.Y[e]);
      const float2 r = csub(cmul(H, U), Y);
      accum_bin(2.0f * fmaf(r.x, r.x, r.y * r.y), fmaf(H.x, H.x, H.y * H.y), nodes, acc);
    } else {
      const float2 Um = d.S[(size_t)((M - k) & (M - 1)) * Lc];
      float2 UA, UB;
      unpack_pair(U, Um, UA, UB);
      const float2 HA = d.H0[k], HB = d.HN[k], YA = d.Y0[k], YB = d.YN[k];
      float rA;
      if (k == 0) {
        const double d00 = __ldcg(&S->d00);
        rA = (float)(d00 * d00);
      } else {
        const float2 r = csub(cmul(HA, UA), YA);
        rA = fmaf(r.x, r.x, r.y * r.y);
      }
      const float2 rb = csub(cmul(HB, UB), YB);
      accum_bin(rA, fmaf(HA.x, HA.x, HA.y * HA.y), nodes, acc);
      accum_bin(fmaf(rb.x, rb.x, rb.y * rb.y), fmaf(HB.x, HB.x, HB.y * HB.y), nodes, acc);
    }
  }
  block_accumulate(acc, red, S);
  if (last_block(&S->cta_done, cpi, &s_flag)) {
    if (threadIdx.x == 0) {
      lambda_update(S, (double)cd.M * cd.N, false, last_chance != 0, iter, d.lam_out, d.res_out);
      S->cta_done = 0;
      __threadfence();
    }
  }
}

// Eq. 9 (u_p) and Eq. 8 (u_I) at one bin:
//   U_p = (conj(H) Y + lam U_E) / (|H|^2 + lam)
//   U_I = (conj(H) Y + lam D2 U_E) / (|H|^2 + lam D2),  D2 = |F(nabla)|^2.
GFD_D void solve_bin(float2 U, float2 H, float2 Y, float lam, float D2, bool branch,
                     float2& UI, float2& Up) {
  if (branch) {  // lambda = inf: u_I = u_p = u_E (Sec. 3.2)
    UI = U;
    Up = U;
    return;
  }
  const float2 HY = make_float2(fmaf(H.x, Y.x, H.y * Y.y), fmaf(H.x, Y.y, -H.y * Y.x));
  const float a = fmaf(H.x, H.x, H.y * H.y);
  const float ip = __frcp_rn(a + lam);
  Up = make_float2(fmaf(lam, U.x, HY.x) * ip, fmaf(lam, U.y, HY.y) * ip);
  const float lg = lam * D2;
  const float den = a + lg;
  if (den > 0.0f) {
    const float ii = __frcp_rn(den);
    UI = make_float2(fmaf(lg, U.x, HY.x) * ii, fmaf(lg, U.y, HY.y) * ii);
  } else {
    UI = U;
  }
}

template <int M>
__global__ void __launch_bounds__(256) k_col_solve_inv(ClassDesc cd, const ImgDesc* __restrict__ imgs,
                                const ImgState* st, const float2* __restrict__ tw,
                                const float* __restrict__ d2tab, int B) {
  extern __shared__ float2 smem[];
  constexpr int R = radix_for(M), T = threads_per_team(M);
  const int N = cd.N, Lc = N / 2;
  const int cpi = Lc / B;
  const int gi = cd.img0 + blockIdx.x / cpi;
  const ImgDesc& d = imgs[gi];
  const int c0 = (blockIdx.x % cpi) * B;
  const int b = threadIdx.x & (B - 1), j = threadIdx.x / B;
  const int col = c0 + b;
  float2* bufI = smem + b * team_stride(M);
  float2* bufP = smem + (B + b) * team_stride(M);
  const double lamd = __ldcg(&st[gi].lam);
  const bool branch = !(lamd < 1e300);
  const float lam = branch ? 0.0f : (float)lamd;
  const int nstep = TW_N / N;  // d2tab stride for the column frequency
  const float d2c = __ldg(&d2tab[col * nstep]);
#pragma unroll 4
  for (int i = 0; i < R; ++i) {
    const int k = j + i * T;
    const size_t e = (size_t)k * Lc + col;
    const float d2r = __ldg(&d2tab[k * (TW_N / M)]);
    const float2 U = d.S[e];
    float2 UI, Up;
    if (col != 0) {
      solve_bin(U, __ldg(&d.H[e]), __ldg(&d.Y[e]), lam, d2r + d2c, branch, UI, Up);
    } else {
      const float2 Um = d.S[(size_t)((M - k) & (M - 1)) * Lc];
      float2 UA, UB, IA, IB, PA, PB;
      unpack_pair(U, Um, UA, UB);
      solve_bin(UA, d.H0[k], d.Y0[k], lam, d2r, branch, IA, PA);
      solve_bin(UB, d.HN[k], d.YN[k], lam, d2r + 4.0f, branch, IB, PB);
      UI = make_float2(IA.x - IB.y, IA.y + IB.x);  // A + i B
      Up = make_float2(PA.x - PB.y, PA.y + PB.x);
    }
    bufI[phys(k)] = UI;
    bufP[phys(k)] = Up;
  }
  __syncthreads();
  fft_team<M, true>(bufI, j, tw);
  fft_team<M, true>(bufP, j, tw);
  float2* qi = d.QI + col;
  float2* qp = d.Qp + col;
#pragma unroll
  for (int i = 0; i < R; ++i) {
    const int k = j + i * T;
    const int p = phys(out_pos<M>(k));
    qi[(size_t)k * Lc] = bufI[p];
    qp[(size_t)k * Lc] = bufP[p];
  }
}

// ---------------------------------------------------------------------------
// launch configuration and dispatch
// ---------------------------------------------------------------------------
// Largest block the kernel can be launched with (registers permitting),
// queried once per kernel.
template <class K>
static int max_threads(K kernel) {
  static int cached = 0;
  if (cached == 0) {
    cudaFuncAttributes a{};
    cached = cudaFuncGetAttributes(&a, (const void*)kernel) == cudaSuccess ? a.maxThreadsPerBlock : 256;
  }
  return cached;
}

static int rows_per_block(int L, int M) {
  const int T = threads_per_team(L);
  int r = 256 / T;
  if (r < 1) r = 1;
  if (r > M) r = M;
  return r;
}

static int cols_per_block(int M, int Lc, int target_threads, int max_threads) {
  const int T = threads_per_team(M);
  if (target_threads > max_threads) target_threads = max_threads;
  int B = target_threads / T;
  if (B < 1) B = 1;
  if (B > Lc) B = Lc;
  return B;
}

static size_t row_smem(int L, int rpc) {
  return (size_t)rpc * team_stride(L) * sizeof(float2) + 32 * sizeof(double);
}

#define GFD_CASE_L(F, ...)             \
  case 4: F<4>(__VA_ARGS__); break;     \
  case 8: F<8>(__VA_ARGS__); break;     \
  case 16: F<16>(__VA_ARGS__); break;   \
  case 32: F<32>(__VA_ARGS__); break;   \
  case 64: F<64>(__VA_ARGS__); break;   \
  case 128: F<128>(__VA_ARGS__); break; \
  case 256: F<256>(__VA_ARGS__); break; \
  case 512: F<512>(__VA_ARGS__); break; \
  case 1024: F<1024>(__VA_ARGS__); break; \
  case 2048: F<2048>(__VA_ARGS__); break;

#define GFD_CASE_M(F, ...)               \
  case 8: F<8>(__VA_ARGS__); break;       \
  case 16: F<16>(__VA_ARGS__); break;     \
  case 32: F<32>(__VA_ARGS__); break;     \
  case 64: F<64>(__VA_ARGS__); break;     \
  case 128: F<128>(__VA_ARGS__); break;   \
  case 256: F<256>(__VA_ARGS__); break;   \
  case 512: F<512>(__VA_ARGS__); break;   \
  case 1024: F<1024>(__VA_ARGS__); break; \
  case 2048: F<2048>(__VA_ARGS__); break; \
  case 4096: F<4096>(__VA_ARGS__); break;

template <int L>
static void do_row_r2c(const ClassLaunch& c, const Tables& t, int src, int dst, int sum,
                       cudaStream_t s) {
  const int rpc = rows_per_block(L, c.cd.M);
  const int nblk = c.cd.n_img * c.cd.M / rpc;
  k_row_r2c<L><<<nblk, rpc * threads_per_team(L), row_smem(L, rpc), s>>>(
      c.cd, c.imgs, c.st, t.tw, rpc, src, dst, sum);
}

cudaError_t launch_row_r2c(const ClassLaunch& c, const Tables& t, int src, int dst,
                           bool do_sum, cudaStream_t s) {
  switch (c.cd.N / 2) {
    GFD_CASE_L(do_row_r2c, c, t, src, dst, do_sum ? 1 : 0, s)
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

template <int L>
static void do_row_c2r(const ClassLaunch& c, const Tables& t, int sel0, int sel1, float scale,
                       cudaStream_t s) {
  const int rpc = rows_per_block(L, c.cd.M);
  int nblk = c.cd.n_img * c.cd.M / rpc;
  if (sel1 >= 0) nblk *= 2;
  k_row_c2r<L><<<nblk, rpc * threads_per_team(L), row_smem(L, rpc), s>>>(
      c.cd, c.imgs, t.tw, rpc, sel0, sel1, scale);
}

cudaError_t launch_row_c2r(const ClassLaunch& c, const Tables& t, int sel0, int sel1,
                           float scale, cudaStream_t s) {
  switch (c.cd.N / 2) {
    GFD_CASE_L(do_row_c2r, c, t, sel0, sel1, scale, s)
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

template <int M>
static void do_col_plain(const ClassLaunch& c, const Tables& t, int src, int dst, bool inv,
                         cudaStream_t s) {
  const int Lc = c.cd.N / 2;
  const int B = cols_per_block(M, Lc, 512,
                               inv ? max_threads(k_col_plain<M, true>) : max_threads(k_col_plain<M, false>));
  const size_t smem = (size_t)B * team_stride(M) * sizeof(float2);
  const int nblk = c.cd.n_img * (Lc / B);
  if (inv)
    k_col_plain<M, true><<<nblk, B * threads_per_team(M), smem, s>>>(c.cd, c.imgs, t.tw, B, src, dst);
  else
    k_col_plain<M, false><<<nblk, B * threads_per_team(M), smem, s>>>(c.cd, c.imgs, t.tw, B, src, dst);
}

cudaError_t launch_col_plain(const ClassLaunch& c, const Tables& t, int src, int dst,
                             bool inverse, cudaStream_t s) {
  switch (c.cd.M) {
    GFD_CASE_M(do_col_plain, c, t, src, dst, inverse, s)
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

template <int M>
static void do_col_fwd_lambda(const ClassLaunch& c, const Tables& t, int iter, cudaStream_t s) {
  const int Lc = c.cd.N / 2;
  const int B = cols_per_block(M, Lc, 256, max_threads(k_col_fwd_lambda<M>));
  const int nthr = B * threads_per_team(M);
  const size_t smem = (size_t)B * team_stride(M) * sizeof(float2) +
                      (size_t)((nthr + 31) / 32) * (KNODES + 1) * sizeof(double);
  const int nblk = c.cd.n_img * (Lc / B);
  k_col_fwd_lambda<M><<<nblk, nthr, smem, s>>>(c.cd, c.imgs, c.st, t.tw, B, iter);
}

cudaError_t launch_col_fwd_lambda(const ClassLaunch& c, const Tables& t, int iter,
                                  cudaStream_t s) {
  switch (c.cd.M) {
    GFD_CASE_M(do_col_fwd_lambda, c, t, iter, s)
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

cudaError_t launch_lambda_pass(const ClassLaunch& c, int iter, bool last_chance,
                               cudaStream_t s) {
  const int per_img = c.cd.M * (c.cd.N / 2);
  const int chunk = per_img < 4096 ? per_img : 4096;
  const int nblk = c.cd.n_img * (per_img / chunk);
  k_lambda_pass<<<nblk, 256, 0, s>>>(c.cd, c.imgs, c.st, chunk, iter, last_chance ? 1 : 0);
  return cudaGetLastError();
}

template <int M>
static void do_col_solve_inv(const ClassLaunch& c, const Tables& t, cudaStream_t s) {
  const int Lc = c.cd.N / 2;
  const int B = cols_per_block(M, Lc, 256, max_threads(k_col_solve_inv<M>));
  const size_t smem = (size_t)2 * B * team_stride(M) * sizeof(float2);
  const int nblk = c.cd.n_img * (Lc / B);
  k_col_solve_inv<M><<<nblk, B * threads_per_team(M), smem, s>>>(c.cd, c.imgs, c.st, t.tw,
                                                                   t.d2, B);
}

cudaError_t launch_col_solve_inv(const ClassLaunch& c, const Tables& t, cudaStream_t s) {
  switch (c.cd.M) {
    GFD_CASE_M(do_col_solve_inv, c, t, s)
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
template <int L>
static cudaError_t cfg_row() {
  cudaError_t e = cudaFuncSetAttribute(k_row_r2c<L>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(k_row_c2r<L>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
}
template <int M>
static cudaError_t cfg_col() {
  cudaError_t e;
  if ((e = cudaFuncSetAttribute(k_col_plain<M, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024)) != cudaSuccess) return e;
  if ((e = cudaFuncSetAttribute(k_col_plain<M, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024)) != cudaSuccess) return e;
  if ((e = cudaFuncSetAttribute(k_col_fwd_lambda<M>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024)) != cudaSuccess) return e;
  return cudaFuncSetAttribute(k_col_solve_inv<M>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
}

cudaError_t configure_fft_kernels() {
  cudaError_t e;
#define GFD_CFG(x) if ((e = (x)) != cudaSuccess) return e;
  GFD_CFG(cfg_row<4>()) GFD_CFG(cfg_row<8>()) GFD_CFG(cfg_row<16>()) GFD_CFG(cfg_row<32>())
  GFD_CFG(cfg_row<64>()) GFD_CFG(cfg_row<128>()) GFD_CFG(cfg_row<256>()) GFD_CFG(cfg_row<512>())
  GFD_CFG(cfg_row<1024>()) GFD_CFG(cfg_row<2048>())
  GFD_CFG(cfg_col<8>()) GFD_CFG(cfg_col<16>()) GFD_CFG(cfg_col<32>()) GFD_CFG(cfg_col<64>())
  GFD_CFG(cfg_col<128>()) GFD_CFG(cfg_col<256>()) GFD_CFG(cfg_col<512>()) GFD_CFG(cfg_col<1024>())
  GFD_CFG(cfg_col<2048>()) GFD_CFG(cfg_col<4096>())
#undef GFD_CFG
  return cudaSuccess;
}

}  // namespace gfd
