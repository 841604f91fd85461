// Reverse mode of the unrolled method: gradients of a loss of u^K with
// respect to the observation y, the PSF h and the guided filter's eps.
//
// One backward step undoes one iteration (Sec. 3.1 Steps 1-2), in reverse
// order of the forward step, from its checkpoint u_E^k and the forward
// solve's lambda_k:
//   recompute: U_E = DFT(u_E^k), U_I and U_p by Eq. 8-9, u_I and u_p by the
//     inverse DFT;
//   guided filter (Eq. 3-5; periodic windows, so the box mean is its own
//   adjoint): three tiled passes of compensated window sums
//     1. mu, pbar, sigma^2 + eps, a from (u_I, u_p)
//     2. window sums of a, g_u u_I, g_u -> the pointwise adjoints of Eq. 5, 4, 3
//     3. window sums of those adjoints -> g_uI, g_up
//   DFT of g_uI, g_up; the spectral solves (Eq. 8-9) per bin, with lambda's
//   adjoint summed over the bins; the implicit derivative of lambda through
//   Eq. 11 (dlambda = -(df - dT) / f'(lambda)) as a second per-bin pass; the
//   adjoint DFT back to g_uE = g_u of the previous step.
// H = DFT(embedded h), Y = DFT(y) and T (Eq. 12) collect their gradients over
// the steps; the last kernels map them to g_h, g_y.  Where lambda = inf the
// step is u_I = u_p = u_E and lambda is a constant.
//
// Arithmetic: FP32 per pixel and per bin, as in the forward step; the window
// sums carry their rounding errors (a running FP32 sum plus the exact error of
// every addition and product, summed apart), and the statistics that cancel
// (sigma^2, the covariance, box(g_u I) - mu box(g_u), the combinations of
// pass 3) are formed from them in double-float; sums over all bins or pixels
// are FP64.  No FP64 arithmetic per pixel: this part's FP64 rate is a small
// fraction of its FP32 rate.
//
// Spectra are the library's packed half spectra, row-major (tile width N/2):
// Z[m][l] = X(m, l) for 1 <= l < N/2 and Z[m][0] = X(m, 0) + i X(m, N/2).
// Complex gradients follow g_z = dL/dRe z + i dL/dIm z; a sum over all bins
// counts the interior columns twice (each stands for its mirror bin too).
#include "common.cuh"
#include "df.cuh"
#include "launch.h"
#include "spectral.cuh"

namespace gfd {

constexpr int ADJ_TILE = 16;

// A compensated sum: hi is the FP32 running sum, lo the sum of the exact
// rounding errors of its additions (and of the low parts of added
// double-float terms).  hi + lo carries about 2^-48 relative error per term.
struct CSum {
  float hi, lo;
};
GFD_D void csum_add(CSum& s, df x) {
  const df t = two_sum(s.hi, x.hi);
  s.hi = t.hi;
  s.lo += t.lo + x.lo;
}
GFD_D df csum_df(CSum s) { return quick_two_sum(s.hi, s.lo); }  // |lo| <= |hi| in practice
GFD_D df val_df(float v) { return df{v, 0.0f}; }

// ---------------------------------------------------------------------------
// Tiled window sums: OP stages NS planes of a TILE x TILE tile plus an r halo
// in shared memory, maps every staged pixel to NQ double-float quantities,
// and gets their compensated window sums (periodic windows) at each output
// pixel: along the tile's rows into shared memory, then down its columns.
// ---------------------------------------------------------------------------
template <class OP>
__global__ void __launch_bounds__(ADJ_TILE * ADJ_TILE)
k_adj_box(const AdjDesc* __restrict__ descs, int M, int N, int rad) {
  extern __shared__ __align__(16) unsigned char adj_sm[];
  constexpr int NS = OP::NS, NQ = OP::NQ;
  const AdjDesc& d = descs[blockIdx.z];
  const int E = ADJ_TILE + 2 * rad;
  float2* rows = reinterpret_cast<float2*>(adj_sm);                           // [E][T][NQ]
  float* tile = reinterpret_cast<float*>(rows + (size_t)E * ADJ_TILE * NQ);   // [NS][E][E]
  const int x0 = blockIdx.x * ADJ_TILE, y0 = blockIdx.y * ADJ_TILE;
  for (int e = threadIdx.x; e < E * E; e += blockDim.x) {
    const int ty = e / E, tx = e - ty * E;
    const size_t off = (size_t)((y0 - rad + ty) & (M - 1)) * N + ((x0 - rad + tx) & (N - 1));
#pragma unroll
    for (int c = 0; c < NS; ++c) tile[c * E * E + e] = __ldg(&OP::plane(d, c)[off]);
  }
  __syncthreads();
  for (int e = threadIdx.x; e < E * ADJ_TILE; e += blockDim.x) {
    const int ty = e / ADJ_TILE, tx = e - ty * ADJ_TILE;
    CSum s[NQ];
#pragma unroll
    for (int q = 0; q < NQ; ++q) s[q] = CSum{0.0f, 0.0f};
    for (int dx = 0; dx <= 2 * rad; ++dx) {
      const int o = ty * E + tx + dx;
      float v[NS];
#pragma unroll
      for (int c = 0; c < NS; ++c) v[c] = tile[c * E * E + o];
      df q[NQ];
      OP::quantities(v, q);
#pragma unroll
      for (int k = 0; k < NQ; ++k) csum_add(s[k], q[k]);
    }
#pragma unroll
    for (int q = 0; q < NQ; ++q) rows[(size_t)e * NQ + q] = make_float2(s[q].hi, s[q].lo);
  }
  __syncthreads();
  const int tx = threadIdx.x % ADJ_TILE, ty = threadIdx.x / ADJ_TILE;
  const int gy = y0 + ty, gx = x0 + tx;
  CSum S[NQ];
#pragma unroll
  for (int q = 0; q < NQ; ++q) S[q] = CSum{0.0f, 0.0f};
  for (int dy = 0; dy <= 2 * rad; ++dy) {
    const float2* rr = rows + ((size_t)(ty + dy) * ADJ_TILE + tx) * NQ;
#pragma unroll
    for (int q = 0; q < NQ; ++q) csum_add(S[q], df{rr[q].x, rr[q].y});
  }
  df W[NQ];
#pragma unroll
  for (int q = 0; q < NQ; ++q) W[q] = csum_df(S[q]);  // window sums
  const float n = (float)((2 * rad + 1) * (2 * rad + 1));
  float eps_part = 0.0f;
  if (gy < M && gx < N) eps_part = OP::output(d, (size_t)gy * N + gx, W, n);
  if (OP::kEps) {  // sum of the pass's eps adjoint over the block (FP64), one atomic
    __shared__ double red[ADJ_TILE * ADJ_TILE / 32];
    double v = eps_part;
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
      double t = 0.0;
      for (int w = 0; w < ADJ_TILE * ADJ_TILE / 32; ++w) t += red[w];
      atomicAdd(d.g_eps, t);
    }
  }
}

GFD_D float df_float(df a) { return a.hi + a.lo; }

// Pass 1: mu = box(I), pbar = box(p), sigma^2 + eps, a (Eq. 3), with
// sigma^2 = (n S_II - S_I^2) / n^2 and cov = (n S_Ip - S_I S_p) / n^2.
struct AdjStats {
  static constexpr int NS = 2, NQ = 4;
  static constexpr bool kEps = false;
  GFD_D static const float* plane(const AdjDesc& d, int c) { return c == 0 ? d.uI : d.up; }
  GFD_D static void quantities(const float (&v)[NS], df (&q)[NQ]) {
    q[0] = val_df(v[0]);
    q[1] = val_df(v[1]);
    q[2] = two_prod(v[0], v[1]);
    q[3] = two_prod(v[0], v[0]);
  }
  GFD_D static float output(const AdjDesc& d, size_t o, const df (&S)[NQ], float n) {
    const float inv_n = 1.0f / n, inv2 = inv_n * inv_n;
    const float mu = df_float(S[0]) * inv_n, pb = df_float(S[1]) * inv_n;
    const float var = df_float(df_sub(df_mul_f(S[3], n), df_mul(S[0], S[0]))) * inv2;
    const float cov = df_float(df_sub(df_mul_f(S[2], n), df_mul(S[0], S[1]))) * inv2;
    const float ve = var + (float)d.eps;  // sigma_k^2 + eps
    d.A[o] = cov / ve;
    d.MU[o] = mu;
    d.PB[o] = pb;
    d.VE[o] = ve;
    return 0.0f;
  }
};

// Pass 2: abar, box(g_u I), box(g_u) -> adjoints of Eq. 5 (u = abar I + bbar),
// Eq. 4 (b = pbar - a mu) and Eq. 3 (a = cov / (var + eps)), and eps's.
struct AdjPoint {
  static constexpr int NS = 3, NQ = 3;
  static constexpr bool kEps = true;
  GFD_D static const float* plane(const AdjDesc& d, int c) {
    return c == 0 ? d.A : (c == 1 ? d.gu : d.uI);
  }
  GFD_D static void quantities(const float (&v)[NS], df (&q)[NQ]) {
    q[0] = val_df(v[0]);
    q[1] = two_prod(v[1], v[2]);
    q[2] = val_df(v[1]);
  }
  GFD_D static float output(const AdjDesc& d, size_t o, const df (&S)[NQ], float n) {
    const float inv_n = 1.0f / n;
    const float a = d.A[o], mu = d.MU[o], pb = d.PB[o], ve = d.VE[o];
    const float abar = df_float(S[0]) * inv_n, g_b = df_float(S[2]) * inv_n;
    const float gI0 = d.gu[o] * abar;                                       // u = abar I + bbar
    const float g_a = df_float(df_sub(S[1], df_mul_f(S[2], mu))) * inv_n;  // b = pbar - a mu
    const float iv = 1.0f / ve;
    const float g_cov = g_a * iv, g_var = -g_a * a * iv;                   // a = cov / (var + eps)
    // cov = m_Ip - mu pbar, var = m_II - mu^2
    const float g_mu = -a * g_b - pb * g_cov - 2.0f * mu * g_var;
    const float g_pb = g_b - mu * g_cov;
    d.GI0[o] = gI0;
    d.GCOV[o] = g_cov;
    d.GVAR[o] = g_var;
    d.GMU[o] = g_mu;
    d.GPB[o] = g_pb;
    return g_var;  // d(var + eps)/d eps = 1
  }
};

// Pass 3: window sums of the Eq. 3-4 adjoints -> g_uI, g_up.
struct AdjInputs {
  static constexpr int NS = 4, NQ = 4;
  static constexpr bool kEps = false;
  GFD_D static const float* plane(const AdjDesc& d, int c) {
    return c == 0 ? d.GCOV : (c == 1 ? d.GVAR : (c == 2 ? d.GMU : d.GPB));
  }
  GFD_D static void quantities(const float (&v)[NS], df (&q)[NQ]) {
#pragma unroll
    for (int k = 0; k < NQ; ++k) q[k] = val_df(v[k]);
  }
  GFD_D static float output(const AdjDesc& d, size_t o, const df (&S)[NQ], float n) {
    const float inv_n = 1.0f / n;
    const float I = d.uI[o], p = d.up[o];
    // m_Ip, m_II and mu terms: p box(g_cov) + 2 I box(g_var) + box(g_mu)
    const df tI = df_add(df_add(df_mul_f(S[0], p), df_mul_f(S[1], 2.0f * I)), S[2]);
    const df tp = df_add(df_mul_f(S[0], I), S[3]);  // m_Ip and pbar terms
    d.guI[o] = d.GI0[o] + df_float(tI) * inv_n;
    d.gup[o] = df_float(tp) * inv_n;
    return 0.0f;
  }
};

template <class OP>
static cudaError_t launch_adj_box(const AdjDesc* descs, int n, int M, int N, int rad,
                                  cudaStream_t s) {
  const int E = ADJ_TILE + 2 * rad;
  const size_t smem = (size_t)E * ADJ_TILE * OP::NQ * sizeof(float2) +
                      (size_t)OP::NS * E * E * sizeof(float);
  const dim3 grid((N + ADJ_TILE - 1) / ADJ_TILE, (M + ADJ_TILE - 1) / ADJ_TILE, n);
  k_adj_box<OP><<<grid, ADJ_TILE * ADJ_TILE, smem, s>>>(descs, M, N, rad);
  return cudaGetLastError();
}

cudaError_t launch_adj_guided_filter(const AdjDesc* descs, int n, int M, int N, int rad,
                                     cudaStream_t s) {
  cudaError_t e = launch_adj_box<AdjStats>(descs, n, M, N, rad, s);
  if (e == cudaSuccess) e = launch_adj_box<AdjPoint>(descs, n, M, N, rad, s);
  if (e == cudaSuccess) e = launch_adj_box<AdjInputs>(descs, n, M, N, rad, s);
  return e;
}

// ---------------------------------------------------------------------------
// Recomputation of a step's spectra
// ---------------------------------------------------------------------------

// lambda_k of the forward solve becomes the step's lambda.
__global__ void k_adj_set_lambda(const AdjDesc* __restrict__ descs, int n, int k) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) *descs[i].lam = descs[i].lam_hist[k];
}

// U_I, U_p of the step (Eq. 8-9 with the forward's FP32 lambda) into UI, Up.
__global__ void k_adj_solve(const AdjDesc* __restrict__ descs, int M, int N,
                            const float* __restrict__ d2tab) {
  const AdjDesc& d = descs[blockIdx.y];
  const double lamd = __ldcg(d.lam);
  const bool branch = !(lamd < 1e300);
  const float lam = branch ? 0.0f : (float)lamd;
  const int L = N / 2;
  const size_t total = (size_t)M * L;
  for (size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
       idx += (size_t)gridDim.x * blockDim.x) {
    const int k = (int)(idx / L), l = (int)(idx - (size_t)k * L);
    const float d2r = __ldg(&d2tab[tab_off(M) + k]);
    float2 UI, Up;
    if (l != 0) {
      solve_bin(d.UE[idx], d.H[idx], d.Y[idx], lam, d2r + __ldg(&d2tab[tab_off(N) + l]), branch,
                UI, Up);
    } else {
      const size_t m = (size_t)((M - k) & (M - 1)) * L;
      float2 EA, EB, HA, HB, YA, YB, IA, IB, PA, PB;
      unpack_pair(d.UE[idx], d.UE[m], EA, EB);
      unpack_pair(d.H[idx], d.H[m], HA, HB);
      unpack_pair(d.Y[idx], d.Y[m], YA, YB);
      solve_bin(EA, HA, YA, lam, d2r, branch, IA, PA);
      solve_bin(EB, HB, YB, lam, d2r + 4.0f, branch, IB, PB);
      UI = pack_pair(IA, IB);
      Up = pack_pair(PA, PB);
    }
    d.UI[idx] = UI;
    d.Up[idx] = Up;
  }
}

static int spec_chunks(int M, int N) {
  const size_t total = (size_t)M * (N / 2);
  int chunks = (int)((total + 256 * 8 - 1) / (256 * 8));
  return chunks > 256 ? 256 : chunks;
}

cudaError_t launch_adj_recompute(const AdjDesc* descs, int n, int M, int N, int k,
                                 const float* d2tab, cudaStream_t s) {
  k_adj_set_lambda<<<(n + 63) / 64, 64, 0, s>>>(descs, n, k);
  k_adj_solve<<<dim3(spec_chunks(M, N), n), 256, 0, s>>>(descs, M, N, d2tab);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Spectral adjoint
// ---------------------------------------------------------------------------

GFD_D float2 cmulf(float2 a, float2 b) {  // a * b
  return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}
GFD_D float2 cmulc(float2 a, float2 b) {  // conj(a) * b
  return make_float2(fmaf(a.x, b.x, a.y * b.y), fmaf(a.x, b.y, -a.y * b.x));
}
GFD_D float redot(float2 a, float2 b) { return fmaf(a.x, b.x, a.y * b.y); }  // Re(conj(a) b)

// Per-bin values of pass A (Eq. 8, 9 reversed) for one full-spectrum bin.
// With e = H U_E - Y: U_E - U_p = conj(H) e / (a + lam) and U_E - U_I =
// conj(H) e / (a + lam D2), so lambda's adjoint is formed without the
// cancellation of U_E - U_p where lam >> a.
struct BinA {
  float2 gUE, gH, gY;
  float glam, fprime;
};
GFD_D BinA adj_bin_a(float2 H, float2 Y, float2 UE, float2 GUI, float2 GUp, float D2, float lam) {
  BinA o;
  const float a = fmaf(H.x, H.x, H.y * H.y);
  const float2 HY = cmulc(H, Y);
  const float ip = __frcp_rn(a + lam);
  const float2 Up = make_float2(fmaf(lam, UE.x, HY.x) * ip, fmaf(lam, UE.y, HY.y) * ip);
  const float2 gNp = cscale(GUp, ip);
  const float gDp = -redot(gNp, Up);  // -Re(conj(g_Up) U_p) / (a + lam)
  const float2 e = csub(cmulf(H, UE), Y);
  const float2 He = cmulc(H, e);
  o.glam = redot(gNp, He) * ip;
  float2 gNI = make_float2(0.0f, 0.0f);
  float gDI = 0.0f;
  const float lg = lam * D2, DI = a + lg;
  if (DI > 0.0f) {
    const float ii = __frcp_rn(DI);
    const float2 UI = make_float2(fmaf(lg, UE.x, HY.x) * ii, fmaf(lg, UE.y, HY.y) * ii);
    gNI = cscale(GUI, ii);
    gDI = -redot(gNI, UI);
    o.glam = fmaf(D2 * ii, redot(gNI, He), o.glam);
  }
  const float2 gN = cadd(gNp, gNI);
  const float gD2 = 2.0f * (gDp + gDI);
  // N = conj(H) Y + ...: g_Y += H g_N, g_H += conj(g_N) Y; D = |H|^2 + ...: g_H += 2 g_D H
  o.gY = cmulf(H, gN);
  const float2 gNY = cmulc(gN, Y);
  o.gH = make_float2(fmaf(gD2, H.x, gNY.x), fmaf(gD2, H.y, gNY.y));
  o.gUE = make_float2(lam * fmaf(D2, gNI.x, gNp.x), lam * fmaf(D2, gNI.y, gNp.y));
  const float s = lam * ip;  // lam / (a + lam)
  o.fprime = redot(e, e) * 2.0f * s * a * ip * ip;  // |e|^2 2 lam a / (a + lam)^3
  return o;
}

// Per-bin values of pass B (the implicit derivative of lambda through Eq. 11):
// f = (1/P) sum lam^2 |e|^2 / (a + lam)^2, e = H U_E - Y; c = -g_lam / f'.
GFD_D void adj_bin_b(float2 H, float2 Y, float2 UE, float lam, float cP, float2& gUE, float2& gH,
                     float2& gY) {
  const float a = fmaf(H.x, H.x, H.y * H.y);
  const float2 e = csub(cmulf(H, UE), Y);
  const float ip = __frcp_rn(a + lam);
  const float s = lam * ip;                         // lam / (a + lam)
  const float ge = 2.0f * cP * s * s;               // g_e = ge e
  const float2 g = cscale(e, ge);
  const float ga = -2.0f * cP * s * s * redot(e, e) * ip;  // -2 lam^2 |e|^2 / (a + lam)^3
  gUE = cmulc(H, g);                                // conj(H) g_e
  const float2 Ug = cmulc(UE, g);                   // conj(U_E) g_e
  gH = make_float2(fmaf(2.0f * ga, H.x, Ug.x), fmaf(2.0f * ga, H.y, Ug.y));
  gY = make_float2(-g.x, -g.y);
}

// Pass A over the packed half spectrum of every image (grid: (chunks, n)).
// Writes g_UE, adds to g_H and g_Y, and sums g_lam and P f'(lam) (FP64).
__global__ void k_adj_spec_a(const AdjDesc* __restrict__ descs, int M, int N,
                             const float* __restrict__ d2tab) {
  const AdjDesc& d = descs[blockIdx.y];
  const double lamd = __ldcg(d.lam);
  const bool branch = !(lamd < 1e300);
  const float lam = branch ? 0.0f : (float)lamd;
  const int L = N / 2;
  const size_t total = (size_t)M * L;
  const float invP = 1.0f / ((float)M * (float)N);
  double sl = 0.0, sf = 0.0;
  for (size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
       idx += (size_t)gridDim.x * blockDim.x) {
    if (branch) {
      d.gUE[idx] = make_float2(0.0f, 0.0f);
      continue;
    }
    const int k = (int)(idx / L), l = (int)(idx - (size_t)k * L);
    const float d2r = __ldg(&d2tab[tab_off(M) + k]);
    if (l != 0) {
      const BinA o = adj_bin_a(d.H[idx], d.Y[idx], d.UE[idx], cscale(d.GUI[idx], invP),
                               cscale(d.GUp[idx], invP), d2r + __ldg(&d2tab[tab_off(N) + l]),
                               lam);
      d.gUE[idx] = o.gUE;
      d.gH[idx] = cadd(d.gH[idx], o.gH);
      d.gY[idx] = cadd(d.gY[idx], o.gY);
      sl += 2.0 * (double)o.glam;  // the bin and its mirror
      sf += 2.0 * (double)o.fprime;
    } else {
      const size_t m = (size_t)((M - k) & (M - 1)) * L;
      float2 HA, HB, YA, YB, EA, EB, GIA, GIB, GPA, GPB;
      unpack_pair(d.H[idx], d.H[m], HA, HB);
      unpack_pair(d.Y[idx], d.Y[m], YA, YB);
      unpack_pair(d.UE[idx], d.UE[m], EA, EB);
      unpack_pair(cscale(d.GUI[idx], invP), cscale(d.GUI[m], invP), GIA, GIB);
      unpack_pair(cscale(d.GUp[idx], invP), cscale(d.GUp[m], invP), GPA, GPB);
      const BinA oa = adj_bin_a(HA, YA, EA, GIA, GPA, d2r, lam);
      const BinA ob = adj_bin_a(HB, YB, EB, GIB, GPB, d2r + 4.0f, lam);
      d.gUE[idx] = pack_pair(oa.gUE, ob.gUE);
      d.gH[idx] = cadd(d.gH[idx], pack_pair(oa.gH, ob.gH));
      d.gY[idx] = cadd(d.gY[idx], pack_pair(oa.gY, ob.gY));
      sl += (double)oa.glam + (double)ob.glam;
      sf += (double)oa.fprime + (double)ob.fprime;
    }
  }
  __shared__ double red[2][32];
  for (int o = 16; o > 0; o >>= 1) {
    sl += __shfl_xor_sync(0xffffffffu, sl, o);
    sf += __shfl_xor_sync(0xffffffffu, sf, o);
  }
  if ((threadIdx.x & 31) == 0) {
    red[0][threadIdx.x >> 5] = sl;
    red[1][threadIdx.x >> 5] = sf;
  }
  __syncthreads();
  if (threadIdx.x == 0 && !branch) {
    double a = 0.0, b = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
      a += red[0][w];
      b += red[1][w];
    }
    atomicAdd(&d.acc[0], a);
    atomicAdd(&d.acc[1], b);
  }
}

// Per image: c = -g_lam / f'(lam) and g_T -= c; clears the sums for the next step.
__global__ void k_adj_lambda(const AdjDesc* __restrict__ descs, int n, double P) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const AdjDesc& d = descs[i];
  const double lam = *d.lam;
  if (lam < 1e300 && d.acc[1] > 0.0) {
    const double fprime = d.acc[1] / P;
    const double c = -d.acc[0] / fprime;
    d.acc[2] = c;
    d.acc[3] -= c;  // g_T
  } else {
    d.acc[2] = 0.0;
  }
  d.acc[0] = 0.0;
  d.acc[1] = 0.0;
}

// Pass B: the c-weighted gradient of f through e = H U_E - Y and a = |H|^2.
__global__ void k_adj_spec_b(const AdjDesc* __restrict__ descs, int M, int N) {
  const AdjDesc& d = descs[blockIdx.y];
  const double lamd = __ldcg(d.lam);
  if (!(lamd < 1e300)) return;
  const float lam = (float)lamd;
  const float cP = (float)(__ldcg(&d.acc[2]) / ((double)M * N));
  const int L = N / 2;
  const size_t total = (size_t)M * L;
  for (size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
       idx += (size_t)gridDim.x * blockDim.x) {
    const int k = (int)(idx / L), l = (int)(idx - (size_t)k * L);
    float2 gUE, gH, gY;
    if (l != 0) {
      adj_bin_b(d.H[idx], d.Y[idx], d.UE[idx], lam, cP, gUE, gH, gY);
    } else {
      const size_t m = (size_t)((M - k) & (M - 1)) * L;
      float2 HA, HB, YA, YB, EA, EB, uA, uB, hA, hB, yA, yB;
      unpack_pair(d.H[idx], d.H[m], HA, HB);
      unpack_pair(d.Y[idx], d.Y[m], YA, YB);
      unpack_pair(d.UE[idx], d.UE[m], EA, EB);
      adj_bin_b(HA, YA, EA, lam, cP, uA, hA, yA);
      adj_bin_b(HB, YB, EB, lam, cP, uB, hB, yB);
      gUE = pack_pair(uA, uB);
      gH = pack_pair(hA, hB);
      gY = pack_pair(yA, yB);
    }
    d.gUE[idx] = cadd(d.gUE[idx], gUE);
    d.gH[idx] = cadd(d.gH[idx], gH);
    d.gY[idx] = cadd(d.gY[idx], gY);
  }
}

// g_u of the previous step: the adjoint DFT of g_UE (in gtmp, scale 1), or
// g_uI + g_up where lambda = inf (u_I = u_p = u_E).
__global__ void k_adj_next(const AdjDesc* __restrict__ descs, int M, int N) {
  const AdjDesc& d = descs[blockIdx.y];
  const bool branch = !(__ldcg(d.lam) < 1e300);
  const size_t P = (size_t)M * N;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < P;
       i += (size_t)gridDim.x * blockDim.x)
    d.gu[i] = branch ? d.guI[i] + d.gup[i] : d.gtmp[i];
}

cudaError_t launch_adj_spectral(const AdjDesc* descs, int n, int M, int N, const float* d2tab,
                                cudaStream_t s) {
  const int chunks = spec_chunks(M, N);
  k_adj_spec_a<<<dim3(chunks, n), 256, 0, s>>>(descs, M, N, d2tab);
  k_adj_lambda<<<(n + 63) / 64, 64, 0, s>>>(descs, n, (double)M * N);
  k_adj_spec_b<<<dim3(chunks, n), 256, 0, s>>>(descs, M, N);
  return cudaGetLastError();
}

cudaError_t launch_adj_next(const AdjDesc* descs, int n, int M, int N, cudaStream_t s) {
  const size_t P = (size_t)M * N;
  int chunks = (int)((P + 256 * 8 - 1) / (256 * 8));
  if (chunks > 256) chunks = 256;
  k_adj_next<<<dim3(chunks, n), 256, 0, s>>>(descs, M, N);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Statistics of Eq. 12 and the final gradients of y and h
// ---------------------------------------------------------------------------

// sum y, sum y^2 (FP64) into acc[4], acc[5]; sum |h| into acc[6] (block 0).
__global__ void k_adj_stats(const AdjDesc* __restrict__ descs, int M, int N) {
  const AdjDesc& d = descs[blockIdx.y];
  const size_t P = (size_t)M * N;
  double sy = 0.0, syy = 0.0;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < P;
       i += (size_t)gridDim.x * blockDim.x) {
    const double v = d.y[i];
    sy += v;
    syy += v * v;
  }
  for (int o = 16; o > 0; o >>= 1) {
    sy += __shfl_xor_sync(0xffffffffu, sy, o);
    syy += __shfl_xor_sync(0xffffffffu, syy, o);
  }
  if ((threadIdx.x & 31) == 0) {
    atomicAdd(&d.acc[4], sy);
    atomicAdd(&d.acc[5], syy);
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    double s = 0.0;
    for (int i = 0; i < d.kh * d.kw; ++i) s += fabs((double)d.h[i]);
    d.acc[6] = s;
  }
}

// dT/dy and dT/dh through rho (Eq. 12): acc[7] = g_num, acc[8] = g_den (zero
// where rho is clamped to 1); writes g_eps.
__global__ void k_adj_rho(const AdjDesc* __restrict__ descs, int n, double P) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const AdjDesc& d = descs[i];
  const double Sy = d.acc[4], Syy = d.acc[5], h1 = d.acc[6], sig2 = d.sigma * d.sigma;
  const double num = Syy - Sy * Sy / P - P * sig2;
  const double den = h1 * h1 * Syy;
  const double rad = 1.0 - num / den;
  double g_num = 0.0, g_den = 0.0;
  if (rad > 0.0 && rad < 1.0 && d.rho_fixed <= 0.0) {
    const double rho = sqrt(rad);
    const double g_rad = d.acc[3] * P * sig2 / (2.0 * rho);
    g_num = -g_rad / den;
    g_den = g_rad * num / (den * den);
  }
  d.acc[7] = g_num;
  d.acc[8] = g_den;
  *d.g_eps_out = *d.g_eps;
}

// g_y = (adjoint DFT of g_Y, in gtmp) + dT/dy terms.
__global__ void k_adj_final_y(const AdjDesc* __restrict__ descs, int M, int N) {
  const AdjDesc& d = descs[blockIdx.y];
  const size_t P = (size_t)M * N;
  const double g_num = d.acc[7], g_den = d.acc[8], Sy = d.acc[4], h1 = d.acc[6];
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < P;
       i += (size_t)gridDim.x * blockDim.x) {
    const double y = d.y[i];
    d.gy_out[i] = (float)((double)d.gtmp[i] + g_num * (2.0 * y - 2.0 * Sy / (double)P) +
                          g_den * h1 * h1 * 2.0 * y);
  }
}

// g_h[i][j] = (adjoint DFT of g_H at the canvas position of h[i][j], in gtmp2)
// + dT/dh (Eq. 12 through sum |h|).
__global__ void k_adj_final_h(const AdjDesc* __restrict__ descs, int M, int N) {
  const AdjDesc& d = descs[blockIdx.y];
  const int rh = d.kh / 2, rw = d.kw / 2;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < d.kh * d.kw; e += gridDim.x * blockDim.x) {
    const int i = e / d.kw, j = e - i * d.kw;
    const int ci = ((i - rh) % M + M) % M, cj = ((j - rw) % N + N) % N;
    const double hv = d.h[e];
    const double sgn = hv > 0.0 ? 1.0 : (hv < 0.0 ? -1.0 : 0.0);
    d.gh_out[e] = (float)((double)d.gtmp2[(size_t)ci * N + cj] +
                          d.acc[8] * 2.0 * d.acc[6] * d.acc[5] * sgn);
  }
}

cudaError_t launch_adj_stats(const AdjDesc* descs, int n, int M, int N, cudaStream_t s) {
  const size_t P = (size_t)M * N;
  int chunks = (int)((P + 256 * 16 - 1) / (256 * 16));
  if (chunks > 64) chunks = 64;
  k_adj_stats<<<dim3(chunks, n), 256, 0, s>>>(descs, M, N);
  return cudaGetLastError();
}

cudaError_t launch_adj_final(const AdjDesc* descs, int n, int M, int N, int max_psf,
                             cudaStream_t s) {
  const size_t P = (size_t)M * N;
  int chunks = (int)((P + 256 * 8 - 1) / (256 * 8));
  if (chunks > 256) chunks = 256;
  k_adj_rho<<<(n + 63) / 64, 64, 0, s>>>(descs, n, (double)P);
  k_adj_final_y<<<dim3(chunks, n), 256, 0, s>>>(descs, M, N);
  k_adj_final_h<<<dim3((max_psf + 255) / 256, n), 256, 0, s>>>(descs, M, N);
  return cudaGetLastError();
}

cudaError_t configure_adj_kernels() {
  const int rmax = 8, E = ADJ_TILE + 2 * rmax;  // shared bytes of launch_adj_box at r = 8
  const int b1 = E * ADJ_TILE * AdjStats::NQ * 8 + AdjStats::NS * E * E * 4;
  const int b2 = E * ADJ_TILE * AdjPoint::NQ * 8 + AdjPoint::NS * E * E * 4;
  const int b3 = E * ADJ_TILE * AdjInputs::NQ * 8 + AdjInputs::NS * E * E * 4;
  cudaError_t e = cudaFuncSetAttribute(k_adj_box<AdjStats>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, b1);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_adj_box<AdjPoint>, cudaFuncAttributeMaxDynamicSharedMemorySize, b2);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_adj_box<AdjInputs>, cudaFuncAttributeMaxDynamicSharedMemorySize, b3);
  return e;
}

}  // namespace gfd
