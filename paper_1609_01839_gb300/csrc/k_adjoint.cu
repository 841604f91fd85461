// Reverse mode of the unrolled method: gradients of a loss of u^K with
// respect to the observation y, the PSF h and the guided filter's eps.
//
// One backward step undoes one iteration (Sec. 3.1 Steps 1-2) from its
// checkpoint u_E^k, in reverse order of the forward step:
//   guided filter (Eq. 3-5; periodic windows, so the box mean is its own
//   adjoint): three tiled passes of FP64 window sums
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
// Spectra are the library's packed half spectra, row-major (tile width N/2):
// Z[m][l] = X(m, l) for 1 <= l < N/2 and Z[m][0] = X(m, 0) + i X(m, N/2).
// Complex gradients follow g_z = dL/dRe z + i dL/dIm z; a sum over all bins
// counts the interior columns twice (each stands for its mirror bin too).
#include "common.cuh"
#include "launch.h"

namespace gfd {

constexpr int ADJ_TILE = 16;

// ---------------------------------------------------------------------------
// Tiled window sums: OP stages NS planes of a TILE x TILE tile plus an r halo
// in shared memory, maps every staged pixel to NQ quantities (FP64), and gets
// their window sums (periodic windows) at each output pixel.
// ---------------------------------------------------------------------------
template <class OP>
__global__ void __launch_bounds__(ADJ_TILE * ADJ_TILE)
k_adj_box(const AdjDesc* __restrict__ descs, int M, int N, int rad) {
  extern __shared__ __align__(16) unsigned char adj_sm[];
  constexpr int NS = OP::NS, NQ = OP::NQ;
  const AdjDesc& d = descs[blockIdx.z];
  const int E = ADJ_TILE + 2 * rad;
  double* rows = reinterpret_cast<double*>(adj_sm);                          // [E][T][NQ]
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
    double s[NQ];
#pragma unroll
    for (int q = 0; q < NQ; ++q) s[q] = 0.0;
    for (int dx = 0; dx <= 2 * rad; ++dx) {
      const int o = ty * E + tx + dx;
      float v[NS];
#pragma unroll
      for (int c = 0; c < NS; ++c) v[c] = tile[c * E * E + o];
      double q[NQ];
      OP::quantities(v, q);
#pragma unroll
      for (int k = 0; k < NQ; ++k) s[k] += q[k];
    }
#pragma unroll
    for (int q = 0; q < NQ; ++q) rows[(size_t)e * NQ + q] = s[q];
  }
  __syncthreads();
  const int tx = threadIdx.x % ADJ_TILE, ty = threadIdx.x / ADJ_TILE;
  const int gy = y0 + ty, gx = x0 + tx;
  double S[NQ];
#pragma unroll
  for (int q = 0; q < NQ; ++q) S[q] = 0.0;
  for (int dy = 0; dy <= 2 * rad; ++dy) {
    const double* rr = rows + ((size_t)(ty + dy) * ADJ_TILE + tx) * NQ;
#pragma unroll
    for (int q = 0; q < NQ; ++q) S[q] += rr[q];
  }
  const double inv_n = 1.0 / (double)((2 * rad + 1) * (2 * rad + 1));
#pragma unroll
  for (int q = 0; q < NQ; ++q) S[q] *= inv_n;  // window means
  double eps_part = 0.0;
  if (gy < M && gx < N) eps_part = OP::output(d, (size_t)gy * N + gx, S);
  if (OP::kEps) {  // sum of the pass's eps adjoint over the block, one atomic
    __shared__ double red[ADJ_TILE * ADJ_TILE / 32];
    for (int o = 16; o > 0; o >>= 1) eps_part += __shfl_xor_sync(0xffffffffu, eps_part, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = eps_part;
    __syncthreads();
    if (threadIdx.x == 0) {
      double t = 0.0;
      for (int w = 0; w < ADJ_TILE * ADJ_TILE / 32; ++w) t += red[w];
      atomicAdd(d.g_eps, t);
    }
  }
}

// Pass 1: mu = box(I), pbar = box(p), sigma^2 + eps, a (Eq. 3).
struct AdjStats {
  static constexpr int NS = 2, NQ = 4;
  static constexpr bool kEps = false;
  GFD_D static const float* plane(const AdjDesc& d, int c) { return c == 0 ? d.uI : d.up; }
  GFD_D static void quantities(const float (&v)[NS], double (&q)[NQ]) {
    const double I = v[0], p = v[1];
    q[0] = I;
    q[1] = p;
    q[2] = I * p;
    q[3] = I * I;
  }
  GFD_D static double output(const AdjDesc& d, size_t o, const double (&S)[NQ]) {
    const double mu = S[0], pb = S[1];
    const double ve = S[3] - mu * mu + d.eps;   // sigma_k^2 + eps
    const double a = (S[2] - mu * pb) / ve;
    d.A[o] = (float)a;
    d.MU[o] = (float)mu;
    d.PB[o] = (float)pb;
    d.VE[o] = (float)ve;
    return 0.0;
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
  GFD_D static void quantities(const float (&v)[NS], double (&q)[NQ]) {
    q[0] = v[0];
    q[1] = (double)v[1] * v[2];
    q[2] = v[1];
  }
  GFD_D static double output(const AdjDesc& d, size_t o, const double (&S)[NQ]) {
    const double abar = S[0], g_b = S[2];
    const double a = d.A[o], mu = d.MU[o], pb = d.PB[o], ve = d.VE[o];
    const double gI0 = (double)d.gu[o] * abar;           // u = abar I + bbar
    const double g_a = S[1] - mu * g_b;                   // box(g_u I), b = pbar - a mu
    double g_mu = -a * g_b, g_pb = g_b;
    const double g_cov = g_a / ve, g_var = -g_a * a / ve; // a = cov / (var + eps)
    g_mu += -pb * g_cov - 2.0 * mu * g_var;               // cov = m_Ip - mu pbar, var = m_II - mu^2
    g_pb += -mu * g_cov;
    d.GI0[o] = (float)gI0;
    d.GCOV[o] = (float)g_cov;
    d.GVAR[o] = (float)g_var;
    d.GMU[o] = (float)g_mu;
    d.GPB[o] = (float)g_pb;
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
  GFD_D static void quantities(const float (&v)[NS], double (&q)[NQ]) {
#pragma unroll
    for (int k = 0; k < NQ; ++k) q[k] = v[k];
  }
  GFD_D static double output(const AdjDesc& d, size_t o, const double (&S)[NQ]) {
    const double I = d.uI[o], p = d.up[o];
    d.guI[o] = (float)((double)d.GI0[o] + p * S[0] + 2.0 * I * S[1] + S[2]);  // m_Ip, m_II, mu
    d.gup[o] = (float)(I * S[0] + S[3]);                                       // m_Ip, pbar
    return 0.0;
  }
};

template <class OP>
static cudaError_t launch_adj_box(const AdjDesc* descs, int n, int M, int N, int rad,
                                  cudaStream_t s) {
  const int E = ADJ_TILE + 2 * rad;
  const size_t smem = (size_t)E * ADJ_TILE * OP::NQ * sizeof(double) +
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
// Spectral adjoint
// ---------------------------------------------------------------------------

// Bins (k, 0) and (k, N/2) of a packed column-0 entry: A = (Z[k] + conj Z[-k]) / 2,
// B = (Z[k] - conj Z[-k]) / (2i); and back: Z[k] = A + i B.
GFD_D void adj_unpack(float2 zk, float2 zm, float2& A, float2& B) {
  const float2 c = cconj(zm);
  A = cscale(cadd(zk, c), 0.5f);
  const float2 D = csub(zk, c);
  B = make_float2(0.5f * D.y, -0.5f * D.x);
}
GFD_D float2 adj_pack(float2 A, float2 B) { return make_float2(A.x - B.y, A.y + B.x); }
GFD_D float2 cmulc(float2 a, float2 b) {  // conj(a) * b
  return make_float2(fmaf(a.x, b.x, a.y * b.y), fmaf(a.x, b.y, -a.y * b.x));
}

// Per-bin values of pass A (Eq. 8, 9 reversed) for one full-spectrum bin.
struct BinA {
  float2 gUE, gH, gY;
  double glam, fprime;
};
GFD_D BinA adj_bin_a(float2 H, float2 Y, float2 UE, float2 UI, float2 Up, float2 GUI, float2 GUp,
                     float D2, double lam) {
  BinA o;
  const double a = (double)H.x * H.x + (double)H.y * H.y;
  const double Dp = a + lam, DI = a + lam * D2;
  const double gNpx = GUp.x / Dp, gNpy = GUp.y / Dp;
  const double gDp = -((double)GUp.x * Up.x + (double)GUp.y * Up.y) / Dp;
  double gNIx = 0.0, gNIy = 0.0, gDI = 0.0;
  if (DI > 0.0) {
    gNIx = GUI.x / DI;
    gNIy = GUI.y / DI;
    gDI = -((double)GUI.x * UI.x + (double)GUI.y * UI.y) / DI;
  }
  const double gNx = gNpx + gNIx, gNy = gNpy + gNIy;
  // N = conj(H) Y + ... : g_Y += H g_N, g_H += conj(g_N) Y; D = |H|^2 + ...: g_H += 2 g_D H
  o.gY = make_float2((float)(H.x * gNx - H.y * gNy), (float)(H.x * gNy + H.y * gNx));
  const double gD = gDp + gDI;
  o.gH = make_float2((float)(gNx * Y.x + gNy * Y.y + 2.0 * gD * H.x),
                     (float)(gNx * Y.y - gNy * Y.x + 2.0 * gD * H.y));
  o.gUE = make_float2((float)(lam * (gNpx + D2 * gNIx)), (float)(lam * (gNpy + D2 * gNIy)));
  o.glam = (gNpx * UE.x + gNpy * UE.y) + gDp + D2 * ((gNIx * UE.x + gNIy * UE.y) + gDI);
  const double ex = (double)H.x * UE.x - (double)H.y * UE.y - Y.x;
  const double ey = (double)H.x * UE.y + (double)H.y * UE.x - Y.y;
  const double r = ex * ex + ey * ey;
  const double ap = a + lam;
  o.fprime = r * 2.0 * lam * a / (ap * ap * ap);
  return o;
}

// Per-bin values of pass B (the implicit derivative of lambda through Eq. 11):
// f = (1/P) sum lam^2 |e|^2 / (a + lam)^2, e = H U_E - Y; c = -g_lam / f'.
GFD_D void adj_bin_b(float2 H, float2 Y, float2 UE, double lam, double cP, float2& gUE, float2& gH,
                     float2& gY) {
  const double a = (double)H.x * H.x + (double)H.y * H.y;
  const double ex = (double)H.x * UE.x - (double)H.y * UE.y - Y.x;
  const double ey = (double)H.x * UE.y + (double)H.y * UE.x - Y.y;
  const double ap = a + lam;
  const double ge = cP * lam * lam / (ap * ap) * 2.0;            // g_e = ge * e
  const double gx = ge * ex, gy = ge * ey;
  const double ga = cP * (-2.0 * lam * lam * (ex * ex + ey * ey)) / (ap * ap * ap);
  gUE = make_float2((float)(H.x * gx + H.y * gy), (float)(H.x * gy - H.y * gx));    // conj(H) g_e
  gH = make_float2((float)(UE.x * gx + UE.y * gy + 2.0 * ga * H.x),
                   (float)(UE.x * gy - UE.y * gx + 2.0 * ga * H.y));               // conj(U_E) g_e
  gY = make_float2((float)-gx, (float)-gy);
}

// Pass A over the packed half spectrum of every image (grid: (chunks, n)).
// Writes g_UE, adds to g_H and g_Y, and sums g_lam and P f'(lam).
__global__ void k_adj_spec_a(const AdjDesc* __restrict__ descs, int M, int N,
                             const float* __restrict__ d2tab) {
  const AdjDesc& d = descs[blockIdx.y];
  const double lam = __ldcg(d.lam);
  const int L = N / 2;
  const size_t total = (size_t)M * L;
  const float invP = 1.0f / ((float)M * (float)N);
  double sl = 0.0, sf = 0.0;
  const bool branch = !(lam < 1e300);
  for (size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
       idx += (size_t)gridDim.x * blockDim.x) {
    if (branch) {
      d.gUE[idx] = make_float2(0.0f, 0.0f);
      continue;
    }
    const int k = (int)(idx / L), l = (int)(idx - (size_t)k * L);
    const float d2r = d2tab[tab_off(M) + k];
    if (l != 0) {
      const BinA o = adj_bin_a(d.H[idx], d.Y[idx], d.UE[idx], d.UI[idx], d.Up[idx],
                               cscale(d.GUI[idx], invP), cscale(d.GUp[idx], invP),
                               d2r + d2tab[tab_off(N) + l], lam);
      d.gUE[idx] = o.gUE;
      d.gH[idx] = cadd(d.gH[idx], o.gH);
      d.gY[idx] = cadd(d.gY[idx], o.gY);
      sl += 2.0 * o.glam;  // the bin and its mirror
      sf += 2.0 * o.fprime;
    } else {
      const size_t m = (size_t)((M - k) & (M - 1)) * L;
      float2 HA, HB, YA, YB, EA, EB, IA, IB, PA, PB, GIA, GIB, GPA, GPB;
      adj_unpack(d.H[idx], d.H[m], HA, HB);
      adj_unpack(d.Y[idx], d.Y[m], YA, YB);
      adj_unpack(d.UE[idx], d.UE[m], EA, EB);
      adj_unpack(d.UI[idx], d.UI[m], IA, IB);
      adj_unpack(d.Up[idx], d.Up[m], PA, PB);
      adj_unpack(cscale(d.GUI[idx], invP), cscale(d.GUI[m], invP), GIA, GIB);
      adj_unpack(cscale(d.GUp[idx], invP), cscale(d.GUp[m], invP), GPA, GPB);
      const BinA oa = adj_bin_a(HA, YA, EA, IA, PA, GIA, GPA, d2r, lam);
      const BinA ob = adj_bin_a(HB, YB, EB, IB, PB, GIB, GPB, d2r + 4.0f, lam);
      d.gUE[idx] = adj_pack(oa.gUE, ob.gUE);
      d.gH[idx] = cadd(d.gH[idx], adj_pack(oa.gH, ob.gH));
      d.gY[idx] = cadd(d.gY[idx], adj_pack(oa.gY, ob.gY));
      sl += oa.glam + ob.glam;
      sf += oa.fprime + ob.fprime;
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
  const double lam = __ldcg(d.lam);
  if (!(lam < 1e300)) return;
  const double cP = __ldcg(&d.acc[2]) / ((double)M * N);
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
      adj_unpack(d.H[idx], d.H[m], HA, HB);
      adj_unpack(d.Y[idx], d.Y[m], YA, YB);
      adj_unpack(d.UE[idx], d.UE[m], EA, EB);
      adj_bin_b(HA, YA, EA, lam, cP, uA, hA, yA);
      adj_bin_b(HB, YB, EB, lam, cP, uB, hB, yB);
      gUE = adj_pack(uA, uB);
      gH = adj_pack(hA, hB);
      gY = adj_pack(yA, yB);
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
  const size_t total = (size_t)M * (N / 2);
  int chunks = (int)((total + 256 * 8 - 1) / (256 * 8));
  if (chunks > 256) chunks = 256;
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
  const int rmax = 8, E = ADJ_TILE + 2 * rmax;
  const int b1 = E * ADJ_TILE * 4 * 8 + 2 * E * E * 4;
  const int b2 = E * ADJ_TILE * 3 * 8 + 3 * E * E * 4;
  const int b3 = E * ADJ_TILE * 4 * 8 + 4 * E * E * 4;
  cudaError_t e = cudaFuncSetAttribute(k_adj_box<AdjStats>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, b1);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_adj_box<AdjPoint>, cudaFuncAttributeMaxDynamicSharedMemorySize, b2);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_adj_box<AdjInputs>, cudaFuncAttributeMaxDynamicSharedMemorySize, b3);
  return e;
}

}  // namespace gfd
