// Regularisation parameter by the discrepancy principle (Sec. 3.2).
//
// With a_b = |H_b|^2 and r_b = |H_b U_E,b - Y_b|^2 over all DFT bins b, the
// residual of u_p is f(lambda) = (1/P) sum_b lambda^2 r_b / (a_b + lambda)^2
// (Eq. 10-11 with Parseval's 1/P).  If ||h*u_E - y||^2 = f(inf) <= T the
// estimate is already in K and lambda = inf; otherwise lambda solves
// f(lambda) = T, whose root is unique because f increases (Eq. 11).
//
// GPU procedure (one spectral pass per evaluation, no host round trip):
//   each pass evaluates f at KNODES Chebyshev-Lobatto points of
//   s = log(lambda) over the current bracket [lo, hi], accumulating the
//   per-bin terms in FP32 per thread and in FP64 across warps and blocks;
//   the last block of the image then either
//     - interpolates f(s) through the nodes (barycentric form, FP64) and
//       takes the root of the interpolant, when the bracket is narrow enough
//       for the interpolant to be exact to ~1e-12 (f is analytic in the strip
//       |Im s| < pi, its poles lying at lambda = -a_b), or
//     - narrows the bracket to the sub-interval between the nodes that
//       straddle T, or extends it past the end node when T is outside,
//   and the next pass runs only for images whose root is still open.
// The first pass of each iteration is fused into the forward column FFT and
// is centred on the previous iteration's lambda.
#pragma once
#include "common.cuh"

namespace gfd {

constexpr double PI_D = 3.14159265358979323846;
// log-width of a bracket over which the 12-node interpolant is trusted as
// the final answer (ratio 4), and over which it is trusted as an estimate
// that a +-2% bracket is placed around (ratio 64).
constexpr double W_EXACT = 1.3862943611198906 * 1.000001;
constexpr double W_ESTIMATE = 4.1588830833596715;
constexpr double EST_HALF_WIDTH = 0.02;
constexpr double PRIMARY_RATIO = 2.0;
constexpr double INITIAL_LO = 1e-10, INITIAL_HI = 1e10;

// cos(pi j / (KNODES - 1)), j = 0..KNODES-1 (Chebyshev-Lobatto points)
__device__ constexpr double kLobatto[KNODES] = {
    1.0, 0.9594929736144974, 0.8412535328311812, 0.6548607339452851,
    0.41541501300188644, 0.14231483827328512, -0.142314838273285, -0.4154150130018863,
    -0.654860733945285, -0.8412535328311811, -0.9594929736144974, -1.0};

// Nodes of the next pass over [lo, hi], computed by the lanes of one warp
// (lane j < KNODES owns node j).  The per-bin arithmetic uses the node
// rounded to float; its exact logarithm (s + log1p(e), e the rounding's
// relative error) is kept as the interpolation abscissa.
GFD_D void set_bracket_warp(ImgState* st, double lo, double hi, int lane) {
  if (lane == 0) {
    st->lo = lo;
    st->hi = hi;
  }
  if (lane < KNODES) {
    const double a = log(lo), b = log(hi);
    const double sj = 0.5 * (a + b) - 0.5 * (b - a) * kLobatto[lane];
    const double e = exp(sj);
    const float lf = (float)e;
    const double rel = (double)lf / e - 1.0;
    st->node[lane] = lf;
    st->snode[lane] = sj + rel - 0.5 * rel * rel;
  }
  __syncwarp();
}

// Single-thread variant for the setup kernel.
GFD_D void set_bracket(ImgState* st, double lo, double hi) {
  st->lo = lo;
  st->hi = hi;
  const double a = log(lo), b = log(hi);
  for (int j = 0; j < KNODES; ++j) {
    const double sj = 0.5 * (a + b) - 0.5 * (b - a) * kLobatto[j];
    const double e = exp(sj);
    const float lf = (float)e;
    const double rel = (double)lf / e - 1.0;
    st->node[j] = lf;
    st->snode[j] = sj + rel - 0.5 * rel * rel;
  }
}

// One bin's contribution: wr = (Hermitian weight) * r, a = |H|^2.
GFD_D void accum_bin(float wr, float a, const float* nodes, float* acc) {
  acc[KNODES] += wr;
#pragma unroll
  for (int j = 0; j < KNODES; ++j) {
    const float t = __fdividef(nodes[j], a + nodes[j]);
    acc[j] = fmaf(wr, t * t, acc[j]);
  }
}

// Block-wide sums of the KNODES+1 per-thread partials (FP32 within a warp,
// FP64 across warps), stored with plain stores to part[0..KNODES].
// red must hold num_warps() * (KNODES+1) doubles.  Ends synchronised.
GFD_D void block_partials(float* acc, double* red, double* part) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int nwarp = num_warps();
#pragma unroll
  for (int j = 0; j <= KNODES; ++j) {
    const float v = warp_sum(acc[j]);
    if (lane == 0) red[warp * (KNODES + 1) + j] = (double)v;
  }
  __syncthreads();
  for (int j = threadIdx.x; j <= KNODES; j += blockDim.x) {
    double s = 0.0;
    for (int w = 0; w < nwarp; ++w) s += red[w * (KNODES + 1) + j];
    part[j] = s;
  }
  __syncthreads();
}

GFD_D double warp_sum_dbl(double v) {
  const unsigned int n = blockDim.x < 32 ? blockDim.x : 32u;
  const unsigned int mask = n == 32 ? 0xffffffffu : ((1u << n) - 1u);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1)
    if ((unsigned)o < n) v += __shfl_xor_sync(mask, v, o);
  return v;
}

// Sum of vals[i * stride + j] over i < n for each j < m, by the whole block
// in FP64 (loads bypass L1: the values were written by other blocks).
// Results land in sums[0..m) (shared), visible to every thread on return.
GFD_D void block_sum_columns(const double* vals, int n, int stride, int m, double* red,
                             double* sums) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int nwarp = num_warps();
  for (int j = 0; j < m; ++j) {
    double s = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) s += __ldcg(&vals[(size_t)i * stride + j]);
    s = warp_sum_dbl(s);
    if (lane == 0) red[warp] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
      double t = 0.0;
      for (int w = 0; w < nwarp; ++w) t += red[w];
      sums[j] = t;
    }
    __syncthreads();
  }
}

// Called by every block after storing its item's partials: true in exactly
// one block per image and pass (the one finishing last), after all partials
// are visible.
GFD_D bool last_item(unsigned int* counter, unsigned int n_items, int* s_flag) {
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) {
    const unsigned int prev = atomicAdd(counter, 1u);
    *s_flag = (prev == n_items - 1);
  }
  __syncthreads();
  const bool last = *s_flag != 0;
  if (last) __threadfence();
  return last;
}

GFD_D double warp_sum_full(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// 1/d in FP64 from an FP32 seed and two Newton steps (|d| within FP32 range).
GFD_D double rcp_d(double d) {
  double r = (double)__frcp_rn((float)d);
  double e = fma(-d, r, 1.0);
  r = fma(r, e, r);
  e = fma(-d, r, 1.0);
  return fma(r, e, r);
}

// Root in s of the interpolant of (s_m, f_m) minus T inside [s_j, s_{j+1}]
// (f increases through T there), as lambda = exp(s).  Lane m < KNODES holds
// node m; the barycentric sums are warp reductions.  Safeguarded Newton:
// steps leaving the bracket fall back to bisection.
GFD_D double interp_root_warp(double sm, double fm, double T, int j, int lane) {
  const bool own = lane < KNODES;
  double prod = 1.0;
  for (int n = 0; n < KNODES; ++n) {
    const double sn = __shfl_sync(0xffffffffu, sm, n);
    if (n != lane) prod *= (sm - sn);
  }
  const double wb = own ? 1.0 / prod : 0.0;
  double a = __shfl_sync(0xffffffffu, sm, j), b = __shfl_sync(0xffffffffu, sm, j + 1);
  const double fa = __shfl_sync(0xffffffffu, fm, j) - T;
  const double fb = __shfl_sync(0xffffffffu, fm, j + 1) - T;
  if (fa == 0.0) return exp(a);
  if (fb == 0.0) return exp(b);
  double x = a - fa * (b - a) / (fb - fa);
  if (!(x > a && x < b)) x = 0.5 * (a + b);
  for (int it = 0; it < 40; ++it) {
    const double d = x - sm;
    const unsigned hit = __ballot_sync(0xffffffffu, own && d == 0.0);
    if (hit) return exp(x);  // x is a node; bracket ends already excluded roots there
    const double rd = own ? rcp_d(d) : 0.0;
    const double t = wb * rd;
    const double N = warp_sum_full(t * fm);
    const double D = warp_sum_full(t);
    const double r = N / D;
    const double dr = warp_sum_full(own ? t * (r - fm) * rd : 0.0) / D;
    const double g = r - T;
    if (g < 0.0)
      a = x;
    else
      b = x;
    double xn = x - g / dr;
    if (!(xn > a && xn < b)) xn = 0.5 * (a + b);
    const double step = fabs(xn - x);
    x = xn;
    if (step <= 1e-15 * fmax(1.0, fabs(x)) || b - a <= 1e-15 * fmax(1.0, fabs(a))) break;
  }
  return exp(x);
}

GFD_D void resolve_warp(ImgState* st, double lam, int iter, double* lam_out, int lane) {
  if (lane == 0) {
    st->lam = lam;
    st->need = 0;
    if (lam_out) lam_out[iter] = lam;
  }
  if (isfinite(lam) && lam > 0.0) set_bracket_warp(st, lam / PRIMARY_RATIO, lam * PRIMARY_RATIO, lane);
}

// Consume the totals of the pass that just completed for this image (tot:
// KNODES node sums and the residual sum, visible to the warp).  Run by the
// 32 lanes of one warp of the image's last block; every lane takes the same
// decisions from the same values.
GFD_D void lambda_update_warp(ImgState* st, const double* tot, double P, bool primary,
                              bool last_chance, int iter, double* lam_out, double* res_out,
                              int lane) {
  const double T = st->T;
  const double resinf = tot[KNODES] / P;
  if (primary) {
    if (lane == 0) {
      st->res = resinf;
      if (res_out) res_out[iter] = resinf;
    }
    if (!isfinite(resinf)) {
      if (lane == 0) st->status |= ST_NONFINITE;
      resolve_warp(st, INFINITY, iter, lam_out, lane);
      return;
    }
    if (resinf <= T) {  // u_E in K (Sec. 3.2): lambda = inf, u_I = u_p = u_E
      resolve_warp(st, INFINITY, iter, lam_out, lane);
      return;
    }
    const double t = sqrt(T / resinf);
    if (lane == 0) st->lam_up = fmin(1e30, st->amax * t / (1.0 - t));
    __syncwarp();
  }
  const double f0 = tot[0] / P, fK = tot[KNODES - 1] / P;
  const double lo = (double)st->node[0], hi = (double)st->node[KNODES - 1];
  bool open = true;
  if (!(f0 <= T)) {  // root below the bracket (or NaN)
    if (!isfinite(f0)) {
      if (lane == 0) st->status |= ST_NONFINITE;
      resolve_warp(st, INFINITY, iter, lam_out, lane);
      return;
    }
    if (lo <= LAMBDA_LO * 1.000001) {
      if (lane == 0) st->status |= ST_NONCONVERGED;
      resolve_warp(st, LAMBDA_LO, iter, lam_out, lane);
      return;
    }
    set_bracket_warp(st, LAMBDA_LO, lo, lane);
  } else if (fK < T) {  // root above the bracket
    set_bracket_warp(st, hi, fmax(st->lam_up, hi * 4.0), lane);
  } else {
    int j = 0;
    while (j < KNODES - 2 && tot[j + 1] / P < T) ++j;
    const double sm = lane < KNODES ? st->snode[lane] : 0.0;
    const double fm = lane < KNODES ? tot[lane] / P : 0.0;
    const double W = st->snode[KNODES - 1] - st->snode[0];
    if (W <= W_EXACT) {
      const double lam = interp_root_warp(sm, fm, T, j, lane);
      resolve_warp(st, lam, iter, lam_out, lane);
      open = false;
    } else if (W <= W_ESTIMATE) {
      const double est = interp_root_warp(sm, fm, T, j, lane);
      __syncwarp();
      set_bracket_warp(st, est * (1.0 - EST_HALF_WIDTH), est * (1.0 + EST_HALF_WIDTH), lane);
    } else {
      const double nlo = (double)st->node[j], nhi = (double)st->node[j + 1];
      __syncwarp();
      set_bracket_warp(st, nlo, nhi, lane);
    }
  }
  if (open) {
    if (lane == 0) st->need = 1;
    if (last_chance) {
      if (lane == 0) st->status |= ST_NONCONVERGED;
      const double mid = sqrt(st->lo * st->hi);
      __syncwarp();
      resolve_warp(st, mid, iter, lam_out, lane);
    }
  }
}

}  // namespace gfd
