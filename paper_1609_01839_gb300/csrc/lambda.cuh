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

GFD_D void set_bracket(ImgState* st, double lo, double hi) {
  st->lo = lo;
  st->hi = hi;
  const double a = log(lo), b = log(hi);
  const double c = 0.5 * (a + b), h = 0.5 * (b - a);
#pragma unroll
  for (int j = 0; j < KNODES; ++j) {
    const double s = c - h * cos(PI_D * j / (KNODES - 1));
    st->node[j] = (float)exp(s);
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

// Barycentric interpolant of (s_m, f_m) at s.
GFD_D double bary_eval(const double* s, const double* f, const double* wb, double x) {
  double num = 0.0, den = 0.0;
#pragma unroll
  for (int m = 0; m < KNODES; ++m) {
    const double d = x - s[m];
    if (d == 0.0) return f[m];
    const double t = wb[m] / d;
    num += t * f[m];
    den += t;
  }
  return num / den;
}

// Root of the interpolant minus T in [s[j], s[j+1]] (Illinois false position
// safeguarded by bisection), returned as lambda.
GFD_D double interp_root(const double* s, const double* f, double T, int j) {
  double wb[KNODES];
#pragma unroll
  for (int m = 0; m < KNODES; ++m) {
    double p = 1.0;
    for (int n = 0; n < KNODES; ++n)
      if (n != m) p *= (s[m] - s[n]);
    wb[m] = 1.0 / p;
  }
  double a = s[j], b = s[j + 1];
  double fa = f[j] - T, fb = f[j + 1] - T;
  if (fa == 0.0) return exp(a);
  if (fb == 0.0) return exp(b);
  int side = 0;
  for (int it = 0; it < 100; ++it) {
    double c = (fb * a - fa * b) / (fb - fa);
    if (!(c > a && c < b)) c = 0.5 * (a + b);
    const double fc = bary_eval(s, f, wb, c) - T;
    if (fc == 0.0) return exp(c);
    if ((fc < 0.0) == (fa < 0.0)) {
      a = c;
      fa = fc;
      if (side == -1) fb *= 0.5;
      side = -1;
    } else {
      b = c;
      fb = fc;
      if (side == 1) fa *= 0.5;
      side = 1;
    }
    if (b - a <= 1e-15 * fmax(1.0, fabs(a))) break;
  }
  return exp(0.5 * (a + b));
}

GFD_D void resolve(ImgState* st, double lam, int iter, double* lam_out) {
  st->lam = lam;
  st->need = 0;
  if (lam_out) lam_out[iter] = lam;
  if (isfinite(lam) && lam > 0.0) set_bracket(st, lam / PRIMARY_RATIO, lam * PRIMARY_RATIO);
}

// Consume the accumulators of the pass that just completed for this image.
// Run by one thread of the image's last block.
GFD_D void lambda_update(ImgState* st, const double* tot, double P, bool primary,
                         bool last_chance, int iter, double* lam_out, double* res_out) {
  double f[KNODES];
  for (int j = 0; j < KNODES; ++j) f[j] = tot[j] / P;
  const double resinf = tot[KNODES] / P;
  const double T = st->T;
  if (primary) {
    st->res = resinf;
    if (res_out) res_out[iter] = resinf;
    if (!isfinite(resinf)) {
      st->status |= ST_NONFINITE;
      resolve(st, INFINITY, iter, lam_out);
      return;
    }
    if (resinf <= T) {  // u_E in K (Sec. 3.2): lambda = inf, u_I = u_p = u_E
      resolve(st, INFINITY, iter, lam_out);
      return;
    }
    const double t = sqrt(T / resinf);
    st->lam_up = fmin(1e30, st->amax * t / (1.0 - t));
  }
  double s[KNODES];
  for (int j = 0; j < KNODES; ++j) s[j] = log((double)st->node[j]);
  const double lo = (double)st->node[0], hi = (double)st->node[KNODES - 1];
  bool open = true;
  if (!(f[0] <= T)) {  // root below the bracket (or NaN)
    if (!isfinite(f[0])) {
      st->status |= ST_NONFINITE;
      resolve(st, INFINITY, iter, lam_out);
      return;
    }
    if (lo <= LAMBDA_LO * 1.000001) {
      st->status |= ST_NONCONVERGED;
      resolve(st, LAMBDA_LO, iter, lam_out);
      return;
    }
    set_bracket(st, LAMBDA_LO, lo);
  } else if (f[KNODES - 1] < T) {  // root above the bracket
    set_bracket(st, hi, fmax(st->lam_up, hi * 4.0));
  } else {
    int j = 0;
    while (j < KNODES - 2 && f[j + 1] < T) ++j;
    const double W = s[KNODES - 1] - s[0];
    if (W <= W_EXACT) {
      resolve(st, interp_root(s, f, T, j), iter, lam_out);
      open = false;
    } else if (W <= W_ESTIMATE) {
      const double est = interp_root(s, f, T, j);
      set_bracket(st, est * (1.0 - EST_HALF_WIDTH), est * (1.0 + EST_HALF_WIDTH));
    } else {
      set_bracket(st, (double)st->node[j], (double)st->node[j + 1]);
    }
  }
  if (open) {
    st->need = 1;
    if (last_chance) {
      st->status |= ST_NONCONVERGED;
      resolve(st, sqrt(st->lo * st->hi), iter, lam_out);
    }
  }
}

}  // namespace gfd
