// Regularisation parameter by the discrepancy principle (Sec. 3.2).
//
// With a_b = |H_b|^2 and r_b = |H_b U_E,b - Y_b|^2 over all DFT bins b, the
// residual of u_p is f(lambda) = (1/P) sum_b lambda^2 r_b / (a_b + lambda)^2
// (Eq. 10-11 with Parseval's 1/P).  If ||h*u_E - y||^2 = f(inf) <= T the
// estimate is already in K and lambda = inf; otherwise lambda solves
// f(lambda) = T, whose root is unique because f increases (Eq. 11).
//
// GPU procedure (one spectral pass per evaluation, no host round trip):
//   each pass evaluates f at KNODES nodes lambda_j of the current bracket,
//   accumulating the per-bin terms in FP32 per thread and in FP64 across
//   warps and blocks; one warp of the image's last block then updates the
//   bracket.  Wide brackets use geometric nodes and are narrowed to the pair
//   of nodes that straddles T.  Brackets of ratio <= 4 use Chebyshev-
//   Lobatto nodes in t = ln(lambda): as a function of t, f is analytic in
//   the strip |Im t| < pi (its poles lie at lambda = -|H_b|^2 <= 0, i.e.
//   t = ln|H_b|^2 + i pi), whatever the spectrum, so the degree-11
//   interpolant in t through the node values has its root within ~1e-10
//   relative of the true one on a bracket of ratio 4 (~1e-14 on ratio 1.6).
//   Node values are rounded to FP32; their logarithms, formed once in FP64,
//   are the exact abscissae.  The interpolant is evaluated in double-float
//   arithmetic (FP64 is slow on this part), and its root is located by
//   multisection with one trial point per lane, which needs only the sign
//   of the interpolant.
// The first pass of each iteration is fused into the forward column FFT and
// uses a bracket of ratio 4 around an extrapolation of the previous lambdas.
// From iteration NARROW_FROM on, where the extrapolation comes within a few
// percent of the root, it evaluates KNARROW = 8 nodes on a bracket of ratio
// 1.56, whose degree-7 interpolant is as accurate as the degree-11 one on
// ratio 4 (the strip of analyticity is the same, the bracket's half-width in
// t three times smaller).  A root outside that bracket lies close to it: the
// fallback pass takes the ratio-4 bracket next to it.
#pragma once
#include "common.cuh"
#include "df.cuh"

namespace gfd {

constexpr float INTERP_RATIO = 4.0f;   // largest bracket ratio interpolated
constexpr float PRIMARY_RATIO = 2.0f;  // primary bracket: [c/2, 2 c]
constexpr float NARROW_RATIO = 1.25f;  // from iteration NARROW_FROM: [c/1.25, 1.25 c]
constexpr float NARROW_INTERP_RATIO = 1.6f;  // largest ratio interpolated with KNARROW nodes
constexpr float INITIAL_LO = 1e-8f, INITIAL_HI = 1e4f;
constexpr int MODE_GEOM = 0, MODE_CHEB = 1;

// Lanes of the warp that runs a per-image update (threads 0..31 of the
// block): the whole warp, or every thread of a block smaller than a warp
// (the column passes of 8- and 16-row canvases run 16 threads per block).
GFD_D int upd_lanes() { return blockDim.x >= 32 ? 32 : (int)blockDim.x; }
GFD_D unsigned int upd_mask() {
  return blockDim.x >= 32 ? 0xffffffffu : ((1u << blockDim.x) - 1u);
}

// cos(pi j / (n - 1)), j = 0..n-1 (Chebyshev-Lobatto points) for n = KNODES
// and n = KNARROW
__device__ constexpr float kLobatto[KNODES] = {
    1.0f, 0.9594929736144974f, 0.8412535328311812f, 0.6548607339452851f,
    0.41541501300188644f, 0.14231483827328512f, -0.142314838273285f, -0.4154150130018863f,
    -0.654860733945285f, -0.8412535328311811f, -0.9594929736144974f, -1.0f};
__device__ constexpr float kLobatto8[KNARROW] = {
    1.0f, 0.9009688679024191f, 0.6234898018587336f, 0.22252093395631445f,
    -0.2225209339563144f, -0.6234898018587335f, -0.900968867902419f, -1.0f};

// Node lambda_j (ascending) of a bracket [lo, hi] of nk nodes for the given
// layout (nodes j >= nk repeat hi and are not evaluated).
GFD_D float bracket_node(float lo, float hi, int mode, int j, int nk) {
  if (j == 0) return lo;
  if (j >= nk - 1) return hi;
  if (mode == MODE_CHEB) {  // Chebyshev-Lobatto in ln(lambda)
    const float c = nk == KNARROW ? kLobatto8[j] : kLobatto[j];
    return lo * exp2f(0.5f * (1.0f - c) * log2f(hi / lo));
  }
  return lo * exp2f((float)j / (nk - 1) * log2f(hi / lo));
}

// Chebyshev nodes (interpolated) for brackets narrow enough for nk nodes,
// geometric nodes (bracketed) otherwise.
GFD_D int bracket_mode(float lo, float hi, int nk) {
  return hi <= (nk == KNARROW ? NARROW_INTERP_RATIO : INTERP_RATIO) * lo ? MODE_CHEB : MODE_GEOM;
}

// Set the next pass's bracket of nk nodes (single thread).
GFD_D void set_bracket(ImgState* st, float lo, float hi, int nk = KNODES) {
  const int mode = bracket_mode(lo, hi, nk);
  st->lo = lo;
  st->hi = hi;
  st->mode = mode;
  st->nk = nk;
  for (int j = 0; j < KNODES; ++j) st->node[j] = bracket_node(lo, hi, mode, j, nk);
}

// Warp variant: lane j < KNODES writes node j.
GFD_D void set_bracket_warp(ImgState* st, float lo, float hi, int lane, int nk = KNODES) {
  const int mode = bracket_mode(lo, hi, nk);
  if (lane == 0) {
    st->lo = lo;
    st->hi = hi;
    st->mode = mode;
    st->nk = nk;
  }
  if (lane < KNODES) st->node[lane] = bracket_node(lo, hi, mode, lane, nk);
  __syncwarp(upd_mask());
}

// One bin's contribution: wr = (Hermitian weight) * r, a = |H|^2.
// t = lambda / (a + lambda) comes from an approximate reciprocal refined by
// one FMA residual step, which makes it (almost always) the correctly
// rounded quotient.  Without the step, every bin with a << lambda would carry
// the same reciprocal error for a given node: a node-dependent bias of ~1e-7
// in f(lambda_j) that moves the root by ~1e-7 / |d ln f / d ln lambda|,
// i.e. by percents where f is nearly flat in lambda.
// NK: the nodes the pass evaluates (acc[NK..KNODES-1] are left alone).
template <int NK = KNODES>
GFD_D void accum_bin(float wr, float a, const float* nodes, float* acc) {
  acc[KNODES] += wr;
#pragma unroll
  for (int j = 0; j < NK; ++j) {
    const float d = a + nodes[j];
    const float q = __fdividef(1.0f, d);
    const float t0 = nodes[j] * q;
    const float t = fmaf(fmaf(-t0, d, nodes[j]), q, t0);
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

// Long sums of the per-bin terms.  Threads keep FP32 partials over a short
// run of bins (one item); warp_fold adds the warp's total of each partial to
// per-warp double-float accumulators in shared memory (hi + lo, exact
// two-sum) and clears the partials; block_partials_folded turns the per-warp
// accumulators into the block's FP64 sums.  This keeps f(lambda) and
// ||h*u_E - y||^2 accurate to about 1e-10 relative over millions of bins,
// which matters where f is nearly flat in lambda.
struct WarpAcc {
  float hi[16][KNODES + 1];
  float lo[16][KNODES + 1];
};

GFD_D void warp_fold(float* acc, WarpAcc* wa) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int j = 0; j <= KNODES; ++j) {
    const float v = warp_sum(acc[j]);
    if (lane == 0) {
      const df t = two_sum(wa->hi[warp][j], v);
      wa->hi[warp][j] = t.hi;
      wa->lo[warp][j] += t.lo;
    }
    acc[j] = 0.0f;
  }
}

// part[j] = sum over warps of hi + lo (FP64); clears the accumulators.
// Synchronises before and after.
GFD_D void block_partials_folded(WarpAcc* wa, double* part) {
  __syncthreads();
  const int nwarp = num_warps();
  for (int j = threadIdx.x; j <= KNODES; j += blockDim.x) {
    double s = 0.0;
    for (int w = 0; w < nwarp; ++w) {
      s += (double)wa->hi[w][j] + (double)wa->lo[w][j];
      wa->hi[w][j] = 0.0f;
      wa->lo[w][j] = 0.0f;
    }
    part[j] = s;
  }
  __syncthreads();
}

// Zero the accumulators (every thread calls; synchronise before use).
GFD_D void warp_acc_clear(WarpAcc* wa) {
  float* p = &wa->hi[0][0];
  for (int i = threadIdx.x; i < 2 * 16 * (KNODES + 1); i += blockDim.x) p[i] = 0.0f;
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
// Several columns: one warp per column (a single barrier); one column: the
// whole block.
GFD_D void block_sum_columns(const double* vals, int n, int stride, int m, double* red,
                             double* sums) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int nwarp = num_warps();
  if (m > 1 && (blockDim.x & 31) == 0) {  // whole warps
    for (int j = warp; j < m; j += nwarp) {
      double s = 0.0;
      for (int i = lane; i < n; i += 32) s += __ldcg(&vals[(size_t)i * stride + j]);
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
      if (lane == 0) sums[j] = s;
    }
    __syncthreads();
    return;
  }
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

// Root of the interpolant in t = ln(lambda) through (t_m, g_m), m < KNODES,
// t_m = ln(x_m) of the FP32 node values x_m (ascending; g increasing through
// 0 between x_j and x_{j+1}).  Lane m < KNODES holds (x_m, g_m).  The
// logarithms are formed in FP64 and carried as double-float, as are the
// barycentric weights w_m = 1 / prod_{n != m} (t_m - t_n) of the actual nodes.
// Inside (t_j, t_{j+1}) the interpolant is p(t) = l(t) S(t) with
// l(t) = prod_m (t - t_m), whose sign there is (-1)^(nk-1-j) (nk nodes), and
// S(t) = sum_m w_m g_m / (t - t_m) (the first barycentric form), so the sign
// of p at a point needs S alone, one double-float quotient per node.  The
// root is bracketed by multisection: every lane evaluates the sign at its own
// trial point and the bracket shrinks to the two trial points that straddle
// the root.  After a plain round (one point per lane, spread evenly across
// the bracket; 32 lanes, or the block's threads if fewer) the next
// round's points sit in a window about the secant estimate from p at the
// bracket's ends (window half-width 1/16, then 1/256, then 1/4096 of the
// bracket while the root keeps falling inside it; a round whose window misses
// still leaves a valid bracket, and the next round is plain again).  Returns
// lambda = exp(t_root) at the bracket's midpoint once its width is <= rtol.
GFD_D df df_div_fast(df a, df b) {  // a / b, error ~2^-44 relative
  const float ib = __fdividef(1.0f, b.hi);
  const float q1 = a.hi * ib;
  const df p = two_prod(b.hi, q1);
  const float r = ((a.hi - p.hi) - p.lo + a.lo) - q1 * b.lo;  // a - q1 b
  return quick_two_sum(q1, r * ib);
}

GFD_D double interp_root_warp(float xm, float gm, int j, double rtol, int lane, int nk) {
  const bool own = lane < nk;
  const df tm = own ? df_from_double(log((double)xm)) : df_make(0.0f);
  // All abscissa differences are scaled by a power of two ~ 1/(node span):
  // exact, and it keeps the products of 11 differences in FP32 range (the
  // sign of S and the root do not depend on the scale).
  const float t0 = __shfl_sync(upd_mask(), tm.hi, 0);
  const float tK = __shfl_sync(upd_mask(), tm.hi, nk - 1);
  int ex;
  frexpf(tK - t0, &ex);
  const float sc = ldexpf(1.0f, -ex);
  df prod = df_make(1.0f);
  for (int n = 0; n < nk; ++n) {
    const df tn{__shfl_sync(upd_mask(), tm.hi, n), __shfl_sync(upd_mask(), tm.lo, n)};
    if (own && n != lane) {
      const df dd = df_sub(tm, tn);
      prod = df_mul(prod, df{dd.hi * sc, dd.lo * sc});
    }
  }
  const df c = own ? df_mul_f(df_rcp(prod), gm) : df_make(0.0f);  // w_m g_m
  __shared__ df s_t[KNODES], s_c[KNODES];
  __shared__ float s_g[KNODES];
  if (own) {
    s_t[lane] = tm;
    s_c[lane] = c;
    s_g[lane] = gm;
  }
  __syncwarp(upd_mask());
  const float sig = ((nk - 1 - j) & 1) ? -1.0f : 1.0f;  // sign of l(t) in the bracket
  df a = s_t[j], b = s_t[j + 1];
  float pa = s_g[j], pb = s_g[j + 1];  // p at the bracket's ends
  int level = 0;                       // windows in a row that held the root
  const int nl = upd_lanes();  // trial points per round
  const float inv_np1 = 1.0f / (float)(nl + 1);
  const float frac32 = (float)(lane + 1) * inv_np1;
  for (int round = 0; round < 24; ++round) {
    const df width = df_sub(b, a);
    if (df_to_double(width) <= rtol) break;  // absolute in t: relative in lambda
    // trial points: across the bracket, or across a window about the secant
    // estimate of the root
    df wlo = a, ww = width;
    if (level > 0) {
      const float est = pa / (pa - pb);
      if (est > 0.0f && est < 1.0f) {
        const float h = level == 1 ? 0.0625f : (level == 2 ? 0.00390625f : 0.000244140625f);
        const float f0 = fmaxf(est - h, 0.0f), f1 = fminf(est + h, 1.0f);
        wlo = df_add(a, df_mul_f(width, f0));
        ww = df_mul_f(width, f1 - f0);
      } else {
        level = 0;
      }
    }
    const df t = df_add(wlo, df_mul_f(ww, frac32));
    df S0 = df_make(0.0f), S1 = df_make(0.0f);  // two partial sums (shorter chains)
    float ell = 1.0f;
    bool at_node = false;
    float node_g = 0.0f;
    // add node m's term w_m g_m / (t - t_m) to S (t at a node: p(t) = g_m)
    auto term = [&](int m, df& S) {
      const df tmm = s_t[m];
      df d = two_sum(t.hi, -tmm.hi);
      d.lo += t.lo - tmm.lo;
      if (d.hi == 0.0f && d.lo == 0.0f) {
        at_node = true;
        node_g = s_g[m];
        return;
      }
      d = quick_two_sum(d.hi, d.lo);
      d.hi *= sc;
      d.lo *= sc;
      ell *= d.hi;
      const df q = df_div_fast(s_c[m], d);
      const df u = two_sum(S.hi, q.hi);
      S.hi = u.hi;
      S.lo += u.lo + q.lo;
    };
#pragma unroll 2
    for (int m = 0; m < nk; m += 2) {  // nk is even; registers stay low in the pass kernels
      term(m, S0);
      term(m + 1, S1);
    }
    const df Sv = df_add(quick_two_sum(S0.hi, S0.lo), quick_two_sum(S1.hi, S1.lo));
    const bool neg = at_node ? (node_g < 0.0f) : (sig * Sv.hi < 0.0f);
    const float pv = at_node ? node_g : ell * (Sv.hi + Sv.lo);  // p(t), for the estimate
    const unsigned below = __ballot_sync(upd_mask(), neg);
    // the interpolant increases: trial points below the root form a prefix
    const int nb = __popc(below);  // lanes 0..nb-1 are below the root
    const float p_lo = __shfl_sync(upd_mask(), pv, nb > 0 ? nb - 1 : 0);
    const float p_hi = __shfl_sync(upd_mask(), pv, nb < nl ? nb : nl - 1);
    const bool hit = nb > 0 && nb < nl;  // the root lies between two trial points
    if (nb > 0) {
      a = df_add(wlo, df_mul_f(ww, (float)nb * inv_np1));
      pa = p_lo;
    }
    if (nb < nl) {
      b = df_add(wlo, df_mul_f(ww, (float)(nb + 1) * inv_np1));
      pb = p_hi;
    }
    level = hit ? level + 1 : 0;
  }
  return exp(0.5 * (df_to_double(a) + df_to_double(b)));
}

// Record lambda_k and set the bracket of iteration k+1's fused first pass.
// lambda jumps by a factor of 2..150 from the first iteration (u_E = 0) to
// the second, and mostly falls to 0.2..1.2 of it in the third; later it
// changes smoothly, so the bracket is centred on the extrapolation
// lambda_k (lambda_k / lambda_{k-1}) (ratio clamped to [1/2, 2]).  The second
// iteration's bracket has geometric nodes, resolved by one more pass; the
// third's, [0.28, 1.1] lambda_1, and the later ones are narrow enough
// (ratio <= 4) for the interpolation to resolve them in the fused pass itself.
GFD_D void resolve_warp(ImgState* st, double lam, int iter, double* lam_out, int lane) {
  if (lane == 0) {
    st->lam = lam;
    st->need = 0;
    if (lam_out) lam_out[iter] = lam;
  }
  // the first pass of iteration iter + 1 evaluates nk nodes
  const int nk = iter + 1 >= NARROW_FROM ? KNARROW : KNODES;
  if (isfinite(lam) && lam > 0.0) {
    const float l = (float)lam;
    float lo, hi;
    if (iter == 0) {
      lo = l;
      hi = 150.0f * l;
    } else if (iter == 1) {
      lo = 0.28f * l;
      hi = 1.1f * l;
    } else {
      const double prev = st->lam_prev;
      float c = l;
      if (isfinite(prev) && prev > 0.0) c = l * fminf(fmaxf((float)(lam / prev), 0.5f), 2.0f);
      const float ratio = nk == KNARROW ? NARROW_RATIO : PRIMARY_RATIO;
      lo = c / ratio;
      hi = c * ratio;
    }
    lo = fmaxf(lo, (float)LAMBDA_LO);
    set_bracket_warp(st, lo, hi, lane, nk);  // ends with __syncwarp()
    if (lane == 0) st->lam_prev = lam;
  } else if (st->nk != nk) {
    // lambda = inf (or no finite root): the pending bracket is kept, laid
    // out for the node count of the next first pass
    const float lo = (float)st->lo, hi = (float)st->hi;
    __syncwarp(upd_mask());
    set_bracket_warp(st, lo, hi, lane, nk);
  }
  __syncwarp(upd_mask());
}

// Consume the totals of the pass that just completed for this image (tot:
// KNODES node sums and the residual sum, visible to the warp).  Run by the
// 32 lanes of one warp of the image's last block; every lane takes the same
// decisions from the same values.  FP64 is limited to a handful of
// operations (the sums themselves are FP64).
GFD_D void lambda_update_warp(ImgState* st, const double* tot, double P, bool primary,
                              bool last_chance, int iter, double* lam_out, double* res_out,
                              int lane) {
  const double invP = 1.0 / P;  // P is a power of two: exact
  const double T = st->T;
  const double resinf = tot[KNODES] * invP;
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
    if (lane == 0) {
      const float t = sqrtf((float)T / (float)resinf);
      st->lam_up = fminf(1e30f, (float)st->amax * t / (1.0f - t));
    }
    __syncwarp(upd_mask());
  }
  // g_m = f(lambda_m) / T - 1, increasing in lambda, for the nk nodes the
  // pass evaluated
  const int nk = st->nk;
  const float gm = lane < nk ? (float)((tot[lane] * invP - T) * st->invT) : 0.0f;
  const float xm = lane < nk ? st->node[lane] : 0.0f;
  const float g0 = __shfl_sync(upd_mask(), gm, 0);
  const float gK = __shfl_sync(upd_mask(), gm, nk - 1);
  const float lo = __shfl_sync(upd_mask(), xm, 0);
  const float hi = __shfl_sync(upd_mask(), xm, nk - 1);
  const int mode = st->mode;
  // a missed first bracket whose root is expected close to it
  const bool near = nk == KNARROW || (primary && iter == 2 && mode == MODE_CHEB);
  bool open = true;
  if (!(g0 <= 0.0f)) {  // root below the bracket (or NaN)
    if (!isfinite(g0)) {
      if (lane == 0) st->status |= ST_NONFINITE;
      resolve_warp(st, INFINITY, iter, lam_out, lane);
      return;
    }
    if (lo <= (float)LAMBDA_LO * 1.000001f) {
      if (lane == 0) st->status |= ST_NONCONVERGED;
      resolve_warp(st, LAMBDA_LO, iter, lam_out, lane);
      return;
    }
    // below a narrow first bracket, or the third iteration's first bracket
    // (four passes to go): the ratio-4 bracket just under it; otherwise
    // everything down to the smallest lambda
    const float nlo = near ? fmaxf(0.25f * lo, (float)LAMBDA_LO) : (float)LAMBDA_LO;
    set_bracket_warp(st, nlo, lo, lane);
  } else if (gK < 0.0f) {  // root above the bracket
    // above a narrow first bracket: the ratio-4 bracket just over it;
    // otherwise up to the bound from res and |H|^2
    set_bracket_warp(st, hi, near ? 4.0f * hi : fmaxf(st->lam_up, hi * 4.0f), lane);
  } else {
    // nodes with g < 0 form a prefix 0..j
    const unsigned below = __ballot_sync(upd_mask(), lane < nk && gm < 0.0f);
    int j = 31 - __clz(below | 1u);
    if (j > nk - 2) j = nk - 2;
    if (mode == MODE_CHEB) {
      const double lam = interp_root_warp(xm, gm, j, st->rtol, lane, nk);
      resolve_warp(st, lam, iter, lam_out, lane);
      open = false;
    } else {
      const float nlo = __shfl_sync(upd_mask(), xm, j), nhi = __shfl_sync(upd_mask(), xm, j + 1);
      set_bracket_warp(st, nlo, nhi, lane);
    }
  }
  if (open) {
    if (lane == 0) st->need = 1;
    if (last_chance) {  // the pass schedule ran out with the bracket still open
      if (lane == 0) st->status |= ST_PASSES_EXHAUSTED;
      const double mid = sqrt((double)st->lo * (double)st->hi);
      __syncwarp(upd_mask());
      resolve_warp(st, mid, iter, lam_out, lane);
    }
  }
}

}  // namespace gfd
