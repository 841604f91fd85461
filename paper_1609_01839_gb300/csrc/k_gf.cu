// Guided filter u = guidfilter(u_I, u_p, w, eps) (Sec. 2, Eq. 3-5), r = (w-1)/2,
// with periodic windows (every window holds w^2 pixels) or windows truncated
// at the canvas edge (every mean divided by the number of pixels it covers).
//
// Every warp works alone, down a strip of GFW_COLS input columns (4 per
// lane): no block barriers.  Input rows enter a per-warp ring in shared
// memory by 16-byte asynchronous copies GFW_AHEAD rows ahead of use; each lane
// copies and reads only its own 4 columns.  For the item's rows the warp
// forms, row by row,
//   1. window sums down its columns of J = I - c_I, Q = p - c_p, J^2, J Q
//      (in registers; slid from row to row, and for plain FP32 sums re-formed
//      directly every 4 rows),
//   2. window sums along the row by warp shuffles (the 2r neighbouring
//      columns come from the adjacent lanes) -> mu_k, pbar_k, sigma_k^2 and
//      the covariance -> a_k (Eq. 3), b_k (Eq. 4) for each column,
//   3. window sums of a and b down the columns (a per-warp ring of the last
//      2r+1 rows of a, b in shared memory, each lane touching only its own
//      columns), re-formed every 4 rows and slid in between,
//   4. window sums along the row by shuffles -> abar, bbar ->
//      u = abar I + bbar (Eq. 5), stored as 16-byte vectors.
// The strip's outer 4*ceil(r/2) columns on each side are halo (their sums
// are incomplete); the columns in between are the item's output, so
// neighbouring strips overlap by the halo.  Input rows and columns wrap
// periodically (truncated windows mask the wrapped ones to zero).  Window
// statistics are taken about reference values (c_I, c_p: the item's centre
// pixel): a_k and b_k do not depend on them, and the sums of J^2 and J Q are
// smaller about a nearby reference.
//
// The arithmetic of the window sums of step 1-2 is a policy (GFD_VAR_*):
// double-float running sums (every addition and product error-free), FP64
// accumulators, or plain FP32.  sigma_k^2 and the covariance are then formed
// as (n S_JJ - S_J^2) / n^2 and (n S_JQ - S_J S_Q) / n^2 in that arithmetic
// and rounded to FP32 once.
#include <type_traits>

#include "common.cuh"
#include "df.cuh"
#include "launch.h"

namespace gfd {

constexpr int GFW_COLS = 128;   // input columns per strip (4 per lane)
constexpr int GFW_SUB = 4;      // rows between direct re-formations of FP32 column sums
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

// ---------------------------------------------------------------------------
// Window-sum arithmetic (one policy per GFD_VAR_* mode).  kSub: rows between
// direct re-formations of the column sums (the exact policies only slide).
// ---------------------------------------------------------------------------
struct SumF32 {
  static constexpr int kSub = GFW_SUB;
  float v;
  GFD_D void clear() { v = 0.0f; }
  GFD_D void add(float x) { v += x; }
  GFD_D void add_prod(float x, float y) { v = fmaf(x, y, v); }
};

struct SumF64 {
  static constexpr int kSub = 1 << 30;
  double v;
  GFD_D void clear() { v = 0.0; }
  GFD_D void add(float x) { v += (double)x; }
  GFD_D void add_prod(float x, float y) { v = fma((double)x, (double)y, v); }  // exact product
};

// hi: the FP32-rounded running sum; lo: the exact rounding errors of every
// addition (two-sum) and product (two-product), summed in FP32.
struct SumDF {
  static constexpr int kSub = 1 << 30;
  float hi, lo;
  GFD_D void clear() { hi = lo = 0.0f; }
  GFD_D void add(float x) {
    const df t = two_sum(hi, x);
    hi = t.hi;
    lo += t.lo;
  }
  GFD_D void add_prod(float x, float y) {
    const float p = x * y;
    const float e = fmaf(x, y, -p);
    const df t = two_sum(hi, p);
    hi = t.hi;
    lo += t.lo + e;
  }
};

// Split sums.  Every deviation x (J or Q) is split on a power-of-two grid g
// chosen per item from a bound on |x| (g >= 2^-b max |x|): x = g m + x_l with
// m = round(x / g), |m| <= 2^b, and x_l = x - g m (exact).  Window sums of m,
// m_J^2 and m_J m_Q are exact in int32 on the integer pipe, and so are
// n S_mm - S_m^2 and n S_mJ mQ - S_mJ S_mQ: b = split_bits(r) is the largest
// with n^2 2^(2b) < 2^31 for windows of n = (2r+1)^2 pixels (11 at most).
// The remainders' parts, x_l, J^2 - (g_J m_J)^2 = J_l (J + g_J m_J) and
// J Q - g_J m_J g_Q m_Q = g_J m_J Q_l + J_l Q, are summed in FP32, where
// their rounding is 2^-b of that of plain sums.
struct SumIG {
  static constexpr int kSub = 1 << 30;
  int h;
  float l;
};

// The grids of one item: g, 1/g and g * kMagic for J and for Q.
struct IGGrid {
  float gJ, igJ, mgJ, gQ, igQ, mgQ;
};

constexpr float kMagic = 12582912.0f;  // 1.5 * 2^23: adding it rounds |v| < 2^22 to an integer

// Bits of the split's integer part for windows of radius r: the largest b
// <= 11 with ((2r+1)^2)^2 2^(2b) < 2^31 (r = 2: 10, r = 3, 4: 9, r = 8: 7).
constexpr int split_bits(int rad) {
  const long long n = (long long)(2 * rad + 1) * (2 * rad + 1);
  int b = 11;
  while (b > 0 && n * n * (1LL << (2 * b)) >= (1LL << 31)) --b;
  return b;
}

static_assert(split_bits(2) == 10 && split_bits(3) == 9 && split_bits(4) == 9 &&
                  split_bits(8) == 7 && split_bits(0) == 11,
              "split bits per window radius");

template <int RAD>
GFD_D void ig_grid(float bound, float& g, float& ig, float& mg) {
  constexpr int B = split_bits(RAD);
  int e = 0;
  if (bound > 0.0f && bound < 3e38f) frexpf(bound, &e);  // bound <= 2^e
  if (e < -100) e = -100;
  g = ldexpf(1.0f, e - B);
  ig = ldexpf(1.0f, B - e);
  mg = kMagic * g;
}

// x = g m + xl: m = round(x / g) (kMagic + x / g rounds to an integer-valued
// float whose low bits are m), g m exact, xl = x - g m exact.
GFD_D void ig_split(float x, float ig, float g, float mg, int& m, float& xh, float& xl) {
  const float t = fmaf(x, ig, kMagic);
  m = __float_as_int(t) - __float_as_int(kMagic);
  xh = fmaf(t, g, -mg);
  xl = x - xh;
}

// int32 |v| < 2^22 to float, exactly, without a conversion instruction
GFD_D float small_int_to_float(int v) {
  return __int_as_float(__float_as_int(kMagic) + v) - kMagic;
}

// Value of lane (lane + off) (compile-time offset after unrolling).
template <class T>
GFD_D T lane_shift(T v, int off) {
  if (off > 0) return __shfl_down_sync(FULL, v, off);
  if (off < 0) return __shfl_up_sync(FULL, v, -off);
  return v;
}

// e[q] = the value of strip column 4*lane + q - RAD, q < 2 RAD + 4, gathered
// from v[k] = column 4*lane + k of every lane.  Columns beyond the warp's
// edges are not available: lanes within RAD columns of an edge get values
// of other columns (those lanes' sums are halo and never used).
template <int RAD, class T>
GFD_D void gather_row(const T (&v)[4], T (&e)[2 * RAD + 4]) {
#pragma unroll
  for (int q = 0; q < 2 * RAD + 4; ++q) {
    const int c = q - RAD;                           // column offset from 4*lane
    const int lo = c >= 0 ? c / 4 : -((3 - c) / 4);  // floor(c / 4): source lane offset
    e[q] = lane_shift(v[c - 4 * lo], lo);
  }
}

// Window sums of radius RAD along the strip: s[k] = sum of columns
// 4*lane + k - RAD .. 4*lane + k + RAD.
template <int RAD, class T>
GFD_D void hsum4_scalar(const T (&v)[4], T (&s)[4]) {
  T e[2 * RAD + 4];
  gather_row<RAD>(v, e);
  T acc = e[0];
#pragma unroll
  for (int q = 1; q <= 2 * RAD; ++q) acc += e[q];
  s[0] = acc;
#pragma unroll
  for (int k = 1; k < 4; ++k) {
    acc += e[k + 2 * RAD] - e[k - 1];
    s[k] = acc;
  }
}

template <int RAD>
GFD_D void hsum4(const float (&v)[4], float (&s)[4]) {
  hsum4_scalar<RAD>(v, s);
}

template <int RAD>
GFD_D void hsum4(const SumF32 (&v)[4], SumF32 (&s)[4]) {
  const float in[4] = {v[0].v, v[1].v, v[2].v, v[3].v};
  float out[4];
  hsum4_scalar<RAD>(in, out);
#pragma unroll
  for (int k = 0; k < 4; ++k) s[k].v = out[k];
}

template <int RAD>
GFD_D void hsum4(const SumF64 (&v)[4], SumF64 (&s)[4]) {
  const double in[4] = {v[0].v, v[1].v, v[2].v, v[3].v};
  double out[4];
  hsum4_scalar<RAD>(in, out);
#pragma unroll
  for (int k = 0; k < 4; ++k) s[k].v = out[k];
}

// Double-float: the hi parts are added with two-sums (errors kept), the lo
// parts (already the errors of the column sums) plainly.
template <int RAD>
GFD_D void hsum4(const SumDF (&v)[4], SumDF (&s)[4]) {
  constexpr int E = 2 * RAD + 4;
  const float vh[4] = {v[0].hi, v[1].hi, v[2].hi, v[3].hi};
  const float vl[4] = {v[0].lo, v[1].lo, v[2].lo, v[3].lo};
  float eh[E], el[E];
  gather_row<RAD>(vh, eh);
  gather_row<RAD>(vl, el);
  float hi = eh[0], err = 0.0f, lo = el[0];
#pragma unroll
  for (int q = 1; q <= 2 * RAD; ++q) {
    const df t = two_sum(hi, eh[q]);
    hi = t.hi;
    err += t.lo;
    lo += el[q];
  }
  s[0].hi = hi;
  s[0].lo = err + lo;
#pragma unroll
  for (int k = 1; k < 4; ++k) {
    df t = two_sum(hi, eh[k + 2 * RAD]);
    err += t.lo;
    t = two_sum(t.hi, -eh[k - 1]);
    hi = t.hi;
    err += t.lo;
    lo += el[k + 2 * RAD] - el[k - 1];
    s[k].hi = hi;
    s[k].lo = err + lo;
  }
}

template <int RAD>
GFD_D void hsum4(const SumIG (&v)[4], SumIG (&s)[4]) {
  const int ih[4] = {v[0].h, v[1].h, v[2].h, v[3].h};
  const float il[4] = {v[0].l, v[1].l, v[2].l, v[3].l};
  int oh[4];
  float ol[4];
  hsum4_scalar<RAD>(ih, oh);
  hsum4_scalar<RAD>(il, ol);
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    s[k].h = oh[k];
    s[k].l = ol[k];
  }
}

// Means and (co)variance of a window of n pixels from S = (sum J, sum Q,
// sum J^2, sum J Q):  var = (n S_JJ - S_J^2) / n^2 (sigma_k^2, the
// population variance), cov = (n S_JQ - S_J S_Q) / n^2.
GFD_D void window_stats(const SumF32& s0, const SumF32& s1, const SumF32& s2, const SumF32& s3,
                        float n, float inv_n, const IGGrid&, float& mJ, float& mQ, float& var,
                        float& cov) {
  (void)n;
  mJ = s0.v * inv_n;
  mQ = s1.v * inv_n;
  var = fmaf(-mJ, mJ, s2.v * inv_n);
  cov = fmaf(-mJ, mQ, s3.v * inv_n);
}

GFD_D void window_stats(const SumF64& s0, const SumF64& s1, const SumF64& s2, const SumF64& s3,
                        float n, float inv_n, const IGGrid&, float& mJ, float& mQ, float& var,
                        float& cov) {
  (void)inv_n;
  const double nn = (double)n, inv2 = 1.0 / (nn * nn);
  mJ = (float)(s0.v / nn);
  mQ = (float)(s1.v / nn);
  var = (float)(fma(nn, s2.v, -s0.v * s0.v) * inv2);
  cov = (float)(fma(nn, s3.v, -s0.v * s1.v) * inv2);
}

GFD_D void window_stats(const SumDF& s0, const SumDF& s1, const SumDF& s2, const SumDF& s3,
                        float n, float inv_n, const IGGrid&, float& mJ, float& mQ, float& var,
                        float& cov) {
  const df S0{s0.hi, s0.lo}, S1{s1.hi, s1.lo}, S2{s2.hi, s2.lo}, S3{s3.hi, s3.lo};
  const df v = df_sub(df_mul_f(S2, n), df_mul(S0, S0));
  const df c = df_sub(df_mul_f(S3, n), df_mul(S0, S1));
  const float inv2 = inv_n * inv_n;
  mJ = (s0.hi + s0.lo) * inv_n;
  mQ = (s1.hi + s1.lo) * inv_n;
  var = (v.hi + v.lo) * inv2;
  cov = (c.hi + c.lo) * inv2;
}

// Split sums: the integer parts of n S_JJ - S_J^2 and n S_JQ - S_J S_Q are
// exact in int32 (the split's bits keep every product below 2^31, and E by
// Cauchy-Schwarz; the differences are formed in modular unsigned arithmetic);
// the remainders' parts are added in FP32.
GFD_D void window_stats(const SumIG& s0, const SumIG& s1, const SumIG& s2, const SumIG& s3,
                        float n, float inv_n, const IGGrid& G, float& mJ, float& mQ, float& var,
                        float& cov) {
  const unsigned ni = (unsigned)(int)n;
  const int D = (int)(ni * (unsigned)s2.h - (unsigned)s0.h * (unsigned)s0.h);
  const int E = (int)(ni * (unsigned)s3.h - (unsigned)s0.h * (unsigned)s1.h);
  const float hJ = G.gJ * small_int_to_float(s0.h);  // g_J sum m_J (exact)
  const float hQ = G.gQ * small_int_to_float(s1.h);
  const float lv = fmaf(n, s2.l, -fmaf(2.0f * hJ + s0.l, s0.l, 0.0f));
  const float lc = fmaf(n, s3.l, -fmaf(hJ, s1.l, fmaf(hQ + s1.l, s0.l, 0.0f)));
  const float inv2 = inv_n * inv_n;
  mJ = (hJ + s0.l) * inv_n;
  mQ = (hQ + s1.l) * inv_n;
  var = fmaf(G.gJ * G.gJ, __int2float_rn(D), lv) * inv2;
  cov = fmaf(G.gJ * G.gQ, __int2float_rn(E), lc) * inv2;
}

// Column-sum update by one input row's deviations (sign +1: the row enters,
// -1: it leaves).
template <class ACC>
GFD_D void col_update(ACC (&V)[4][4], const float (&J)[4], const float (&Q)[4], float sgn,
                      const IGGrid&) {
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    V[0][k].add(sgn * J[k]);
    V[1][k].add(sgn * Q[k]);
    V[2][k].add_prod(sgn * J[k], J[k]);
    V[3][k].add_prod(sgn * J[k], Q[k]);
  }
}

GFD_D void col_update(SumIG (&V)[4][4], const float (&J)[4], const float (&Q)[4], float sgn,
                      const IGGrid& G) {
  const int si = sgn > 0.0f ? 1 : -1;
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    int mJ, mQ;
    float Jh, Jl, Qh, Ql;
    ig_split(J[k], G.igJ, G.gJ, G.mgJ, mJ, Jh, Jl);
    ig_split(Q[k], G.igQ, G.gQ, G.mgQ, mQ, Qh, Ql);
    const int smJ = si * mJ;
    V[0][k].h += smJ;
    V[1][k].h += si * mQ;
    V[2][k].h += smJ * mJ;
    V[3][k].h += smJ * mQ;
    const float sJl = sgn * Jl;
    V[0][k].l += sJl;
    V[1][k].l += sgn * Ql;
    V[2][k].l = fmaf(sJl, J[k] + Jh, V[2][k].l);
    V[3][k].l = fmaf(sgn * Jh, Ql, fmaf(sJl, Q[k], V[3][k].l));
  }
}

template <class ACC>
GFD_D void col_clear(ACC (&V)[4][4]) {
#pragma unroll
  for (int q = 0; q < 4; ++q)
#pragma unroll
    for (int k = 0; k < 4; ++k) V[q][k].clear();
}
GFD_D void col_clear(SumIG (&V)[4][4]) {
#pragma unroll
  for (int q = 0; q < 4; ++q)
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      V[q][k].h = 0;
      V[q][k].l = 0.0f;
    }
}

// Pixels of the window of radius RAD about position x in [0, L) that lie in
// [0, L) (truncated windows).
GFD_D int window_count(int x, int L, int RAD) {
  const int a = x - RAD < 0 ? 0 : x - RAD;
  const int b = x + RAD > L - 1 ? L - 1 : x + RAD;
  return b - a + 1;
}

template <int RAD, class ACC, bool TRUNC>
GFD_D void gfw_items(const ClassDesc& cd, const ImgDesc* __restrict__ imgs, ImgState* st,
                     int iter, bool shifted, int H, float* ring, int gwarp, int nwarps) {
  using G = GfwGeom<RAD>;
  constexpr int WIN = G::WIN, HALO = G::HALO, WOUT = G::WOUT, RI = G::RI;
  const int lane = threadIdx.x & 31;
  const int M = cd.M, N = cd.N;
  const int strips = (N + WOUT - 1) / WOUT;
  const int per_img = strips * (M / H);
  const int n_items = cd.n_img * per_img;
  const float n_full = (float)(WIN * WIN);
  const float inv_full = 1.0f / n_full;
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
    const int xs = x0 - HALO + 4 * lane;  // unwrapped column of the lane's first value
    const int gx = xs & (N - 1);
    const bool store = out_lane && x0 + 4 * lane - HALO < N;
    // truncated windows: columns outside the canvas hold zero, and every
    // window's pixel count along the row
    float cmask[4] = {1.0f, 1.0f, 1.0f, 1.0f}, ncol[4] = {0.0f, 0.0f, 0.0f, 0.0f};
    if constexpr (TRUNC) {
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const int x = xs + k;
        const bool in = x >= 0 && x < N;
        cmask[k] = in ? 1.0f : 0.0f;
        ncol[k] = in ? (float)window_count(x, N, RAD) : 1.0f;
      }
    }
    float cI = 0.0f, cP = 0.0f;
    if (shifted) {
      const size_t c = (size_t)((y0 + H / 2) & (M - 1)) * N + ((x0 + WOUT / 2) & (N - 1));
      cI = __ldg(&I[c]);
      cP = __ldg(&P[c]);
    }
    const float eps = (float)d.eps;
    IGGrid G{};
    if constexpr (std::is_same<ACC, SumIG>::value) {
      // |J| <= max |u_I| + |c_I| (the bound the inverse row pass recorded)
      const ImgState* S = st + gi;
      ig_grid<RAD>(__uint_as_float(__ldcg(&S->absmax[0])) + fabsf(cI), G.gJ, G.igJ, G.mgJ);
      ig_grid<RAD>(__uint_as_float(__ldcg(&S->absmax[1])) + fabsf(cP), G.gQ, G.igQ, G.mgQ);
    }
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
    // deviations of input row j about the references (zero outside the
    // canvas for truncated windows)
    auto devs = [&](int j, float (&J)[4], float (&Q)[4]) {
      const float4 iv = ring4(rI, j), pv = ring4(rP, j);
      J[0] = iv.x - cI; J[1] = iv.y - cI; J[2] = iv.z - cI; J[3] = iv.w - cI;
      Q[0] = pv.x - cP; Q[1] = pv.y - cP; Q[2] = pv.z - cP; Q[3] = pv.w - cP;
      if constexpr (TRUNC) {
        const int yy = y0 - 2 * RAD + j;
        const float rm = (yy >= 0 && yy < M) ? 1.0f : 0.0f;
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          J[k] *= rm * cmask[k];
          Q[k] *= rm * cmask[k];
        }
      }
    };
    for (int j = 0; j <= 2 * RAD; ++j) fetch(j);
    cp_async_commit();
#pragma unroll
    for (int a = 1; a < GFW_AHEAD; ++a) {
      fetch(2 * RAD + a);
      cp_async_commit();
    }
    ACC V[4][4];     // [J, Q, J^2, J Q][column]: window sums down the columns
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
      if (s % ACC::kSub == 0) {
        col_clear(V);
#pragma unroll
        for (int dd = 0; dd < WIN; ++dd) {
          float J[4], Q[4];
          devs(s + dd, J, Q);
          col_update(V, J, Q, 1.0f, G);
        }
      } else {
        float Jn[4], Qn[4], Jo[4], Qo[4];
        devs(s + 2 * RAD, Jn, Qn);
        devs(s - 1, Jo, Qo);
        col_update(V, Jn, Qn, 1.0f, G);
        col_update(V, Jo, Qo, -1.0f, G);
      }
      // 2. row window sums -> a_k (Eq. 3), b_k (Eq. 4)
      ACC S0[4], S1[4], S2[4], S3[4];
      hsum4<RAD>(V[0], S0);
      hsum4<RAD>(V[1], S1);
      hsum4<RAD>(V[2], S2);
      hsum4<RAD>(V[3], S3);
      float A[4], B[4];
      float nrow = 0.0f, srow_mask = 1.0f;
      if constexpr (TRUNC) {
        const int ys = y0 - RAD + s;
        const bool in = ys >= 0 && ys < M;
        srow_mask = in ? 1.0f : 0.0f;
        nrow = in ? (float)window_count(ys, M, RAD) : 1.0f;
      }
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        float n = n_full, inv_n = inv_full;
        if constexpr (TRUNC) {
          n = nrow * ncol[k];
          inv_n = __frcp_rn(n);
        }
        float mJ, mQ, var, cov;
        window_stats(S0[k], S1[k], S2[k], S3[k], n, inv_n, G, mJ, mQ, var, cov);
        A[k] = __fdividef(cov, var + eps);  // var + eps >= eps > 0
        // b_k about the references: b_k = B_k + c_p - a_k c_I (Eq. 4), and the
        // constant parts are restored in the output below
        B[k] = fmaf(-A[k], mJ, mQ);
        if constexpr (TRUNC) {  // windows centred outside the canvas do not exist
          const float m = srow_mask * cmask[k];
          A[k] *= m;
          B[k] *= m;
        }
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
      //    at output row t is input row j = t + 2r = s.  With b_k = B_k + c_p
      //    - a_k c_I, u = abar (I - c_I) + Bbar + c_p: no large terms cancel
      //    where I and p are large (small lambda amplifies noise in them)
      float SA[4], SB[4];
      hsum4<RAD>(VA[0], SA);
      hsum4<RAD>(VA[1], SB);
      const float4 iv = ring4(rI, s);
      const float ic[4] = {iv.x - cI, iv.y - cI, iv.z - cI, iv.w - cI};
      float nout = 0.0f;
      if constexpr (TRUNC) nout = (float)window_count(y0 + t, M, RAD);
      float o[4];
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        float inv_n = inv_full;
        if constexpr (TRUNC) inv_n = __frcp_rn(nout * ncol[k]);
        o[k] = fmaf(fmaf(SA[k], ic[k], SB[k]), inv_n, cP);
      }
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

template <class ACC, bool TRUNC>
__global__ void __launch_bounds__(GFW_WARPS * 32)
k_guided_filter(ClassDesc cd, const ImgDesc* __restrict__ imgs, ImgState* st, int iter,
                int shifted_i, int rad, int H) {
  extern __shared__ __align__(16) float gsm[];
  const int warp = threadIdx.x >> 5;
  const int gwarp = blockIdx.x * GFW_WARPS + warp;
  const int nwarps = gridDim.x * GFW_WARPS;
  float* ring = gsm + (size_t)warp * gfw_ring_floats(rad);
  const bool shifted = shifted_i != 0;
#define GFD_GF_CASE(R) \
  case R: gfw_items<R, ACC, TRUNC>(cd, imgs, st, iter, shifted, H, ring, gwarp, nwarps); break;
  switch (rad) {
    GFD_GF_CASE(0) GFD_GF_CASE(1) GFD_GF_CASE(2) GFD_GF_CASE(3) GFD_GF_CASE(4)
    GFD_GF_CASE(5) GFD_GF_CASE(6) GFD_GF_CASE(7)
    default: gfw_items<8, ACC, TRUNC>(cd, imgs, st, iter, shifted, H, ring, gwarp, nwarps); break;
  }
#undef GFD_GF_CASE
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

using GfKernel = void (*)(ClassDesc, const ImgDesc*, ImgState*, int, int, int, int);

static GfKernel gf_kernel(int var_mode, int boundary) {
  const bool tr = boundary == GFD_BOUNDARY_TRUNCATED;
  switch (var_mode) {
    case GFD_VAR_FP64: return tr ? k_guided_filter<SumF64, true> : k_guided_filter<SumF64, false>;
    case GFD_VAR_FP32:
    case GFD_VAR_FP32_RAW: return tr ? k_guided_filter<SumF32, true> : k_guided_filter<SumF32, false>;
    case GFD_VAR_DOUBLE_FLOAT:
      return tr ? k_guided_filter<SumDF, true> : k_guided_filter<SumDF, false>;
    default: return tr ? k_guided_filter<SumIG, true> : k_guided_filter<SumIG, false>;
  }
}

// Largest |I| and |p| of each image of a class into ImgState::absmax (the
// bound of the split sums when no inverse row pass has recorded it).
__global__ void k_plane_absmax(ClassDesc cd, const ImgDesc* __restrict__ imgs, ImgState* st) {
  const int gi = cd.img0 + blockIdx.y;
  const ImgDesc& d = imgs[gi];
  const size_t P = (size_t)cd.M * cd.N;
  float mi = 0.0f, mp = 0.0f;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < P;
       i += (size_t)gridDim.x * blockDim.x) {
    mi = fmaxf(mi, fabsf(__ldg(&d.uI[i])));
    mp = fmaxf(mp, fabsf(__ldg(&d.up[i])));
  }
  mi = warp_max(mi);
  mp = warp_max(mp);
  if ((threadIdx.x & 31) == 0) {
    atomicMax(&st[gi].absmax[0], __float_as_uint(mi));
    atomicMax(&st[gi].absmax[1], __float_as_uint(mp));
  }
}

cudaError_t launch_plane_absmax(const ClassLaunch& c, cudaStream_t s) {
  const size_t P = (size_t)c.cd.M * c.cd.N;
  int chunks = (int)((P + 256 * 8 - 1) / (256 * 8));
  if (chunks > 128) chunks = 128;
  k_plane_absmax<<<dim3(chunks, c.cd.n_img), 256, 0, s>>>(c.cd, c.imgs, c.st);
  return cudaGetLastError();
}

// One launch per window radius present in the class (the images of a class
// are ordered by radius, so each group is a contiguous range).  Items are
// (image, strip, block of H rows); H is halved (down to 16) while there are
// fewer items than resident warps.
cudaError_t launch_guided_filter(const ClassLaunch& c, int iter, int var_mode, int boundary,
                                 cudaStream_t s) {
  const GfKernel kern = gf_kernel(var_mode, boundary);
  const int shifted = var_mode == GFD_VAR_FP32_RAW ? 0 : 1;
  for (int g = 0; g < c.n_rad_groups; ++g) {
    const RadGroup& rg = c.rad_groups[g];
    ClassDesc cd = c.cd;
    cd.img0 = rg.img0;
    cd.n_img = rg.n_img;
    const size_t smem = (size_t)GFW_WARPS * gfw_ring_floats(rg.rad) * sizeof(float);
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, GFW_WARPS * 32, smem) !=
            cudaSuccess ||
        per_sm < 1)
      per_sm = 1;
    const int div = c.grid_div > 1 ? c.grid_div : 1;
    const int warps = (per_sm * gf_sm_count() + div - 1) / div * GFW_WARPS;
    const int strips = (cd.N + gfw_wout(rg.rad) - 1) / gfw_wout(rg.rad);
    const int hmax = c.gf_rows > 0 ? c.gf_rows : DEF_GF_ROWS;
    int H = cd.M < hmax ? cd.M : hmax;
    while (H > 16 && cd.n_img * strips * (cd.M / H) < warps) H /= 2;
    const int n_items = cd.n_img * strips * (cd.M / H);
    int grid = (per_sm * gf_sm_count() + div - 1) / div;
    const int need = (n_items + GFW_WARPS - 1) / GFW_WARPS;
    if (grid > need) grid = need;
    kern<<<grid, GFW_WARPS * 32, smem, s>>>(cd, c.imgs, c.st, iter, shifted, rg.rad, H);
  }
  return cudaGetLastError();
}

cudaError_t configure_gf_kernel() {
  const int bytes = (int)(GFW_WARPS * gfw_ring_floats(GF_RMAX) * sizeof(float));
  const GfKernel ks[8] = {k_guided_filter<SumIG, false>,  k_guided_filter<SumIG, true>,
                          k_guided_filter<SumDF, false>,  k_guided_filter<SumDF, true>,
                          k_guided_filter<SumF64, false>, k_guided_filter<SumF64, true>,
                          k_guided_filter<SumF32, false>, k_guided_filter<SumF32, true>};
  for (GfKernel k : ks) {
    const cudaError_t e =
        cudaFuncSetAttribute((const void*)k, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

}  // namespace gfd
