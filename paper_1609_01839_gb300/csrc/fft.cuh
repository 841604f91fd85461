// Power-of-two complex FFT on a team of threads, staged in shared memory.
//
// The transform X[k] = sum_n x[n] W_L^{nk}, W_L = exp(-2 pi i / L) (forward)
// or with W_L^{-nk} (inverse, unnormalised), is computed by the mixed-radix
// decimation-in-frequency recursion L = r_0 * L_1:
//   X[i + r_0 k1] = sum_{n1} W_{L_1}^{n1 k1} [ W_L^{n1 i} sum_{n2} x[n1 + L_1 n2] W_{r_0}^{n2 i} ].
// Stage s holds prod_{s'<s} r_{s'} independent sub-transforms of length L_s,
// stored contiguously; a butterfly (g, j) loads the r_s elements
// g*L_s + j + i*L_{s+1}, applies a radix-r_s DFT in registers and the twiddle
// W_{L_s}^{j i}, and stores them back in place.  After the last stage X[k]
// sits at the digit-reversed position out_pos(k).
//
// A team has L/R threads, each doing R/r_s butterflies per stage; all teams of
// a block run the same L and synchronise with __syncthreads between stages.
// Shared addresses are padded by one element per 16 (phys()) to spread banks.
#pragma once
#include "common.cuh"

namespace gfd {

constexpr int radix_for(int L) { return L >= 256 ? 16 : (L >= 64 ? 8 : (L >= 16 ? 4 : 2)); }

constexpr int stage_radix(int L, int R, int s) {
  int rem = L;
  for (int i = 0; i < s; ++i) {
    int r = rem < R ? rem : R;
    rem /= r;
  }
  return rem < R ? rem : R;
}
constexpr int stage_len(int L, int R, int s) {
  int rem = L;
  for (int i = 0; i < s; ++i) {
    int r = rem < R ? rem : R;
    rem /= r;
  }
  return rem;
}
constexpr int num_stages(int L, int R) {
  int n = 0, rem = L;
  while (rem > 1) {
    int r = rem < R ? rem : R;
    rem /= r;
    ++n;
  }
  return n;
}

GFD_HD int phys(int a) { return a + (a >> 4); }
// elements of one team's buffer (odd, so that teams interleave across banks)
GFD_HD int team_stride(int L) { return L + (L >> 4) + 1; }
// Buffer stride of the B interleaved column teams of a column pass.  Loads
// and stores that walk B columns fastest put B columns x 16/B consecutive
// elements in a half-warp; a stride of 16/B (mod 16) float2 places them on
// distinct bank pairs.
GFD_HD int col_team_stride(int L, int B) { return L + (L >> 4) + (B < 16 ? 16 / B : 1); }

// cos / sin of 2 pi m / 16
__device__ constexpr float kCos16[16] = {
    1.0f, 0.92387953251128674f, 0.70710678118654752f, 0.38268343236508977f,
    0.0f, -0.38268343236508977f, -0.70710678118654752f, -0.92387953251128674f,
    -1.0f, -0.92387953251128674f, -0.70710678118654752f, -0.38268343236508977f,
    0.0f, 0.38268343236508977f, 0.70710678118654752f, 0.92387953251128674f};
__device__ constexpr float kSin16[16] = {
    0.0f, 0.38268343236508977f, 0.70710678118654752f, 0.92387953251128674f,
    1.0f, 0.92387953251128674f, 0.70710678118654752f, 0.38268343236508977f,
    0.0f, -0.38268343236508977f, -0.70710678118654752f, -0.92387953251128674f,
    -1.0f, -0.92387953251128674f, -0.70710678118654752f, -0.38268343236508977f};

// The rounding residuals of kCos16 / kSin16 (value minus its float), so that
// hi + lo carries cos and sin to about 48 bits.  With the floats alone every
// non-trivial constant twiddle has |w| < 1 (all six round towards zero), and
// a transform shrinks every output by ~7e-8 of its magnitude: a bias, not a
// random error, which sums of squares of spectra (the residual of Eq. 10-11)
// inherit in full.
constexpr float kC1 = 2.830748968563057e-08f;   // cos(pi/8) residual
constexpr float kS1 = 6.2233507236442165e-09f;  // sin(pi/8) residual
constexpr float kC2 = 1.2101617485882343e-08f;  // cos(pi/4) residual
__device__ constexpr float kCos16Lo[16] = {0.0f, kC1,  kC2,  kS1,  0.0f, -kS1, -kC2, -kC1,
                                           0.0f, -kC1, -kC2, -kS1, 0.0f, kS1,  kC2,  kC1};
__device__ constexpr float kSin16Lo[16] = {0.0f, kS1,  kC2,  kC1,  0.0f, kC1,  kC2,  kS1,
                                           0.0f, -kS1, -kC2, -kC1, 0.0f, -kC1, -kC2, -kS1};

// v * W_R^k (forward: exp(-2 pi i k/R); inverse: exp(+2 pi i k/R)), R <= 16.
// The product uses the constants' residuals (two more FMAs per component), so
// it is the exact product up to roundings of either sign.
template <int R, int k, bool INV>
GFD_D float2 const_twiddle(float2 v) {
  if constexpr (k == 0) {
    return v;
  } else if constexpr (4 * k == R) {
    return cmul_mi<INV>(v);
  } else {
    constexpr int m = k * (16 / R);
    const float c = kCos16[m], cl = kCos16Lo[m];
    const float s = INV ? kSin16[m] : -kSin16[m];
    const float sl = INV ? kSin16Lo[m] : -kSin16Lo[m];
    return make_float2(fmaf(v.x, c, fmaf(-v.y, s, fmaf(v.x, cl, -v.y * sl))),
                       fmaf(v.x, s, fmaf(v.y, c, fmaf(v.x, sl, v.y * cl))));
  }
}

// In-register DFT of length R (natural-order input and output).
template <int R, bool INV>
struct DFT {
  template <int k>
  GFD_D static void combine(float2* x, const float2* e, const float2* o) {
    if constexpr (k < R / 2) {
      const float2 t = const_twiddle<R, k, INV>(o[k]);
      x[k] = cadd(e[k], t);
      x[k + R / 2] = csub(e[k], t);
      combine<k + 1>(x, e, o);
    }
  }
  GFD_D static void run(float2* x) {
    float2 e[R / 2], o[R / 2];
#pragma unroll
    for (int i = 0; i < R / 2; ++i) {
      e[i] = x[2 * i];
      o[i] = x[2 * i + 1];
    }
    DFT<R / 2, INV>::run(e);
    DFT<R / 2, INV>::run(o);
    combine<0>(x, e, o);
  }
};
template <bool INV>
struct DFT<1, INV> {
  GFD_D static void run(float2*) {}
};
template <bool INV>
struct DFT<2, INV> {
  GFD_D static void run(float2* x) {
    const float2 a = x[0], b = x[1];
    x[0] = cadd(a, b);
    x[1] = csub(a, b);
  }
};

// tw: the table of the transform length L (W_L^m, m < L)
// (a generic load: the table may sit in shared or global memory)
GFD_D float2 twiddle(const float2* __restrict__ tw, int m, bool inv) {
  float2 w = tw[m];
  if (inv) w.y = -w.y;
  return w;
}

// Shared-memory address of element a of a team's sequence.
struct PaddedIdx {  // contiguous with one pad element per 16
  GFD_D int operator()(int a) const { return phys(a); }
};
struct IdentIdx {  // contiguous, unpadded (landing buffers of rows)
  GFD_D int operator()(int a) const { return a; }
};
struct StridedIdx {  // element a of column b of an interleaved [a][B] tile
  int stride;
  GFD_D int operator()(int a) const { return a * stride; }
};

template <int L, int R, bool INV, int s>
struct Stage {
  template <class Idx>
  GFD_D static void run(float2* buf, int j, const float2* __restrict__ tw, Idx idx) {
    constexpr int Ls = stage_len(L, R, s);
    if constexpr (Ls > 1) {
      constexpr int r = Ls < R ? Ls : R;
      constexpr int Ln = Ls / r;
      constexpr int T = L / R;
      constexpr int twstep = L / Ls;  // W_Ls = W_L^(L / Ls)
#pragma unroll
      for (int q = 0; q < R / r; ++q) {
        const int beta = j + T * q;
        const int g = beta / Ln;
        const int jj = beta % Ln;
        const int base = g * Ls + jj;
        float2 x[r];
#pragma unroll
        for (int i = 0; i < r; ++i) x[i] = buf[idx(base + i * Ln)];
        DFT<r, INV>::run(x);
        if constexpr (Ln > 1) {
#pragma unroll
          for (int i = 1; i < r; ++i) x[i] = cmul(x[i], twiddle(tw, jj * i * twstep, INV));
        }
#pragma unroll
        for (int i = 0; i < r; ++i) buf[idx(base + i * Ln)] = x[i];
      }
      __syncthreads();
      Stage<L, R, INV, s + 1>::run(buf, j, tw, idx);
    }
  }
};

// Two transforms of the same length on one team (buffers A and B), stage by
// stage: each butterfly's twiddles are loaded once and applied to both.
template <int L, int R, bool INV, int s>
struct Stage2 {
  template <class Idx>
  GFD_D static void run(float2* bufA, float2* bufB, int j, const float2* __restrict__ tw, Idx idx) {
    constexpr int Ls = stage_len(L, R, s);
    if constexpr (Ls > 1) {
      constexpr int r = Ls < R ? Ls : R;
      constexpr int Ln = Ls / r;
      constexpr int T = L / R;
      constexpr int twstep = L / Ls;
#pragma unroll
      for (int q = 0; q < R / r; ++q) {
        const int beta = j + T * q;
        const int g = beta / Ln;
        const int jj = beta % Ln;
        const int base = g * Ls + jj;
        float2 w[r];
        if constexpr (Ln > 1) {
#pragma unroll
          for (int i = 1; i < r; ++i) w[i] = twiddle(tw, jj * i * twstep, INV);
        }
#pragma unroll 1
        for (int h = 0; h < 2; ++h) {
          float2* buf = h ? bufB : bufA;
          float2 x[r];
#pragma unroll
          for (int i = 0; i < r; ++i) x[i] = buf[idx(base + i * Ln)];
          DFT<r, INV>::run(x);
          if constexpr (Ln > 1) {
#pragma unroll
            for (int i = 1; i < r; ++i) x[i] = cmul(x[i], w[i]);
          }
#pragma unroll
          for (int i = 0; i < r; ++i) buf[idx(base + i * Ln)] = x[i];
        }
      }
      __syncthreads();
      Stage2<L, R, INV, s + 1>::run(bufA, bufB, j, tw, idx);
    }
  }
};

// First stage reading from a separate (landing) buffer `in` addressed by
// iidx, writing to buf addressed by idx; the remaining stages run in buf.
template <int L, int R, bool INV>
struct Stage0From {
  template <class InIdx, class Idx>
  GFD_D static void run(const float2* in, InIdx iidx, float2* buf, int j,
                        const float2* __restrict__ tw, Idx idx) {
    constexpr int Ls = L;
    constexpr int r = Ls < R ? Ls : R;
    constexpr int Ln = Ls / r;
    constexpr int T = L / R;
    constexpr int twstep = L / Ls;
#pragma unroll
    for (int q = 0; q < R / r; ++q) {
      const int beta = j + T * q;
      const int g = beta / Ln;
      const int jj = beta % Ln;
      const int base = g * Ls + jj;
      float2 x[r];
#pragma unroll
      for (int i = 0; i < r; ++i) x[i] = in[iidx(base + i * Ln)];
      DFT<r, INV>::run(x);
      if constexpr (Ln > 1) {
#pragma unroll
        for (int i = 1; i < r; ++i) x[i] = cmul(x[i], twiddle(tw, jj * i * twstep, INV));
      }
#pragma unroll
      for (int i = 0; i < r; ++i) buf[idx(base + i * Ln)] = x[i];
    }
  }
};

// Transform whose input sits in `in` (read once, by the first stage) and
// whose stages and output live in buf.  Ends block-synchronised, after which
// `in` may be overwritten.
template <int L, bool INV, class InIdx, class Idx = PaddedIdx>
GFD_D void fft_team_from(const float2* in, InIdx iidx, float2* buf, int j,
                         const float2* __restrict__ tw, Idx idx = Idx()) {
  constexpr int R = radix_for(L);
  Stage0From<L, R, INV>::run(in, iidx, buf, j, tw, idx);
  __syncthreads();
  Stage<L, R, INV, 1>::run(buf, j, tw, idx);
}

// Run the whole transform of one team (thread j of L/R) in place on buf.
// Precondition: buf filled and a __syncthreads() issued by the caller.
// Postcondition: X[k] at buf[idx(out_pos<L>(k))], block synchronised.
template <int L, bool INV, class Idx = PaddedIdx>
GFD_D void fft_team(float2* buf, int j, const float2* __restrict__ tw, Idx idx = Idx()) {
  Stage<L, radix_for(L), INV, 0>::run(buf, j, tw, idx);
}

// fft_team on two buffers of the same team at once (shared twiddles).
template <int L, bool INV, class Idx = PaddedIdx>
GFD_D void fft_team2(float2* bufA, float2* bufB, int j, const float2* __restrict__ tw,
                     Idx idx = Idx()) {
  Stage2<L, radix_for(L), INV, 0>::run(bufA, bufB, j, tw, idx);
}

// position of output k after the in-place stages (digit reversal)
template <int L>
GFD_D int out_pos(int k) {
  constexpr int R = radix_for(L);
  constexpr int S = num_stages(L, R);
  int p = 0, rem = k;
#pragma unroll
  for (int s = 0; s < S; ++s) {
    const int r = stage_radix(L, R, s);
    const int Ln = stage_len(L, R, s) / r;
    p += (rem % r) * Ln;
    rem /= r;
  }
  return p;
}

// inverse of out_pos: the output index stored at position p
template <int L>
GFD_D int in_pos(int p) {
  constexpr int R = radix_for(L);
  constexpr int S = num_stages(L, R);
  int k = 0, mul = 1, rem = p;
#pragma unroll
  for (int s = 0; s < S; ++s) {
    const int r = stage_radix(L, R, s);
    const int Ln = stage_len(L, R, s) / r;
    k += (rem / Ln) * mul;
    rem %= Ln;
    mul *= r;
  }
  return k;
}

}  // namespace gfd
