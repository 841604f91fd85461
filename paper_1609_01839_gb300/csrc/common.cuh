// Shared device helpers for the guided-filter deconvolution kernels (sm_103a).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/gfdeconv.h"

#define GFD_HD __host__ __device__ __forceinline__
#define GFD_D __device__ __forceinline__

namespace gfd {

// Twiddle table: W_4096^m = exp(-2 pi i m / 4096), m = 0..4095, computed on the
// host in double and rounded once to float.  Any W_L^x with L | 4096 is
// tw[x * (4096 / L)].
constexpr int TW_LOG2 = 12;
constexpr int TW_N = 1 << TW_LOG2;
// Per-size tables: for every L = 2, 4, ..., TW_N the L entries of size L
// (W_L^m = exp(-2 pi i m / L), or 4 sin^2(pi m / L)) start at offset L - 2, so
// a transform of length L touches one compact table of L entries.
constexpr int TAB_ENTRIES = 2 * TW_N - 2;
GFD_HD int tab_off(int L) { return L - 2; }

// Number of interpolation nodes for the regularisation-parameter equation
// (Sec. 3.2, Eq. 11) evaluated per spectral pass.
constexpr int KNODES = 12;
constexpr int KNARROW = 8;  // nodes of the first pass from iteration NARROW_FROM on
constexpr int NARROW_FROM = 5;
// Fallback passes launched after the fused pass of each iteration (default).
constexpr int LAMBDA_FALLBACK_PASSES = 4;
constexpr double LAMBDA_LO = 1e-14;

// status bits (per image)
constexpr int ST_NONCONVERGED = 1;
constexpr int ST_NONFINITE = 2;
constexpr int ST_BAD_PSF = 4;
constexpr int ST_BAD_RHO = 8;
constexpr int ST_PASSES_EXHAUSTED = 16;
constexpr int ST_COPY_TIMEOUT = 32;

GFD_HD float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
GFD_HD float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
GFD_HD float2 cmul(float2 a, float2 b) {
  return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}
GFD_HD float2 cconj(float2 a) { return make_float2(a.x, -a.y); }
GFD_HD float2 cscale(float2 a, float s) { return make_float2(a.x * s, a.y * s); }
// multiply by -i (forward) or +i (inverse)
template <bool INV>
GFD_HD float2 cmul_mi(float2 a) {
  return INV ? make_float2(-a.y, a.x) : make_float2(a.y, -a.x);
}

// Sum over the threads of a warp.  Blocks smaller than a warp (tiny images)
// have blockDim a power of two < 32: the mask and offsets stay inside it.
GFD_D float warp_sum(float v) {
  const unsigned int n = blockDim.x < 32 ? blockDim.x : 32u;
  const unsigned int mask = n == 32 ? 0xffffffffu : ((1u << n) - 1u);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1)
    if ((unsigned)o < n) v += __shfl_xor_sync(mask, v, o);
  return v;
}
// Maximum over the threads of a warp (same partial-warp rule as warp_sum).
GFD_D float warp_max(float v) {
  const unsigned int n = blockDim.x < 32 ? blockDim.x : 32u;
  const unsigned int mask = n == 32 ? 0xffffffffu : ((1u << n) - 1u);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1)
    if ((unsigned)o < n) v = fmaxf(v, __shfl_xor_sync(mask, v, o));
  return v;
}
GFD_D int num_warps() { return (int)((blockDim.x + 31) >> 5); }

// Asynchronous global -> shared copies (16-byte chunks, L2 only) with
// commit groups; waits are hardware waits on the thread's own groups.
GFD_D unsigned int smem_u32(const void* p) { return (unsigned int)__cvta_generic_to_shared(p); }
GFD_D void cp_async16(void* smem_dst, const void* gsrc) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(smem_u32(smem_dst)), "l"(gsrc)
               : "memory");
}
GFD_D void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
GFD_D void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

// One-dimensional bulk copies (the TMA engine) completed on an mbarrier.
// A block stages a contiguous tile with one instruction from one thread:
//   mbar_init once; per tile, the issuing thread calls bulk_load (which arms
//   the barrier with the byte count) and every thread waits with mbar_wait on
//   the barrier's current phase parity, which then flips.
// Addresses are 16-byte aligned and sizes multiples of 16 (the tiles are whole
// column slabs of 256-byte aligned planes).
GFD_D void mbar_init(unsigned long long* bar) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(smem_u32(bar)) : "memory");
  asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
}
GFD_D void bulk_load(void* smem_dst, const void* gsrc, unsigned int bytes, unsigned long long* bar) {
  // earlier generic-proxy reads of the buffer are ordered before the async write
  asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(smem_u32(bar)),
               "r"(bytes)
               : "memory");
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n" ::"r"(
          smem_u32(smem_dst)),
      "l"(gsrc), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}
GFD_D bool mbar_try_wait(unsigned long long* bar, unsigned int parity) {
  unsigned int done;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      " selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(done)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return done != 0;
}
// Wait for the phase of the given parity; false if it has not completed after
// the iteration limit (each try_wait blocks for at most a short, hardware-set
// time), so that a copy that never lands cannot hang the kernel.
constexpr int MBAR_WAIT_LIMIT = 1 << 22;
GFD_D bool mbar_wait(unsigned long long* bar, unsigned int parity) {
  for (int i = 0; i < MBAR_WAIT_LIMIT; ++i)
    if (mbar_try_wait(bar, parity)) return true;
  return false;
}

// Bulk prefetch of [p, p + bytes) into L2 (p 16-byte aligned, bytes a
// multiple of 16), split into pieces of at most 16 KB issued by the lanes of
// warp 0.  No completion to wait for: later loads simply find the lines in L2.
GFD_D void prefetch_l2(const void* p, unsigned int bytes) {
  constexpr unsigned int PIECE = 16384;
  if (threadIdx.x >= 32) return;
  for (unsigned int o = threadIdx.x * PIECE; o < bytes; o += 32 * PIECE) {
    const unsigned int n = bytes - o < PIECE ? bytes - o : PIECE;
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;\n" ::"l"((const char*)p + o), "r"(n)
                 : "memory");
  }
}

// Per-image solver state, one per image of a batch, in device memory.
struct ImgState {
  double T;          // discrepancy target rho * P * sigma^2 (Sec. 3.2)
  double rho;        // rho of Eq. 12 (or the fixed value)
  double sum_y;      // sum of y   (= Y(0,0), kept in FP64)
  double sum_yy;     // sum of y^2
  double sum_h;      // sum of h   (= H(0,0))
  double amax;       // (sum |h|)^2 >= max |H|^2
  double den_isnr;   // ||y - u_orig||^2
  double lam;        // lambda of the current iteration (inf: branch u_E in K)
  double lo, hi;     // bracket of the nodes of the next pass
  double invT;       // 1 / T
  int mode;          // node layout of the next pass: 0 geometric, 1 Chebyshev in lambda
  double lam_up;     // upper bound of the root from res and amax
  double res;        // ||h*u_E - y||^2 of the current iteration
  double sum_u;      // FP64 sum of the current iterate u_E (its DC bin)
  double d00;        // DC residual sum(h) sum(u_E) - sum(y), FP64
  double err2;       // FP64 sum (u - u_orig)^2
  double lam_prev;   // last finite lambda resolved before the current one
  float node[KNODES];// node values lambda_j (float) of the pending pass
  unsigned int cta_done;   // items of the current spectral pass completed
  unsigned int gf_done;    // last-block-done counter (guided filter)
  int need;          // 1: lambda unresolved, a fallback pass must run
  int status;        // ST_* bits
  int iter;          // iteration index of the pending outputs
  int nk;            // nodes of the pending pass (KNODES, or KNARROW for a narrow first pass)
  double rtol;       // relative width of lambda at which the root search stops
  unsigned int absmax[2];  // bits of max |u_I|, max |u_p| of the current iteration
};

// Per-image parameters and pointers, device memory.
struct ImgDesc {
  const float* y;     // M*N
  const float* h;     // kh*kw
  float* u;           // M*N, the iterate (caller's output buffer)
  const float* uo;    // M*N or null
  const float* u0;    // starting u_E, M*N, or null (u_E = 0)
  double* lam_out;    // [iters] or null
  double* isnr_out;   // [iters] or null
  double* res_out;    // [iters] or null
  int kh, kw, w, pad_;
  double sigma, eps, rho_fixed;
  double lam_rtol;    // relative width of lambda at which the root search stops
  // workspace planes (M*N/2 complex each)
  // spectra are packed half spectra in the class's column-tiled layout
  float2* S;          // forward spectrum scratch (row pass output, then U_E)
  float2* QI;         // U_I (Eq. 8)
  float2* Qp;         // U_p (Eq. 9)
  float2* H;          // PSF spectrum
  float2* Y;          // observation spectrum
  float* uI;          // u_I, real M*N (row-major)
  float* up;          // u_p, real M*N (row-major)
  float2* H0;         // H(k, 0),   k < M (unpacked DC column)
  float2* HN;         // H(k, N/2)
  float2* Y0;         // Y(k, 0)
  float2* YN;         // Y(k, N/2)
  double* part;       // per-item partial sums of a spectral pass, (KNODES+1) each
  double* rowsum;     // per-item sums of the iterate from the forward row pass
  float* u_iters;     // [iters][M*N] the iterate entering each iteration, or null
};

// One size class of a batch: all images with the same canvas M x N.
struct ClassDesc {
  int M, N, n_img, img0;   // images img0 .. img0+n_img-1 of the batch
  int TB;                  // tile width of the class's spectra (columns per tile)
};

}  // namespace gfd
