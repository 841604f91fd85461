// 2-D real DFT passes and the spectral steps of the deblurring solve.
//
// Packed half spectrum (M rows x N/2 complex): S(m, l) = X(m, l) for
// 1 <= l < N/2 and S(m, 0) = X(m, 0) + i X(m, N/2), X the full 2-D DFT.  A
// row pass maps each real row to its packed row DFT; a column pass is a plain
// complex FFT down every packed column (column 0 included, since its two real
// row spectra pack into one complex signal).  Bins (m, 0) and (m, N/2) are
// unpacked where a spectral formula needs them.
//
// Spectra are stored column-tiled: S(m, l) at (l / TB) * M * TB + m * TB +
// l % TB, TB the class's tile width.  A column item (TB columns, all M rows)
// is then one contiguous block of memory, and a row item (rpc rows) writes a
// contiguous run of rpc * TB values per tile.  TB = N/2 is plain row-major.
#include "fft.cuh"
#include "lambda.cuh"
#include "spectral.cuh"
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
    case SEL_UI: return d.uI;
    case SEL_UP: return d.up;
    default: return reinterpret_cast<float*>(d.Y);
  }
}
GFD_D float2* cplx_plane(const ImgDesc& d, int sel) {
  return reinterpret_cast<float2*>(real_plane(d, sel));
}

constexpr int threads_per_team(int L) { return L / radix_for(L); }
// Largest column length whose twiddle table the column passes keep in
// shared memory (8 KB at 1024).
constexpr int SMEM_TW_MAX = 1024;

// Persistent pass kernels.  Each block walks the work items item =
// blockIdx.x + k * gridDim.x; the inputs of the next item are copied
// asynchronously into a landing buffer while the current item's transform
// runs in a separate (padded) work buffer, so that global loads stay in
// flight while the block computes.

// ---------------------------------------------------------------------------
// Row pass, forward: real rows -> packed row spectra (tiled).  An item is
// rpc consecutive rows of one image.  Each row of N reals is read as N/2
// complex z[n] = x[2n] + i x[2n+1]; Z = FFT_{N/2}(z); then
// X[k] = (Z[k] + conj Z[-k])/2 + W_N^k (Z[k] - conj Z[-k])/(2i), and
// X[0], X[N/2] = Re Z[0] +- Im Z[0] (packed as X[0] + i X[N/2]).
// ---------------------------------------------------------------------------
// float2 elements of the row-pass work area of rpc teams, rounded up to even.
GFD_HD int row_work_elems(int L, int rpc) { return (rpc * team_stride(L) + 1) & ~1; }

template <int L>
__global__ void __launch_bounds__(256, 2)
k_row_r2c(ClassDesc cd, const ImgDesc* __restrict__ imgs, const float2* __restrict__ tw, int rpc,
          int src_sel, int dst_sel, int do_sum) {
  extern __shared__ __align__(16) float2 smem[];
  constexpr int R = radix_for(L), T = threads_per_team(L);
  constexpr int N = 2 * L;
  const int TB = cd.TB, M = cd.M;
  const int item_elems = rpc * L;
  float2* land = smem;
  float2* work = land + item_elems;
  // team_stride(L) is odd: round the work area up to an even number of float2
  // so that the output rows (read as 16-byte vectors) start 16-byte aligned
  float2* outb = work + row_work_elems(L, rpc);
  double* red = reinterpret_cast<double*>(outb + item_elems);
  // length-L twiddle table in shared memory (L <= SMEM_TW_MAX)
  const float2* twL = tw + tab_off(L);
  if constexpr (L <= SMEM_TW_MAX) {
    float2* stw = reinterpret_cast<float2*>(red + 32);
    for (int i = threadIdx.x; i < L; i += blockDim.x) stw[i] = twL[i];
    twL = stw;  // visible after the loop's first __syncthreads()
  }
  const int team = threadIdx.x / T, j = threadIdx.x % T;
  const int n_items = cd.n_img * M / rpc;
  auto issue = [&](int item) {
    if (item < n_items) {
      const int row_c = item * rpc;
      const ImgDesc& d = imgs[cd.img0 + row_c / M];
      const float2* src =
          reinterpret_cast<const float2*>(real_plane(d, src_sel)) + (size_t)(row_c % M) * L;
      for (int c = threadIdx.x; c < item_elems / 2; c += blockDim.x)
        cp_async16(land + 2 * c, src + 2 * c);
    }
    cp_async_commit();
  };
  issue(blockIdx.x);
  for (int item = blockIdx.x; item < n_items; item += gridDim.x) {
    cp_async_wait<0>();
    __syncthreads();
    const int row0 = (item * rpc) % M;
    const ImgDesc& d = imgs[cd.img0 + (item * rpc) / M];
    float2* buf = work + team * team_stride(L);
    const float2* in = land + team * L;
    if (do_sum) {
      float part = 0.0f;
#pragma unroll
      for (int i = 0; i < R; ++i) {
        const float2 v = in[j + i * T];
        part += v.x + v.y;
      }
      part = warp_sum(part);
      if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = (double)part;
    }
    fft_team_from<L, false>(in, IdentIdx(), buf, j, twL);  // first stage reads land
    issue(item + gridDim.x);                               // land is free again
    if (do_sum && threadIdx.x == 0) {
      double s = 0.0;
      for (int w = 0; w < num_warps(); ++w) s += red[w];
      d.rowsum[row0 / rpc] = s;  // one partial per item, summed by the column pass
    }
    float2* ob = outb + team * L;
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
        out = cadd(E, cmul(__ldg(&tw[tab_off(N) + k]), O));
      }
      ob[k] = out;
    }
    __syncthreads();
    // copy out tile by tile: rows row0 .. row0+rpc-1 of tile t are contiguous
    float2* dst = cplx_plane(d, dst_sel);
    // 16-byte chunks: rpc * TB / 2 per tile, TB / 2 per row (powers of two)
    const int lg_pt = __ffs(rpc * TB / 2) - 1, lg_hr = __ffs(TB / 2) - 1;
    for (int c = threadIdx.x; c < item_elems / 2; c += blockDim.x) {
      const int t = c >> lg_pt, w = c & ((1 << lg_pt) - 1);
      const int r = w >> lg_hr, q = w & ((1 << lg_hr) - 1);
      const float4 v = *reinterpret_cast<const float4*>(outb + r * L + t * TB + 2 * q);
      *reinterpret_cast<float4*>(dst + (size_t)t * M * TB + (size_t)(row0 + r) * TB + 2 * q) = v;
    }
  }
  cp_async_wait<0>();
}

// ---------------------------------------------------------------------------
// Row pass, inverse: packed row spectra (tiled) -> real rows (scaled).
// Z[k] = (R[k] + conj R[L-k]) + i (R[k] - conj R[L-k]) W_N^{-k}, with
// R[0], R[N/2] the real and imaginary parts of the packed entry 0; the
// unnormalised inverse FFT of Z gives x[2n] + i x[2n+1] times N.
// Items cover spectrum sel0 -> real plane dsel0, then sel1 -> dsel1.
// ---------------------------------------------------------------------------
template <int L>
__global__ void __launch_bounds__(256, 3)
k_row_c2r(ClassDesc cd, const ImgDesc* __restrict__ imgs, const float2* __restrict__ tw, int rpc,
          int sel0, int sel1, int dsel0, int dsel1, float scale, ImgState* st) {
  extern __shared__ __align__(16) float2 smem[];
  constexpr int R = radix_for(L), T = threads_per_team(L);
  constexpr int N = 2 * L;
  const int TB = cd.TB, M = cd.M;
  const int item_elems = rpc * L;
  float2* land = smem;
  float2* work = smem + item_elems;
  const float2* twL = tw + tab_off(L);
  if constexpr (L <= SMEM_TW_MAX) {
    float2* stw = work + rpc * team_stride(L);
    for (int i = threadIdx.x; i < L; i += blockDim.x) stw[i] = twL[i];
    twL = stw;  // visible after the loop's first __syncthreads()
  }
  const int team = threadIdx.x / T, j = threadIdx.x % T;
  const int per_plane = cd.n_img * M / rpc;
  const int n_items = sel1 >= 0 ? 2 * per_plane : per_plane;
  // 16-byte chunks: rpc * TB / 2 per tile, TB / 2 per row (powers of two)
  const int lg_pt = __ffs(rpc * TB / 2) - 1, lg_hr = __ffs(TB / 2) - 1;
  auto issue = [&](int item) {
    if (item < n_items) {
      int sel = sel0;
      if (item >= per_plane) {
        item -= per_plane;
        sel = sel1;
      }
      const int row_c = item * rpc;
      const ImgDesc& d = imgs[cd.img0 + row_c / M];
      const float2* src = cplx_plane(d, sel) + (size_t)(row_c % M) * TB;
      for (int c = threadIdx.x; c < item_elems / 2; c += blockDim.x) {
        const int t = c >> lg_pt, w = c & ((1 << lg_pt) - 1);
        const int r = w >> lg_hr, q = w & ((1 << lg_hr) - 1);
        cp_async16(land + r * L + t * TB + 2 * q, src + (size_t)t * M * TB + r * TB + 2 * q);
      }
    }
    cp_async_commit();
  };
  issue(blockIdx.x);
  for (int item = blockIdx.x; item < n_items; item += gridDim.x) {
    cp_async_wait<0>();
    __syncthreads();
    int it = item, dsel = dsel0;
    if (it >= per_plane) {
      it -= per_plane;
      dsel = dsel1;
    }
    const int row_c = it * rpc + team;
    const int li = row_c / M, row = row_c % M;
    const ImgDesc& d = imgs[cd.img0 + li];
    float2* buf = work + team * team_stride(L);
    const float2* in = land + team * L;
    for (int k = j; k <= L / 2; k += T) {
      if (k == 0) {
        const float2 t0 = in[0];
        buf[phys(0)] = make_float2(t0.x + t0.y, t0.x - t0.y);
      } else {
        const int km = L - k;
        const float2 Rk = in[k], Rm = in[km];
        {
          const float2 E = cadd(Rk, cconj(Rm));
          const float2 O = cmul(csub(Rk, cconj(Rm)), cconj(__ldg(&tw[tab_off(N) + k])));
          buf[phys(k)] = make_float2(E.x - O.y, E.y + O.x);
        }
        if (km != k) {
          const float2 E = cadd(Rm, cconj(Rk));
          const float2 O = cmul(csub(Rm, cconj(Rk)), cconj(__ldg(&tw[tab_off(N) + km])));
          buf[phys(km)] = make_float2(E.x - O.y, E.y + O.x);
        }
      }
    }
    __syncthreads();
    issue(item + gridDim.x);
    fft_team<L, true>(buf, j, twL);
    float2* rowp = reinterpret_cast<float2*>(real_plane(d, dsel)) + (size_t)row * L;
    float amax = 0.0f;
#pragma unroll
    for (int i = 0; i < R; ++i) {
      const int n = j + i * T;
      const float2 v = cscale(buf[phys(out_pos<L>(n))], scale);
      rowp[n] = v;
      amax = fmaxf(amax, fmaxf(fabsf(v.x), fabsf(v.y)));
    }
    // largest |value| of the plane (u_I, u_p): bounds the guided filter's
    // split window sums; non-negative floats order like their bit patterns
    if (st) {
      amax = warp_max(amax);  // the teams of a warp share one image and plane
      if ((threadIdx.x & 31) == 0)
        atomicMax(&st[cd.img0 + li].absmax[dsel == dsel0 ? 0 : 1], __float_as_uint(amax));
    }
  }
  cp_async_wait<0>();
}

// ---------------------------------------------------------------------------
// Column passes.  An item is B adjacent packed columns of one image (B = TB
// in the iteration kernels: one contiguous tile).  It lands as an [M][B]
// tile and team b (threads b, b+B, ...) transforms column c0+b.
// ---------------------------------------------------------------------------

// Setup / utility column FFT (not pipelined): plane src -> dst, in place
// allowed; B columns (inside one tile) per block.  Loads and stores walk the
// B columns fastest (coalesced rows of the tile); the in-place stages walk a
// column's team fastest (conflict-free with the phys() padding); results are
// read in storage (digit-reversed) order so that shared reads stay
// conflict-free, and scattered to their rows.
template <int M, bool INV>
__global__ void k_col_plain(ClassDesc cd, const ImgDesc* __restrict__ imgs,
                            const float2* __restrict__ tw, int B, int src_sel, int dst_sel) {
  extern __shared__ float2 smem[];
  constexpr int R = radix_for(M), T = threads_per_team(M);
  const int Lc = cd.N / 2, TB = cd.TB;
  const int cpi = Lc / B;
  const ImgDesc& d = imgs[cd.img0 + blockIdx.x / cpi];
  const int c0 = (blockIdx.x % cpi) * B;
  const int ts = col_team_stride(M, B);
  const int bs = threadIdx.x % B, js = threadIdx.x / B;
  const int bf = T >= 16 ? threadIdx.x / T : bs, jf = T >= 16 ? threadIdx.x % T : js;
  const size_t off = (size_t)(c0 / TB) * M * TB + (c0 % TB) + bs;
  float2* bufs = smem + bs * ts;
  const float2* src = cplx_plane(d, src_sel) + off;
  float2* dst = cplx_plane(d, dst_sel) + off;
#pragma unroll
  for (int i = 0; i < R; ++i) {
    const int a = js + i * T;
    bufs[phys(a)] = src[(size_t)a * TB];
  }
  __syncthreads();
  fft_team<M, INV>(smem + bf * ts, jf, tw + tab_off(M));
#pragma unroll
  for (int i = 0; i < R; ++i) {
    const int p = js + i * T;
    dst[(size_t)in_pos<M>(p) * TB] = bufs[phys(p)];
  }
}

// Forward column FFT of the iterate's row spectra (in place on S), fused with
// the first evaluation of Eq. 11 at the nodes of the image's bracket.  Only
// the S tile lands in shared memory; it is consumed by the first FFT stage,
// after which the next item's tile is requested, so the copy overlaps the
// remaining stages and the Eq. 11 sums (H and Y are read from global memory
// in that loop).  A block takes a contiguous range of items and keeps its
// per-node sums in registers while consecutive items belong to the same
// image; it publishes them (one partial slot, one counter update) only when
// the image changes.  NK: the nodes of the pass (KNODES, or KNARROW for the
// narrow brackets of iterations NARROW_FROM on).
template <int M, int NK>
__global__ void __launch_bounds__(M >= 4096 ? 512 : 256, M >= 4096 ? 1 : 2)
k_col_fwd_lambda(ClassDesc cd, const ImgDesc* __restrict__ imgs, ImgState* st,
                 const float2* __restrict__ tw, int iter, int row_items) {
  extern __shared__ __align__(16) float2 smem[];
  constexpr int R = radix_for(M), T = threads_per_team(M);
  __shared__ float s_nodes[KNODES];
  __shared__ double s_tot[KNODES + 1];
  __shared__ int s_flag;
  __shared__ WarpAcc s_wacc;
  __shared__ __align__(8) unsigned long long s_bar;  // completion of the landing tile
  const int B = cd.TB;
  const int Lc = cd.N / 2;
  const int cpi = Lc / B;
  const int n_items = cd.n_img * cpi;
  const int per_cta = (n_items + gridDim.x - 1) / gridDim.x;
  const int first = blockIdx.x * per_cta;
  const int stop = min(first + per_cta, n_items);
  const int tile = M * B;
  const int ts = col_team_stride(M, B);
  float2* landS = smem;
  float2* work = landS + tile;
  double* red = reinterpret_cast<double*>(work + B * ts);
  // the length-M twiddle table, copied once per (persistent) block for
  // M <= SMEM_TW_MAX; larger tables stay in global memory
  const float2* twM = tw + tab_off(M);
  if constexpr (M <= SMEM_TW_MAX) {
    float2* stw = reinterpret_cast<float2*>(red + num_warps() * (KNODES + 1));
    for (int i = threadIdx.x; i < M; i += blockDim.x) stw[i] = twM[i];
    twM = stw;  // visible after the loop's first __syncthreads()
  }
  // b-fastest mapping for tile I/O, team-fastest for the in-place stages
  const int b = threadIdx.x % B, j = threadIdx.x / B;
  const int bf = T >= 16 ? threadIdx.x / T : b, jf = T >= 16 ? threadIdx.x % T : j;
  // the item's S tile is one contiguous slab: one bulk copy by thread 0,
  // completed on s_bar; H and Y of the item are read after its transform,
  // so they are only prefetched into L2
  if (threadIdx.x == 0) mbar_init(&s_bar);
  __syncthreads();
  unsigned int parity = 0;
  auto issue = [&](int item) {
    if (item < stop) {
      const ImgDesc& d = imgs[cd.img0 + item / cpi];
      const size_t off = (size_t)(item % cpi) * tile;
      if (threadIdx.x == 0) bulk_load(landS, d.S + off, (unsigned int)(tile * sizeof(float2)), &s_bar);
      prefetch_l2(d.H + off, (unsigned int)(tile * sizeof(float2)));
      prefetch_l2(d.Y + off, (unsigned int)(tile * sizeof(float2)));
    }
  };
  float acc[KNODES + 1];
#pragma unroll
  for (int q = 0; q <= KNODES; ++q) acc[q] = 0.0f;
  int cur = -1, slot = 0, count = 0;
  // publish the sums of `count` items of image `cur` (slot = its first tile);
  // the block completing the image's count reduces all slots and updates
  // the image's lambda
  auto flush = [&]() {
    ImgState* S = st + cur;
    const ImgDesc& d = imgs[cur];
    block_partials_folded(&s_wacc, d.part + (size_t)slot * (KNODES + 1));
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) {
      const unsigned int prev = atomicAdd(&S->cta_done, (unsigned int)count);
      s_flag = (prev + count == (unsigned int)cpi);
    }
    __syncthreads();
    if (s_flag) {
      __threadfence();
      block_sum_columns(d.part, cpi, KNODES + 1, KNODES + 1, red, s_tot);
      for (int q = threadIdx.x; q < cpi * (KNODES + 1); q += blockDim.x) d.part[q] = 0.0;
      if (threadIdx.x < 32)
        lambda_update_warp(S, s_tot, (double)cd.M * cd.N, true, false, iter, d.lam_out, d.res_out,
                           threadIdx.x);
      if (threadIdx.x == 0) {
        S->cta_done = 0;
        __threadfence();
      }
    }
    count = 0;
  };
  warp_acc_clear(&s_wacc);  // first use follows the loop's __syncthreads()
  issue(first);
  for (int item = first; item < stop; ++item) {
    const int gi = cd.img0 + item / cpi;
    const int t = item % cpi;
    if (!mbar_wait(&s_bar, parity)) atomicOr(&st[gi].status, ST_COPY_TIMEOUT);
    parity ^= 1;
    __syncthreads();
    if (gi != cur) {
      if (count > 0) flush();
      cur = gi;
      slot = t;
      for (int q = threadIdx.x; q < KNODES; q += blockDim.x) s_nodes[q] = __ldcg(&st[gi].node[q]);
    }
    const ImgDesc& d = imgs[gi];
    ImgState* S = st + gi;
    const int col = t * B + b;
    const size_t off = (size_t)t * tile;
    if (t == 0) {  // the DC bin needs sum(u_E): total of the row pass's partials
      block_sum_columns(d.rowsum, row_items, 1, 1, red, s_tot);
      if (threadIdx.x == 0) S->sum_u = s_tot[0];
    }
    float2* buf = work + b * ts;
    Stage0From<M, R, false>::run(landS + b, StridedIdx{B}, buf, j, twM, PaddedIdx());
    __syncthreads();  // the landing tile is consumed
    issue(item + 1);
    Stage<M, R, false, 1>::run(work + bf * ts, jf, twM, PaddedIdx());  // ends synchronised
    float nodes[KNODES];
#pragma unroll
    for (int q = 0; q < KNODES; ++q) nodes[q] = s_nodes[q];
    float2* spec = d.S + off + b;
    const float2* Hc = d.H + off + b;
    const float2* Yc = d.Y + off + b;
    if (col != 0) {
      // positions p in storage order; p holds output row k = in_pos(p)
#pragma unroll 4
      for (int i = 0; i < R; ++i) {
        const int p = j + i * T;
        const int k = in_pos<M>(p);
        const float2 Hk = __ldg(&Hc[(size_t)k * B]);
        const float2 Yk = __ldg(&Yc[(size_t)k * B]);
        const float2 U = buf[phys(p)];
        spec[(size_t)k * B] = U;
        const float2 r = csub(cmul(Hk, U), Yk);
        const float rr = fmaf(r.x, r.x, r.y * r.y);
        const float a = fmaf(Hk.x, Hk.x, Hk.y * Hk.y);
        accum_bin<NK>(2.0f * rr, a, nodes, acc);  // bins l and N-l
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
          const double su = s_tot[0];
          const double d00 = S->sum_h * su - S->sum_y;
          S->d00 = d00;
          rA = (float)(d00 * d00);
          U.x = (float)su;
        } else {
          const float2 r = csub(cmul(HA, UA), YA);
          rA = fmaf(r.x, r.x, r.y * r.y);
        }
        const float2 rb = csub(cmul(HB, UB), YB);
        accum_bin<NK>(rA, fmaf(HA.x, HA.x, HA.y * HA.y), nodes, acc);
        accum_bin<NK>(fmaf(rb.x, rb.x, rb.y * rb.y), fmaf(HB.x, HB.x, HB.y * HB.y), nodes, acc);
        spec[(size_t)k * B] = U;
      }
    }
    warp_fold(acc, &s_wacc);
    ++count;
  }
  if (count > 0) flush();
}

// Fallback evaluation of Eq. 11 over the stored spectrum U_E for images whose
// root is still open; a block covers `chunk` elements (in tiled order) of one
// image.
__global__ void __launch_bounds__(256)
k_lambda_pass(ClassDesc cd, const ImgDesc* __restrict__ imgs, ImgState* st, int chunk, int iter,
              int last_chance) {
  __shared__ float s_nodes[KNODES];
  __shared__ double red[32 * (KNODES + 1)];
  __shared__ double s_tot[KNODES + 1];
  __shared__ int s_flag;
  __shared__ WarpAcc s_wacc;
  const int Lc = cd.N / 2, TB = cd.TB, M = cd.M;
  const int per_img = M * Lc;
  const int cpi = per_img / chunk;
  const int gi = cd.img0 + blockIdx.x / cpi;
  ImgState* S = st + gi;
  if (__ldcg(&S->need) == 0) return;
  const ImgDesc& d = imgs[gi];
  for (int q = threadIdx.x; q < KNODES; q += blockDim.x) s_nodes[q] = __ldcg(&S->node[q]);
  warp_acc_clear(&s_wacc);
  __syncthreads();
  float nodes[KNODES];
#pragma unroll
  for (int q = 0; q < KNODES; ++q) nodes[q] = s_nodes[q];
  float acc[KNODES + 1];
#pragma unroll
  for (int q = 0; q <= KNODES; ++q) acc[q] = 0.0f;
  const int e0 = (blockIdx.x % cpi) * chunk;
  const int lg_tile = __ffs(M * TB) - 1, lg_tb = __ffs(TB) - 1;  // powers of two
  // bins in pairs (b, b+1) of one tile row, read as 16-byte vectors; runs of
  // 8 pairs per thread between folds (uniform control flow)
  const float4* S4 = reinterpret_cast<const float4*>(d.S);
  const float4* H4 = reinterpret_cast<const float4*>(d.H);
  const float4* Y4 = reinterpret_cast<const float4*>(d.Y);
  const int pairs = chunk / 2, p0 = e0 / 2;
  for (int base = 0; base < pairs; base += 8 * blockDim.x) {
#pragma unroll 4
    for (int q = 0; q < 8; ++q) {
      const int pi = base + q * blockDim.x + threadIdx.x;
      if (pi < pairs) {
        const int e = 2 * (p0 + pi);
        const int t = e >> lg_tile, rem = e & ((1 << lg_tile) - 1);
        const int k = rem >> lg_tb, b = rem & (TB - 1);  // b even
        const float4 U2 = __ldcs(&S4[p0 + pi]);
        const float4 H2 = __ldg(&H4[p0 + pi]), Y2 = __ldg(&Y4[p0 + pi]);
        {  // bin b + 1 (never column 0)
          const float2 H = make_float2(H2.z, H2.w);
          const float2 r = csub(cmul(H, make_float2(U2.z, U2.w)), make_float2(Y2.z, Y2.w));
          accum_bin(2.0f * fmaf(r.x, r.x, r.y * r.y), fmaf(H.x, H.x, H.y * H.y), nodes, acc);
        }
        if (t != 0 || b != 0) {
          const float2 H = make_float2(H2.x, H2.y);
          const float2 r = csub(cmul(H, make_float2(U2.x, U2.y)), make_float2(Y2.x, Y2.y));
          accum_bin(2.0f * fmaf(r.x, r.x, r.y * r.y), fmaf(H.x, H.x, H.y * H.y), nodes, acc);
        } else {  // packed column 0: bins (k, 0) and (k, N/2)
          const float2 U = make_float2(U2.x, U2.y);
          const float2 Um = d.S[(size_t)((M - k) & (M - 1)) * TB];
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
    }
    warp_fold(acc, &s_wacc);
  }
  block_partials_folded(&s_wacc, d.part + (size_t)(blockIdx.x % cpi) * (KNODES + 1));
  if (last_item(&S->cta_done, cpi, &s_flag)) {
    block_sum_columns(d.part, cpi, KNODES + 1, KNODES + 1, red, s_tot);
    for (int q = threadIdx.x; q < cpi * (KNODES + 1); q += blockDim.x) d.part[q] = 0.0;
    if (threadIdx.x < 32)
      lambda_update_warp(S, s_tot, (double)cd.M * cd.N, false, last_chance != 0, iter,
                         d.lam_out, d.res_out, threadIdx.x);
    if (threadIdx.x == 0) {
      S->cta_done = 0;
      __threadfence();
    }
  }
}


// Spectral solves fused with the inverse column FFTs: an item's U_E tile
// lands in shared memory (H and Y are read from global memory next to it);
// Eq. 8 and 9 fill two work tiles (U_I, U_p) that are inverse-transformed
// while the next item's tile is fetched.
template <int M>
__global__ void __launch_bounds__(M >= 4096 ? 512 : 256, M >= 4096 ? 1 : 2)
k_col_solve_inv(ClassDesc cd, const ImgDesc* __restrict__ imgs, ImgState* st,
                const float2* __restrict__ tw, const float* __restrict__ d2tab) {
  extern __shared__ __align__(16) float2 smem[];
  constexpr int R = radix_for(M), T = threads_per_team(M);
  const int N = cd.N, Lc = N / 2, B = cd.TB;
  const int cpi = Lc / B;
  const int n_items = cd.n_img * cpi;
  const int tile = M * B;
  const int ts = col_team_stride(M, B);
  float2* landU = smem;
  float2* workI = landU + tile;
  float2* workP = workI + B * ts;
  __shared__ __align__(8) unsigned long long s_bar;  // completion of the landing tile
  const float2* twM = tw + tab_off(M);
  if constexpr (M <= SMEM_TW_MAX) {
    float2* stw = workP + B * ts;
    for (int i = threadIdx.x; i < M; i += blockDim.x) stw[i] = twM[i];
    twM = stw;  // visible after the loop's first __syncthreads()
  }
  if (threadIdx.x == 0) mbar_init(&s_bar);
  __syncthreads();
  unsigned int parity = 0;
  // b-fastest mapping for tile I/O, team-fastest for the in-place stages
  const int b = threadIdx.x % B, j = threadIdx.x / B;
  const int bf = T >= 16 ? threadIdx.x / T : b, jf = T >= 16 ? threadIdx.x % T : j;
  // the item's U_E tile: one bulk copy by thread 0, completed on s_bar; H and
  // Y of the item are prefetched into L2
  auto issue = [&](int item) {
    if (item < n_items) {
      const ImgDesc& d = imgs[cd.img0 + item / cpi];
      const size_t off = (size_t)(item % cpi) * tile;
      if (threadIdx.x == 0) bulk_load(landU, d.S + off, (unsigned int)(tile * sizeof(float2)), &s_bar);
      prefetch_l2(d.H + off, (unsigned int)(tile * sizeof(float2)));
      prefetch_l2(d.Y + off, (unsigned int)(tile * sizeof(float2)));
    }
  };
  issue(blockIdx.x);
  for (int item = blockIdx.x; item < n_items; item += gridDim.x) {
    const int gi = cd.img0 + item / cpi;
    if (!mbar_wait(&s_bar, parity)) atomicOr(&st[gi].status, ST_COPY_TIMEOUT);
    parity ^= 1;
    __syncthreads();
    const ImgDesc& d = imgs[gi];
    const int t = item % cpi;
    const int col = t * B + b;
    const size_t off = (size_t)t * tile;
    const double lamd = __ldcg(&st[gi].lam);
    const bool branch = !(lamd < 1e300);
    if (t == 0 && threadIdx.x == 0) {  // the inverse row pass re-forms them
      st[gi].absmax[0] = 0u;
      st[gi].absmax[1] = 0u;
    }
    const float lam = branch ? 0.0f : (float)lamd;
    const float d2c = __ldg(&d2tab[tab_off(N) + col]);
    float2* bufI = workI + b * ts;
    float2* bufP = workP + b * ts;
    const float2* Hc = d.H + off + b;
    const float2* Yc = d.Y + off + b;
#pragma unroll 4
    for (int i = 0; i < R; ++i) {
      const int k = j + i * T;
      const int e = k * B + b;
      const float d2r = __ldg(&d2tab[tab_off(M) + k]);
      const float2 U = landU[e];
      float2 UI, Up;
      if (col != 0) {
        const float2 Hv = __ldg(&Hc[(size_t)k * B]);
        const float2 Yv = __ldg(&Yc[(size_t)k * B]);
        solve_bin(U, Hv, Yv, lam, d2r + d2c, branch, UI, Up);
      } else {
        const float2 Um = landU[((M - k) & (M - 1)) * B + b];
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
    issue(item + gridDim.x);
    fft_team2<M, true>(workI + bf * ts, workP + bf * ts, jf, twM);
    float2* qi = d.QI + off + b;
    float2* qp = d.Qp + off + b;
#pragma unroll 4
    for (int i = 0; i < R; ++i) {
      const int p = j + i * T;  // storage order; row in_pos(p)
      const size_t k = (size_t)in_pos<M>(p);
      qi[k * B] = bufI[phys(p)];
      qp[k * B] = bufP[phys(p)];
    }
  }
}

// ---------------------------------------------------------------------------
// launch configuration and dispatch
// ---------------------------------------------------------------------------
template <class K>
static int max_threads(K kernel) {
  static int cached = 0;
  if (cached == 0) {
    cudaFuncAttributes a{};
    cached = cudaFuncGetAttributes(&a, (const void*)kernel) == cudaSuccess ? a.maxThreadsPerBlock : 256;
  }
  return cached;
}

static int sm_count() {
  static int n = 0;
  if (n == 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n <= 0) n = 1;
  }
  return n;
}

// Persistent grid: as many blocks as fit on the device at once (never more
// than there are items).
template <class K>
static int persistent_grid(K kernel, int threads, size_t smem, int n_items, int div = 1) {
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, threads, smem) != cudaSuccess ||
      per_sm < 1)
    per_sm = 1;
  long long g = (long long)per_sm * sm_count();
  if (div > 1) g = (g + div - 1) / div;
  return (int)(g < n_items ? g : n_items);
}

// Largest power of two <= v (v >= 1): rows per item and tile widths are
// powers of two, so the tile copies index by shifts.
static int floor_pow2(int v) {
  int p = 1;
  while (2 * p <= v) p *= 2;
  return p;
}

int rows_per_item(int L, int M, int row_threads) {
  const int T = threads_per_team(L);
  int r = (row_threads > 0 ? row_threads : DEF_ROW_THREADS) / T;
  if (r < 1) r = 1;
  if (r > M) r = M;
  return floor_pow2(r);
}

// Tile width of a class's spectra = columns per column item: a block of about
// col_threads threads (512 for M = 4096), at least 2 columns (16-byte
// copies), at most N/2.
int class_tile_width(int M, int N, int col_threads) {
  const int T = M / radix_for(M);
  const int ct = col_threads > 0 ? (col_threads > 256 ? 256 : col_threads) : DEF_COL_THREADS;
  const int threads = M >= 4096 ? 512 : ct;
  int B = threads / T;
  if (B < 2) B = 2;
  if (B > N / 2) B = N / 2;
  return floor_pow2(B);
}

static size_t row_r2c_smem(int L, int rpc) {
  return (size_t)2 * rpc * L * sizeof(float2) + (size_t)row_work_elems(L, rpc) * sizeof(float2) +
         32 * sizeof(double) + (L <= SMEM_TW_MAX ? (size_t)L * sizeof(float2) : 0);
}
static size_t row_c2r_smem(int L, int rpc) {
  return (size_t)rpc * L * sizeof(float2) + (size_t)rpc * team_stride(L) * sizeof(float2) +
         (L <= SMEM_TW_MAX ? (size_t)L * sizeof(float2) : 0);
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
  const int rpc = rows_per_item(L, c.cd.M, c.row_threads);
  const int n_items = c.cd.n_img * c.cd.M / rpc;
  const int thr = rpc * threads_per_team(L);
  const size_t smem = row_r2c_smem(L, rpc);
  const int grid = persistent_grid(k_row_r2c<L>, thr, smem, n_items, c.grid_div);
  k_row_r2c<L><<<grid, thr, smem, s>>>(c.cd, c.imgs, t.tw, rpc, src, dst, sum);
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
static void do_row_c2r(const ClassLaunch& c, const Tables& t, int sel0, int sel1, int dsel0,
                       int dsel1, float scale, cudaStream_t s) {
  const int rpc = rows_per_item(L, c.cd.M, c.row_threads);
  int n_items = c.cd.n_img * c.cd.M / rpc;
  if (sel1 >= 0) n_items *= 2;
  const int thr = rpc * threads_per_team(L);
  const size_t smem = row_c2r_smem(L, rpc);
  const int grid = persistent_grid(k_row_c2r<L>, thr, smem, n_items, c.grid_div);
  k_row_c2r<L><<<grid, thr, smem, s>>>(c.cd, c.imgs, t.tw, rpc, sel0, sel1, dsel0, dsel1, scale,
                                       dsel0 == SEL_UI ? c.st : nullptr);
}

cudaError_t launch_row_c2r(const ClassLaunch& c, const Tables& t, int sel0, int sel1, int dsel0,
                           int dsel1, float scale, cudaStream_t s) {
  switch (c.cd.N / 2) {
    GFD_CASE_L(do_row_c2r, c, t, sel0, sel1, dsel0, dsel1, scale, s)
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

template <int M>
static void do_col_plain(const ClassLaunch& c, const Tables& t, int src, int dst, bool inv,
                         cudaStream_t s) {
  const int Lc = c.cd.N / 2;
  const int T = threads_per_team(M);
  const int mt = inv ? max_threads(k_col_plain<M, true>) : max_threads(k_col_plain<M, false>);
  int B = (mt < 512 ? mt : 512) / T;
  if (B < 1) B = 1;
  if (B > Lc) B = Lc;
  if (B > c.cd.TB) B = c.cd.TB;  // a block stays inside one tile
  const size_t smem = (size_t)B * col_team_stride(M, B) * sizeof(float2);
  const int nblk = c.cd.n_img * (Lc / B);
  if (inv)
    k_col_plain<M, true><<<nblk, B * T, smem, s>>>(c.cd, c.imgs, t.tw, B, src, dst);
  else
    k_col_plain<M, false><<<nblk, B * T, smem, s>>>(c.cd, c.imgs, t.tw, B, src, dst);
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
static size_t col_smem(int B, int landings, int works, int nthr) {
  return (size_t)landings * M * B * sizeof(float2) +
         (size_t)works * B * col_team_stride(M, B) * sizeof(float2) +
         (size_t)((nthr + 31) / 32) * (KNODES + 1) * sizeof(double) +
         (M <= SMEM_TW_MAX ? (size_t)M * sizeof(float2) : 0);
}

template <int M, int NK>
static void do_col_fwd_lambda_nk(const ClassLaunch& c, const Tables& t, int iter, cudaStream_t s) {
  const int Lc = c.cd.N / 2, B = c.cd.TB;
  const int nthr = B * threads_per_team(M);
  const size_t smem = col_smem<M>(B, 1, 1, nthr);
  const int n_items = c.cd.n_img * (Lc / B);
  const int grid = persistent_grid(k_col_fwd_lambda<M, NK>, nthr, smem, n_items, c.grid_div);
  const int row_items = c.cd.M / rows_per_item(c.cd.N / 2, c.cd.M, c.row_threads);
  k_col_fwd_lambda<M, NK><<<grid, nthr, smem, s>>>(c.cd, c.imgs, c.st, t.tw, iter, row_items);
}

// The brackets resolve_warp lays out for iteration `iter` have KNARROW nodes
// from NARROW_FROM on: the pass evaluates exactly those.
template <int M>
static void do_col_fwd_lambda(const ClassLaunch& c, const Tables& t, int iter, cudaStream_t s) {
  if (iter >= NARROW_FROM)
    do_col_fwd_lambda_nk<M, KNARROW>(c, t, iter, s);
  else
    do_col_fwd_lambda_nk<M, KNODES>(c, t, iter, s);
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
  const int chunk = per_img < 16384 ? per_img : 16384;
  const int nblk = c.cd.n_img * (per_img / chunk);
  k_lambda_pass<<<nblk, 256, 0, s>>>(c.cd, c.imgs, c.st, chunk, iter, last_chance ? 1 : 0);
  return cudaGetLastError();
}

template <int M>
static void do_col_solve_inv(const ClassLaunch& c, const Tables& t, cudaStream_t s) {
  const int Lc = c.cd.N / 2, B = c.cd.TB;
  const int nthr = B * threads_per_team(M);
  const size_t smem = col_smem<M>(B, 1, 2, 0);
  const int n_items = c.cd.n_img * (Lc / B);
  const int grid = persistent_grid(k_col_solve_inv<M>, nthr, smem, n_items, c.grid_div);
  k_col_solve_inv<M><<<grid, nthr, smem, s>>>(c.cd, c.imgs, c.st, t.tw, t.d2);
}

cudaError_t launch_col_solve_inv(const ClassLaunch& c, const Tables& t, cudaStream_t s) {
  switch (c.cd.M) {
    GFD_CASE_M(do_col_solve_inv, c, t, s)
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
static int smem_optin() {
  static int v = 0;
  if (v == 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    if (cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess || v <= 0)
      v = 48 * 1024;
  }
  return v;
}

// Allow the kernel the device's opt-in shared memory minus its static part.
template <class K>
static cudaError_t allow_smem(K kernel) {
  cudaFuncAttributes a{};
  cudaError_t e = cudaFuncGetAttributes(&a, (const void*)kernel);
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute((const void*)kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              smem_optin() - (int)a.sharedSizeBytes);
}

template <int L>
static cudaError_t cfg_row() {
  cudaError_t e = allow_smem(k_row_r2c<L>);
  if (e != cudaSuccess) return e;
  return allow_smem(k_row_c2r<L>);
}
template <int M>
static cudaError_t cfg_col() {
  cudaError_t e;
  if ((e = allow_smem(k_col_plain<M, false>)) != cudaSuccess) return e;
  if ((e = allow_smem(k_col_plain<M, true>)) != cudaSuccess) return e;
  if ((e = allow_smem(k_col_fwd_lambda<M, KNODES>)) != cudaSuccess) return e;
  if ((e = allow_smem(k_col_fwd_lambda<M, KNARROW>)) != cudaSuccess) return e;
  return allow_smem(k_col_solve_inv<M>);
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
