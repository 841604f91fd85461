// C-ABI of the guided-filter deconvolution library: argument validation,
// workspace and plan management, launch sequencing and CUDA-graph replay.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdint>
#include <cstdlib>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "launch.h"

#ifndef GFD_CHAINS
#define GFD_CHAINS 4
#endif

using namespace gfd;

namespace {

constexpr int AUX_SLOTS = 8;
// Fallback lambda passes launched per iteration from the fourth iteration on.
constexpr int LATE_LAMBDA_PASSES = 2;
constexpr int CHAINS = GFD_CHAINS;

// A host <-> device copy that the host entry point asks a solve to issue.
struct HostCopy {
  void* dst;
  const void* src;
  size_t bytes;
  cudaMemcpyKind kind;
};

// Copies around a solve from host buffers: `pre` before everything, per
// image (user order) `in` before its setup and `out` after its last
// iteration, `post` after everything.  Recorded into the solve's graph, so
// that one chain's copies overlap the other chains' work.
struct HostCopies {
  std::vector<HostCopy> pre, post;
  std::vector<std::vector<HostCopy>> in, out;
};

struct Plan {
  std::vector<unsigned char> key;
  const HostCopies* copies = nullptr;  // set for the duration of a capture / record
  int n = 0, iters = 0;
  std::vector<int> order;                // internal index -> user index
  std::vector<ClassLaunch> classes;
  // the iterations of the graph-captured solve run as CHAINS concurrent
  // chains over parts of every class, so that the blocks of different phases
  // share the SMs (a kernel's tail overlaps the next kernel of another chain)
  std::vector<ClassLaunch> parts[CHAINS];
  int nparts = CHAINS;
  bool checkpoints = false;  // some image keeps its iterates (u_iters)
  std::vector<ImgDesc> h_imgs;           // internal order
  std::vector<gfdeconv_image> user;      // internal order
  cudaGraphExec_t exec = nullptr;
  long long launches = 0;
};

// Optional event pairs around every launch of record() (instrumentation).
struct Timer {
  std::vector<cudaEvent_t> ev;   // 2 per launch
  std::vector<int> phase;
  std::vector<int> cls;          // class index of each launch (-1: none)
  int cur_cls = -1;
  size_t used = 0;
  cudaError_t begin(cudaStream_t s, int ph) {
    if (2 * used + 2 > ev.size()) {
      for (int i = 0; i < 64; ++i) {
        cudaEvent_t e;
        const cudaError_t r = cudaEventCreate(&e);
        if (r != cudaSuccess) return r;
        ev.push_back(e);
      }
    }
    if (phase.size() <= used) {
      phase.resize(used + 1);
      cls.resize(used + 1);
    }
    phase[used] = ph;
    cls[used] = cur_cls;
    return cudaEventRecord(ev[2 * used], s);
  }
  cudaError_t end(cudaStream_t s) {
    const cudaError_t r = cudaEventRecord(ev[2 * used + 1], s);
    ++used;
    return r;
  }
  ~Timer() {
    for (cudaEvent_t e : ev) cudaEventDestroy(e);
  }
};

// Tile shapes of one canvas size (see gfdeconv_autotune).
struct ClassTune {
  int M, N, col_threads, row_threads, gf_rows;
};

struct TuneTable {
  int chains = CHAINS;  // concurrent chains of a captured solve (1..CHAINS)
  std::vector<ClassTune> cls;
  ClassTune get(int M, int N) const {
    for (const ClassTune& t : cls)
      if (t.M == M && t.N == N) return t;
    return ClassTune{M, N, DEF_COL_THREADS, DEF_ROW_THREADS, DEF_GF_ROWS};
  }
  void set(const ClassTune& t) {
    for (ClassTune& u : cls)
      if (u.M == t.M && u.N == t.N) {
        u = t;
        return;
      }
    cls.push_back(t);
  }
};

struct AuxSlot {
  ImgDesc* d_img = nullptr;
  char* ws = nullptr;
  size_t ws_bytes = 0;
  cudaEvent_t done = nullptr;
  bool used = false;
};

}  // namespace

struct gfdeconv_ctx {
  int device = 0;
  gfdeconv_opts opts{};
  float2* tw = nullptr;
  float* d2 = nullptr;
  float4* twdf = nullptr;
  cudaStream_t cap = nullptr;
  cudaStream_t side[CHAINS - 1] = {};  // further chains of a captured solve
  cudaEvent_t ev_fork = nullptr;
  cudaEvent_t ev_join[CHAINS - 1] = {};
  cudaEvent_t ev_in[CHAINS - 1] = {};  // a chain's host inputs have landed
  char* ws = nullptr;
  size_t ws_bytes = 0;
  ImgDesc* d_imgs = nullptr;
  ImgState* d_st = nullptr;
  int cap_imgs = 0;
  Plan plan;
  bool have_plan = false;
  cudaStream_t last_stream = nullptr;
  long long last_launches = 0;
  ImgState* aux_st = nullptr;
  AuxSlot aux[AUX_SLOTS];
  int aux_next = 0;
  char* stage = nullptr;
  size_t stage_bytes = 0;
  char* hstage = nullptr;  // pinned host staging of the small per-image arrays
  size_t hstage_bytes = 0;
  TuneTable tune;          // tile shapes per canvas size
  char* adj_ws = nullptr;  // workspace of gfdeconv_backward_batched
  size_t adj_ws_bytes = 0;
};

namespace {

bool pow2_in(int v, int lo, int hi) { return v >= lo && v <= hi && (v & (v - 1)) == 0; }

thread_local cudaError_t g_last_cuda_error = cudaSuccess;

int map_err(cudaError_t e) {
  if (e == cudaSuccess) return GFD_OK;
  g_last_cuda_error = e;
  if (e == cudaErrorMemoryAllocation) return GFD_ERR_ALLOC;
  return GFD_ERR_CUDA;
}

bool aligned16(const void* p) { return ((uintptr_t)p & 15) == 0; }

// Device image planes are read and written with 16-byte accesses.
int validate_device_planes(const gfdeconv_image& im) {
  if (!aligned16(im.y) || !aligned16(im.u_out) || !aligned16(im.u_orig) || !aligned16(im.u_init) ||
      !aligned16(im.uI_out) || !aligned16(im.up_out) || !aligned16(im.u_iters))
    return GFD_ERR_INVALID_ARG;
  return GFD_OK;
}

int validate_image(const gfdeconv_image& im, int iters) {
  if (!im.y || !im.h || !im.u_out) return GFD_ERR_INVALID_ARG;
  if (!pow2_in(im.M, 8, 4096) || !pow2_in(im.N, 8, 4096)) return GFD_ERR_UNSUPPORTED_SIZE;
  if (im.kh < 1 || im.kw < 1 || im.kh > 255 || im.kw > 255 || !(im.kh & 1) || !(im.kw & 1))
    return GFD_ERR_INVALID_ARG;
  if (!std::isfinite(im.sigma) || !std::isfinite(im.eps)) return GFD_ERR_NONFINITE_INPUT;
  if (!(im.sigma > 0.0) || !(im.eps > 0.0)) return GFD_ERR_INVALID_ARG;
  if (im.w < 1 || im.w > 17 || !(im.w & 1)) return GFD_ERR_INVALID_ARG;
  if (im.isnr_out && !im.u_orig) return GFD_ERR_INVALID_ARG;
  if (iters < 0) return GFD_ERR_INVALID_ARG;
  return GFD_OK;
}

size_t align256(size_t b) { return (b + 255) & ~(size_t)255; }

// per-item partial sums of the spectral passes: column items hold >= 2
// columns, fallback-pass items >= 4096 bins (or the whole image)
size_t part_doubles(int M, int N) {
  const size_t Lc = (size_t)N / 2;
  const size_t col_items = Lc / 2;
  const size_t pass_items = (size_t)M * Lc / 4096 + 1;
  return (KNODES + 1) * (col_items > pass_items ? col_items : pass_items);
}

size_t image_ws_bytes(int M, int N) {
  const size_t P = (size_t)M * N;
  return 7 * align256(P * sizeof(float)) + 4 * align256((size_t)M * sizeof(float2)) +
         align256(part_doubles(M, N) * sizeof(double)) + align256((size_t)M * sizeof(double));
}

cudaError_t ensure_ws(gfdeconv_ctx* c, size_t bytes) {
  if (bytes <= c->ws_bytes) return cudaSuccess;
  cudaError_t e = cudaDeviceSynchronize();
  if (e != cudaSuccess) return e;
  if (c->ws) cudaFree(c->ws);
  c->ws = nullptr;
  c->ws_bytes = 0;
  e = cudaMalloc(&c->ws, bytes);
  if (e != cudaSuccess) return e;
  c->ws_bytes = bytes;
  return cudaSuccess;
}

cudaError_t ensure_imgs(gfdeconv_ctx* c, int n) {
  if (n <= c->cap_imgs) return cudaSuccess;
  cudaError_t e = cudaDeviceSynchronize();
  if (e != cudaSuccess) return e;
  if (c->d_imgs) cudaFree(c->d_imgs);
  if (c->d_st) cudaFree(c->d_st);
  c->d_imgs = nullptr;
  c->d_st = nullptr;
  c->cap_imgs = 0;
  if ((e = cudaMalloc(&c->d_imgs, sizeof(ImgDesc) * n)) != cudaSuccess) return e;
  if ((e = cudaMalloc(&c->d_st, sizeof(ImgState) * n)) != cudaSuccess) return e;
  c->cap_imgs = n;
  return cudaSuccess;
}

std::vector<unsigned char> make_key(const gfdeconv_ctx* c, int n, const gfdeconv_image* imgs,
                                    int iters) {
  std::vector<unsigned char> k(sizeof(int) * 2 + sizeof(gfdeconv_opts) +
                               sizeof(gfdeconv_image) * (size_t)n);
  unsigned char* p = k.data();
  std::memcpy(p, &n, sizeof(int));
  p += sizeof(int);
  std::memcpy(p, &iters, sizeof(int));
  p += sizeof(int);
  std::memcpy(p, &c->opts, sizeof(gfdeconv_opts));
  p += sizeof(gfdeconv_opts);
  std::memcpy(p, imgs, sizeof(gfdeconv_image) * (size_t)n);
  return k;
}

void drop_plan(gfdeconv_ctx* c) {
  if (c->plan.exec) cudaGraphExecDestroy(c->plan.exec);
  c->plan = Plan();
  c->have_plan = false;
}

cudaError_t build_plan(gfdeconv_ctx* c, int n, const gfdeconv_image* imgs, int iters) {
  Plan& pl = c->plan;
  pl.n = n;
  pl.iters = iters;
  // group images by canvas, in order of first appearance
  std::vector<std::pair<int, int>> sizes;
  std::vector<std::vector<int>> members;
  for (int i = 0; i < n; ++i) {
    const std::pair<int, int> sz(imgs[i].M, imgs[i].N);
    size_t ci = 0;
    while (ci < sizes.size() && sizes[ci] != sz) ++ci;
    if (ci == sizes.size()) {
      sizes.push_back(sz);
      members.emplace_back();
    }
    members[ci].push_back(i);
  }
  size_t total = 0;
  for (int i = 0; i < n; ++i) total += image_ws_bytes(imgs[i].M, imgs[i].N);
  cudaError_t e = ensure_ws(c, total);
  if (e != cudaSuccess) return e;
  if ((e = ensure_imgs(c, n)) != cudaSuccess) return e;
  pl.order.clear();
  pl.h_imgs.clear();
  pl.user.clear();
  pl.classes.clear();
  char* cur = c->ws;
  for (size_t ci = 0; ci < sizes.size(); ++ci) {
    ClassLaunch cl{};
    cl.cd.M = sizes[ci].first;
    cl.cd.N = sizes[ci].second;
    cl.cd.n_img = (int)members[ci].size();
    cl.cd.img0 = (int)pl.order.size();
    const ClassTune tn = c->tune.get(cl.cd.M, cl.cd.N);
    cl.cd.TB = class_tile_width(cl.cd.M, cl.cd.N, tn.col_threads);
    cl.row_threads = tn.row_threads;
    cl.gf_rows = tn.gf_rows;
    cl.class_id = (int)ci;
    cl.imgs = c->d_imgs;
    cl.st = c->d_st;
    cl.max_rad = 0;
    cl.n_rad_groups = 0;
    // order the class by window radius: one guided-filter launch per radius
    std::stable_sort(members[ci].begin(), members[ci].end(),
                     [&](int a, int b) { return imgs[a].w < imgs[b].w; });
    for (int ui : members[ci]) {
      const int rad = (imgs[ui].w - 1) / 2;
      if (cl.n_rad_groups == 0 || cl.rad_groups[cl.n_rad_groups - 1].rad != rad)
        cl.rad_groups[cl.n_rad_groups++] = RadGroup{(int)pl.order.size(), 0, rad};
      cl.rad_groups[cl.n_rad_groups - 1].n_img += 1;
      const gfdeconv_image& im = imgs[ui];
      const size_t P = (size_t)im.M * im.N;
      ImgDesc d{};
      d.y = im.y;
      d.h = im.h;
      d.u = im.u_out;
      d.uo = im.u_orig;
      d.u0 = im.u_init;
      d.u_iters = im.u_iters;
      d.lam_out = im.lambda_out;
      d.isnr_out = im.isnr_out;
      d.res_out = im.res_out;
      d.kh = im.kh;
      d.kw = im.kw;
      d.w = im.w;
      d.sigma = im.sigma;
      d.eps = im.eps;
      d.rho_fixed = c->opts.rho;
      d.lam_rtol = c->opts.lambda_rtol;
      float2** planes[5] = {&d.S, &d.QI, &d.Qp, &d.H, &d.Y};
      for (float2** pp : planes) {
        *pp = reinterpret_cast<float2*>(cur);
        cur += align256(P * sizeof(float));
      }
      float** rplanes[2] = {&d.uI, &d.up};
      for (float** pp : rplanes) {
        *pp = reinterpret_cast<float*>(cur);
        cur += align256(P * sizeof(float));
      }
      float2** cols[4] = {&d.H0, &d.HN, &d.Y0, &d.YN};
      for (float2** pp : cols) {
        *pp = reinterpret_cast<float2*>(cur);
        cur += align256((size_t)im.M * sizeof(float2));
      }
      d.part = reinterpret_cast<double*>(cur);
      cur += align256(part_doubles(im.M, im.N) * sizeof(double));
      d.rowsum = reinterpret_cast<double*>(cur);
      cur += align256((size_t)im.M * sizeof(double));
      cl.max_rad = std::max(cl.max_rad, (im.w - 1) / 2);
      if (im.u_iters) pl.checkpoints = true;
      pl.order.push_back(ui);
      pl.h_imgs.push_back(d);
      pl.user.push_back(im);
    }
    pl.classes.push_back(cl);
  }
  // parts: CHAINS consecutive runs of the images of every class, with their
  // window-radius groups cut to the range
  for (auto& v : pl.parts) v.clear();
  const int nparts = std::max(1, std::min(CHAINS, c->tune.chains));
  pl.nparts = nparts;
  for (const ClassLaunch& cl : pl.classes) {
    for (int part = 0; part < nparts; ++part) {
      const int lo = cl.cd.img0 + (int)((long long)cl.cd.n_img * part / nparts);
      const int hi = cl.cd.img0 + (int)((long long)cl.cd.n_img * (part + 1) / nparts);
      if (hi <= lo) continue;
      ClassLaunch q = cl;
      q.cd.img0 = lo;
      q.cd.n_img = hi - lo;
      q.n_rad_groups = 0;
      q.max_rad = 0;
      for (int g = 0; g < cl.n_rad_groups; ++g) {
        const RadGroup& rg = cl.rad_groups[g];
        const int a0 = std::max(rg.img0, lo), a1 = std::min(rg.img0 + rg.n_img, hi);
        if (a1 <= a0) continue;
        q.rad_groups[q.n_rad_groups++] = RadGroup{a0, a1 - a0, rg.rad};
        q.max_rad = std::max(q.max_rad, rg.rad);
      }
      pl.parts[part].push_back(q);
    }
  }
  return cudaMemcpy(c->d_imgs, pl.h_imgs.data(), sizeof(ImgDesc) * n, cudaMemcpyHostToDevice);
}

#define GFD_CK(x)                            \
  do {                                       \
    cudaError_t e_ = (x);                    \
    if (e_ != cudaSuccess) return e_;        \
  } while (0)

// Enqueue the whole solve: setup (a0), then Steps 1-3 for every iteration.
// With a timer, every launch is bracketed by an event pair tagged by phase.
#define GFD_T(ph, call)                                  \
  do {                                                   \
    if (tm) GFD_CK(tm->begin(s, ph));                    \
    GFD_CK(call);                                        \
    if (tm) GFD_CK(tm->end(s));                          \
  } while (0)

cudaError_t record(gfdeconv_ctx* c, Plan& pl, cudaStream_t s, Timer* tm = nullptr,
                   bool chains = false) {
  long long L = 0;
  const Tables t{c->tw, c->d2, c->twdf};
  const int var_mode = c->opts.var_precision, boundary = c->opts.boundary;
  const int passes = c->opts.lambda_max_passes;
  const HostCopies* hc = pl.copies;
  auto issue = [&](const std::vector<HostCopy>& v, cudaStream_t q) -> cudaError_t {
    for (const HostCopy& cp : v) GFD_CK(cudaMemcpyAsync(cp.dst, cp.src, cp.bytes, cp.kind, q));
    return cudaSuccess;
  };
  // per-image copies of the images of a list of classes (internal order ->
  // user order), inputs or outputs
  auto issue_imgs = [&](std::vector<ClassLaunch>& classes, bool in, cudaStream_t q) -> cudaError_t {
    if (!hc) return cudaSuccess;
    for (const ClassLaunch& cl : classes)
      for (int i = cl.cd.img0; i < cl.cd.img0 + cl.cd.n_img; ++i)
        GFD_CK(issue(in ? hc->in[pl.order[i]] : hc->out[pl.order[i]], q));
    return cudaSuccess;
  };
  if (hc) GFD_CK(issue(hc->pre, s));
  GFD_T(GFD_PHASE_COPY, cudaMemsetAsync(c->d_st, 0, sizeof(ImgState) * pl.n, s));
  // setup (once per solve) over a list of classes, on stream q
  auto setup = [&](std::vector<ClassLaunch>& classes, cudaStream_t q) -> cudaError_t {
    cudaStream_t s = q;  // the GFD_T macro records on `s`
    for (auto& cl : classes) {
      if (tm) tm->cur_cls = cl.class_id;
      GFD_T(GFD_PHASE_COPY, launch_init_u(cl, s));  // u_E = u_init or 0
      GFD_T(GFD_PHASE_SETUP, launch_setup_stats(cl, s));
      L += 2;
    }
    for (auto& cl : classes) {
      if (tm) tm->cur_cls = cl.class_id;
      GFD_T(GFD_PHASE_SETUP, launch_setup_init(cl, c->opts.rho, s));
      L += 2;  // k_setup_init, k_zero_parts
    }
    for (auto& cl : classes) {
      if (tm) tm->cur_cls = cl.class_id;
      GFD_T(GFD_PHASE_SETUP, launch_embed_psf(cl, SEL_UI, s));
      // H and Y in double-float, rounded once (they fix the residual of Eq. 10-11)
      GFD_T(GFD_PHASE_SETUP, launch_fft2_r2c_df(cl, t.twdf, SEL_UI, SEL_H, s));
      GFD_T(GFD_PHASE_SETUP, launch_fft2_r2c_df(cl, t.twdf, SEL_Y, SEL_YS, s));
      GFD_T(GFD_PHASE_SETUP, launch_unpack_dc(cl, s));
      L += 6;
    }
    return cudaSuccess;
  };
  // Steps 1-3 for every iteration over a list of classes, on stream q
  auto iterate = [&](std::vector<ClassLaunch>& classes, cudaStream_t q) -> cudaError_t {
    cudaStream_t s = q;  // the GFD_T macro records on `s`
    for (int k = 0; k < pl.iters; ++k) {
      for (auto& cl : classes) {
        if (tm) tm->cur_cls = cl.class_id;
        if (pl.checkpoints) {  // u_E^k of the images that keep checkpoints
          GFD_T(GFD_PHASE_COPY, launch_save_iterate(cl, k, s));
          ++L;
        }
        GFD_T(GFD_PHASE_ROW_FWD, launch_row_r2c(cl, t, SEL_U, SEL_S, true, s));
        GFD_T(GFD_PHASE_COL_FWD_LAMBDA, launch_col_fwd_lambda(cl, t, k, s));
        L += 2;
      }
      // iterations 0-2 start from wide brackets; later ones from the
      // extrapolated root, which the fused pass almost always resolves
      const int npass = k < 3 ? passes : std::min(passes, LATE_LAMBDA_PASSES);
      for (int p = 1; p <= npass; ++p)
        for (auto& cl : classes) {
          if (tm) tm->cur_cls = cl.class_id;
          GFD_T(GFD_PHASE_LAMBDA_PASS, launch_lambda_pass(cl, k, p == npass, s));
          ++L;
        }
      for (auto& cl : classes) {
        if (tm) tm->cur_cls = cl.class_id;
        GFD_T(GFD_PHASE_COL_SOLVE_INV, launch_col_solve_inv(cl, t, s));
        GFD_T(GFD_PHASE_ROW_INV, launch_row_c2r(cl, t, SEL_QI, SEL_QP, SEL_UI, SEL_UP,
                                                1.0f / ((float)cl.cd.M * (float)cl.cd.N), s));
        GFD_T(GFD_PHASE_GUIDED_FILTER, launch_guided_filter(cl, k, var_mode, boundary, s));
        L += 2 + cl.n_rad_groups;  // one guided-filter launch per window radius
      }
    }
    return cudaSuccess;
  };
  if (tm) tm->cur_cls = -1;
  if (chains && !tm && pl.nparts > 1 && !pl.parts[1].empty()) {
    GFD_CK(cudaEventRecord(c->ev_fork, s));
    for (int q = 1; q < pl.nparts; ++q) GFD_CK(cudaStreamWaitEvent(c->side[q - 1], c->ev_fork, 0));
    // host inputs chain after chain: each chain's copies start once the
    // previous chain's have landed, so the first chain computes after its own
    // share of the transfer instead of after the interleaved whole
    GFD_CK(issue_imgs(pl.parts[0], true, s));
    if (hc) GFD_CK(cudaEventRecord(c->ev_in[0], s));
    GFD_CK(setup(pl.parts[0], s));
    GFD_CK(iterate(pl.parts[0], s));
    GFD_CK(issue_imgs(pl.parts[0], false, s));
    for (int q = 1; q < pl.nparts; ++q) {
      if (hc) GFD_CK(cudaStreamWaitEvent(c->side[q - 1], c->ev_in[q - 1], 0));
      GFD_CK(issue_imgs(pl.parts[q], true, c->side[q - 1]));
      if (hc && q < pl.nparts - 1) GFD_CK(cudaEventRecord(c->ev_in[q], c->side[q - 1]));
      GFD_CK(setup(pl.parts[q], c->side[q - 1]));
      GFD_CK(iterate(pl.parts[q], c->side[q - 1]));
      GFD_CK(issue_imgs(pl.parts[q], false, c->side[q - 1]));
      GFD_CK(cudaEventRecord(c->ev_join[q - 1], c->side[q - 1]));
      GFD_CK(cudaStreamWaitEvent(s, c->ev_join[q - 1], 0));
    }
  } else {
    GFD_CK(issue_imgs(pl.classes, true, s));
    GFD_CK(setup(pl.classes, s));
    GFD_CK(iterate(pl.classes, s));
    GFD_CK(issue_imgs(pl.classes, false, s));
  }
  for (int i = 0; i < pl.n; ++i) {
    const gfdeconv_image& u = pl.user[i];
    const size_t bytes = (size_t)u.M * u.N * sizeof(float);
    if (u.uI_out && pl.iters > 0)
      GFD_T(GFD_PHASE_COPY, cudaMemcpyAsync(u.uI_out, pl.h_imgs[i].uI, bytes, cudaMemcpyDeviceToDevice, s));
    if (u.up_out && pl.iters > 0)
      GFD_T(GFD_PHASE_COPY, cudaMemcpyAsync(u.up_out, pl.h_imgs[i].up, bytes, cudaMemcpyDeviceToDevice, s));
  }
  if (hc) GFD_CK(issue(hc->post, s));
  pl.launches = L;
  return cudaSuccess;
}

cudaError_t capture(gfdeconv_ctx* c, Plan& pl) {
  GFD_CK(cudaStreamBeginCapture(c->cap, cudaStreamCaptureModeThreadLocal));
  const cudaError_t e = record(c, pl, c->cap, nullptr, true);
  cudaGraph_t g = nullptr;
  const cudaError_t e2 = cudaStreamEndCapture(c->cap, &g);
  if (e != cudaSuccess) {
    if (g) cudaGraphDestroy(g);
    return e;
  }
  if (e2 != cudaSuccess) return e2;
  const cudaError_t e3 = cudaGraphInstantiate(&pl.exec, g, 0);
  cudaGraphDestroy(g);
  return e3;
}

// Reserve an aux slot (descriptor + workspace) for a single-image utility call.
cudaError_t aux_slot(gfdeconv_ctx* c, size_t ws_bytes, AuxSlot** out) {
  AuxSlot& a = c->aux[c->aux_next];
  c->aux_next = (c->aux_next + 1) % AUX_SLOTS;
  if (a.used) GFD_CK(cudaEventSynchronize(a.done));
  if (!a.d_img) GFD_CK(cudaMalloc(&a.d_img, sizeof(ImgDesc)));
  if (!a.done) GFD_CK(cudaEventCreateWithFlags(&a.done, cudaEventDisableTiming));
  if (ws_bytes > a.ws_bytes) {
    if (a.ws) cudaFree(a.ws);
    a.ws = nullptr;
    a.ws_bytes = 0;
    GFD_CK(cudaMalloc(&a.ws, ws_bytes));
    a.ws_bytes = ws_bytes;
  }
  *out = &a;
  return cudaSuccess;
}

cudaError_t aux_upload(AuxSlot* a, const ImgDesc& d, cudaStream_t s) {
  return cudaMemcpyAsync(a->d_img, &d, sizeof(ImgDesc), cudaMemcpyHostToDevice, s);
}

cudaError_t aux_finish(AuxSlot* a, cudaStream_t s) {
  a->used = true;
  return cudaEventRecord(a->done, s);
}

int solve_batched_dev(gfdeconv_ctx* c, int n, const gfdeconv_image* imgs, int iters,
                      cudaStream_t s, const HostCopies* hc = nullptr) {
  std::vector<unsigned char> key = make_key(c, n, imgs, iters);
  if (hc) {  // the copies are part of the graph: their addresses are part of the key
    auto put = [&](const std::vector<HostCopy>& v) {
      auto raw = [&](const void* p, size_t b) {
        const size_t o = key.size();
        key.resize(o + b);
        std::memcpy(key.data() + o, p, b);
      };
      const size_t cnt = v.size();
      raw(&cnt, sizeof(cnt));
      for (const HostCopy& cp : v) {  // field by field (no padding bytes)
        const int kind = (int)cp.kind;
        raw(&cp.dst, sizeof(cp.dst));
        raw(&cp.src, sizeof(cp.src));
        raw(&cp.bytes, sizeof(cp.bytes));
        raw(&kind, sizeof(kind));
      }
    };
    put(hc->pre);
    put(hc->post);
    for (const auto& v : hc->in) put(v);
    for (const auto& v : hc->out) put(v);
  }
  c->plan.copies = nullptr;
  if (!(c->have_plan && c->plan.key == key)) {
    cudaError_t e = cudaDeviceSynchronize();
    if (e != cudaSuccess) return map_err(e);
    drop_plan(c);
    e = build_plan(c, n, imgs, iters);
    if (e != cudaSuccess) {
      drop_plan(c);
      return map_err(e);
    }
    if (c->opts.use_graphs) {
      c->plan.copies = hc;
      e = capture(c, c->plan);
      c->plan.copies = nullptr;
      if (e != cudaSuccess) {
        drop_plan(c);
        cudaGetLastError();
        return map_err(e);
      }
    }
    c->plan.key.swap(key);
    c->have_plan = true;
  }
  cudaError_t e;
  if (c->opts.use_graphs) {
    e = cudaGraphLaunch(c->plan.exec, s);
  } else {
    c->plan.copies = hc;
    e = record(c, c->plan, s);
    c->plan.copies = nullptr;
  }
  c->last_stream = s;
  c->last_launches = c->plan.launches;
  return map_err(e);
}

// Tile-shape file: text lines "chains C" and
// "class M N col_threads CT row_threads RT gf_rows GR"; '#' starts a comment.
// A missing file is an empty table.  Returns false on a malformed line or a
// value outside the kernels' ranges.
bool valid_tune(const ClassTune& t) {
  auto p2 = [](int v, int lo, int hi) { return v >= lo && v <= hi && (v & (v - 1)) == 0; };
  return p2(t.M, 8, 4096) && p2(t.N, 8, 4096) && p2(t.col_threads, 32, 256) &&
         p2(t.row_threads, 32, 256) && p2(t.gf_rows, 16, 64);
}

bool load_tune(const char* path, TuneTable* out) {
  TuneTable t;
  std::FILE* f = std::fopen(path, "r");
  if (!f) {
    *out = t;
    return true;
  }
  char line[256];
  bool ok = true;
  while (ok && std::fgets(line, sizeof line, f)) {
    char* h = std::strchr(line, '#');
    if (h) *h = 0;
    char word[32] = {0};
    if (std::sscanf(line, "%31s", word) != 1) continue;  // blank
    if (!std::strcmp(word, "chains")) {
      int q = 0;
      ok = std::sscanf(line, "%*s %d", &q) == 1 && q >= 1 && q <= CHAINS;
      if (ok) t.chains = q;
    } else if (!std::strcmp(word, "class")) {
      ClassTune c{};
      ok = std::sscanf(line, "%*s %d %d col_threads %d row_threads %d gf_rows %d", &c.M, &c.N,
                       &c.col_threads, &c.row_threads, &c.gf_rows) == 5 &&
           valid_tune(c);
      if (ok) t.set(c);
    } else {
      ok = false;
    }
  }
  std::fclose(f);
  if (ok) *out = t;
  return ok;
}

bool save_tune(const char* path, const TuneTable& t) {
  const std::string tmp = std::string(path) + ".tmp";
  std::FILE* f = std::fopen(tmp.c_str(), "w");
  if (!f) return false;
  std::fprintf(f, "# gfdeconv tile shapes, written by gfdeconv_autotune\n");
  std::fprintf(f, "chains %d\n", t.chains);
  for (const ClassTune& c : t.cls)
    std::fprintf(f, "class %d %d col_threads %d row_threads %d gf_rows %d\n", c.M, c.N,
                 c.col_threads, c.row_threads, c.gf_rows);
  const bool ok = std::fclose(f) == 0;
  return ok && std::rename(tmp.c_str(), path) == 0;
}

}  // namespace

// ---------------------------------------------------------------------------
// C-ABI
// ---------------------------------------------------------------------------
extern "C" {

const char* gfdeconv_strerror(int code) {
  switch (code) {
    case GFD_OK: return "ok";
    case GFD_ERR_INVALID_ARG: return "invalid argument";
    case GFD_ERR_UNSUPPORTED_SIZE: return "unsupported size (M, N must be powers of two in [8, 4096])";
    case GFD_ERR_NONFINITE_INPUT: return "non-finite scalar argument";
    case GFD_ERR_ALLOC: return "device allocation failed";
    case GFD_ERR_CUDA: return "CUDA runtime error";
    case GFD_ERR_NONCONVERGED: return "regularisation parameter did not converge";
    case GFD_ERR_TIMEOUT: return "timeout";
    case GFD_ERR_SCRATCH_LIMIT:
      return "size exceeds the static scratch of gfdeconv_fft2_r2c_noalloc (M*N <= 1024*1024)";
    default: return "unknown error";
  }
}

int gfdeconv_create(gfdeconv_ctx** out, int cuda_device, const gfdeconv_opts* opts) {
  if (!out) return GFD_ERR_INVALID_ARG;
  *out = nullptr;
  int ndev = 0;
  cudaError_t e = cudaGetDeviceCount(&ndev);
  if (e != cudaSuccess) return map_err(e);
  if (cuda_device < 0 || cuda_device >= ndev) return GFD_ERR_INVALID_ARG;
  if (opts) {
    if (opts->rho > 1.0 || !std::isfinite(opts->rho)) return GFD_ERR_INVALID_ARG;
    if (opts->var_precision < GFD_VAR_COMPENSATED || opts->var_precision > GFD_VAR_DOUBLE_FLOAT)
      return GFD_ERR_INVALID_ARG;
    if (opts->boundary != GFD_BOUNDARY_PERIODIC && opts->boundary != GFD_BOUNDARY_TRUNCATED)
      return GFD_ERR_INVALID_ARG;
    if (opts->lambda_max_passes > 16) return GFD_ERR_INVALID_ARG;
    if (!std::isfinite(opts->lambda_rtol) ||
        (opts->lambda_rtol > 0.0 && (opts->lambda_rtol < 1e-14 || opts->lambda_rtol > 1e-2)))
      return GFD_ERR_INVALID_ARG;
  }
  TuneTable tune;
  if (opts && opts->tune_cache && opts->tune_cache[0] && !load_tune(opts->tune_cache, &tune))
    return GFD_ERR_INVALID_ARG;
  if ((e = cudaSetDevice(cuda_device)) != cudaSuccess) return map_err(e);
  gfdeconv_ctx* c = new (std::nothrow) gfdeconv_ctx();
  if (!c) return GFD_ERR_ALLOC;
  c->device = cuda_device;
  if (opts) {
    c->opts = *opts;
  } else {
    c->opts.var_precision = GFD_VAR_COMPENSATED;
    c->opts.rho = 0.0;
    c->opts.use_graphs = 1;
    c->opts.boundary = GFD_BOUNDARY_PERIODIC;
  }
  if (c->opts.lambda_max_passes <= 0) c->opts.lambda_max_passes = LAMBDA_FALLBACK_PASSES;
  if (c->opts.lambda_rtol <= 0.0) c->opts.lambda_rtol = 1e-13;
  c->opts.tune_cache = nullptr;  // not retained
  c->tune = tune;
  e = configure_kernels();
  if (e != cudaSuccess) {
    delete c;
    return map_err(e);
  }
  // twiddles W_L^m and gradient weights 4 sin^2(pi m / L) for every
  // power-of-two L <= 4096 (size L at offset L - 2), in double, rounded once
  std::vector<float2> tw(TAB_ENTRIES);
  std::vector<float> d2(TAB_ENTRIES);
  const double pi = 3.14159265358979323846;
  for (int L = 2; L <= TW_N; L *= 2) {
    for (int m = 0; m < L; ++m) {
      const double th = 2.0 * pi * m / L;
      tw[tab_off(L) + m] = make_float2((float)std::cos(th), (float)-std::sin(th));
      const double sn = std::sin(pi * m / L);
      d2[tab_off(L) + m] = (float)(4.0 * sn * sn);
    }
  }
  std::vector<float4> twdf(TAB_ENTRIES);
  for (int L = 2; L <= TW_N; L *= 2) {
    for (int m = 0; m < L; ++m) {
      const double th = 2.0 * pi * m / L;
      const double re = std::cos(th), im = -std::sin(th);
      const float rh = (float)re, ih = (float)im;
      twdf[tab_off(L) + m] = make_float4(rh, (float)(re - rh), ih, (float)(im - ih));
    }
  }
  if ((e = cudaMalloc(&c->tw, sizeof(float2) * TAB_ENTRIES)) != cudaSuccess ||
      (e = cudaMalloc(&c->twdf, sizeof(float4) * TAB_ENTRIES)) != cudaSuccess ||
      (e = cudaMemcpy(c->twdf, twdf.data(), sizeof(float4) * TAB_ENTRIES, cudaMemcpyHostToDevice)) != cudaSuccess ||
      (e = cudaMalloc(&c->d2, sizeof(float) * TAB_ENTRIES)) != cudaSuccess ||
      (e = cudaMemcpy(c->tw, tw.data(), sizeof(float2) * TAB_ENTRIES, cudaMemcpyHostToDevice)) != cudaSuccess ||
      (e = cudaMemcpy(c->d2, d2.data(), sizeof(float) * TAB_ENTRIES, cudaMemcpyHostToDevice)) != cudaSuccess ||
      (e = cudaMalloc(&c->aux_st, sizeof(ImgState))) != cudaSuccess ||
      (e = cudaMemset(c->aux_st, 0, sizeof(ImgState))) != cudaSuccess ||
      (e = cudaStreamCreateWithFlags(&c->cap, cudaStreamNonBlocking)) != cudaSuccess ||
      (e = cudaEventCreateWithFlags(&c->ev_fork, cudaEventDisableTiming)) != cudaSuccess) {
    gfdeconv_destroy(c);
    return map_err(e);
  }
  for (int q = 0; q < CHAINS - 1; ++q) {
    if ((e = cudaStreamCreateWithFlags(&c->side[q], cudaStreamNonBlocking)) != cudaSuccess ||
        (e = cudaEventCreateWithFlags(&c->ev_join[q], cudaEventDisableTiming)) != cudaSuccess ||
        (e = cudaEventCreateWithFlags(&c->ev_in[q], cudaEventDisableTiming)) != cudaSuccess) {
      gfdeconv_destroy(c);
      return map_err(e);
    }
  }

  *out = c;
  return GFD_OK;
}

void gfdeconv_destroy(gfdeconv_ctx* c) {
  if (!c) return;
  cudaSetDevice(c->device);
  cudaDeviceSynchronize();
  drop_plan(c);
  for (AuxSlot& a : c->aux) {
    if (a.d_img) cudaFree(a.d_img);
    if (a.ws) cudaFree(a.ws);
    if (a.done) cudaEventDestroy(a.done);
  }
  if (c->tw) cudaFree(c->tw);
  if (c->twdf) cudaFree(c->twdf);
  if (c->d2) cudaFree(c->d2);
  if (c->ws) cudaFree(c->ws);
  if (c->d_imgs) cudaFree(c->d_imgs);
  if (c->d_st) cudaFree(c->d_st);
  if (c->aux_st) cudaFree(c->aux_st);
  if (c->stage) cudaFree(c->stage);
  if (c->adj_ws) cudaFree(c->adj_ws);
  if (c->hstage) cudaFreeHost(c->hstage);
  if (c->cap) cudaStreamDestroy(c->cap);
  for (int q = 0; q < CHAINS - 1; ++q) {
    if (c->side[q]) cudaStreamDestroy(c->side[q]);
    if (c->ev_join[q]) cudaEventDestroy(c->ev_join[q]);
    if (c->ev_in[q]) cudaEventDestroy(c->ev_in[q]);
  }
  if (c->ev_fork) cudaEventDestroy(c->ev_fork);
  delete c;
}

int gfdeconv_solve_batched(gfdeconv_ctx* c, int n, const gfdeconv_image* imgs, int iters,
                           void* stream) {
  if (!c || !imgs || n <= 0) return GFD_ERR_INVALID_ARG;
  for (int i = 0; i < n; ++i) {
    int r = validate_image(imgs[i], iters);
    if (r == GFD_OK) r = validate_device_planes(imgs[i]);
    if (r != GFD_OK) return r;
  }
  if (cudaSetDevice(c->device) != cudaSuccess) return GFD_ERR_CUDA;
  return solve_batched_dev(c, n, imgs, iters, (cudaStream_t)stream);
}

int gfdeconv_autotune(gfdeconv_ctx* c, int n, const gfdeconv_image* imgs, int iters,
                      const char* path, void* stream) {
  if (!c || !imgs || n <= 0) return GFD_ERR_INVALID_ARG;
  for (int i = 0; i < n; ++i) {
    int r = validate_image(imgs[i], iters);
    if (r == GFD_OK) r = validate_device_planes(imgs[i]);
    if (r != GFD_OK) return r;
  }
  if (cudaSetDevice(c->device) != cudaSuccess) return GFD_ERR_CUDA;
  cudaStream_t s = (cudaStream_t)stream;
  TuneTable saved = c->tune;
  if (path && path[0] && !load_tune(path, &saved)) return GFD_ERR_INVALID_ARG;
  // the batch's canvas sizes, in order of first appearance (build_plan's order)
  std::vector<std::pair<int, int>> sizes;
  for (int i = 0; i < n; ++i) {
    const std::pair<int, int> sz(imgs[i].M, imgs[i].N);
    if (std::find(sizes.begin(), sizes.end(), sz) == sizes.end()) sizes.push_back(sz);
  }
  TuneTable cur = saved;
  for (const auto& sz : sizes) cur.set(cur.get(sz.first, sz.second));
  // Event-timed direct launches of the whole solve; per class and phase, the
  // summed device milliseconds of the second of two runs.
  auto measure = [&](std::vector<std::vector<double>>* per) -> cudaError_t {
    c->tune = cur;
    cudaError_t e = cudaDeviceSynchronize();
    if (e != cudaSuccess) return e;
    drop_plan(c);
    if ((e = build_plan(c, n, imgs, iters)) != cudaSuccess) return e;
    c->have_plan = true;
    c->plan.key = make_key(c, n, imgs, iters);
    for (int rep = 0; rep < 2; ++rep) {
      Timer tm;
      if ((e = record(c, c->plan, s, &tm)) != cudaSuccess) return e;
      if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return e;
      if (rep == 0) continue;
      per->assign(sizes.size(), std::vector<double>(GFD_NUM_PHASES, 0.0));
      for (size_t i = 0; i < tm.used; ++i) {
        float ms = 0.0f;
        if ((e = cudaEventElapsedTime(&ms, tm.ev[2 * i], tm.ev[2 * i + 1])) != cudaSuccess) return e;
        const int ci = tm.cls[i], ph = tm.phase[i];
        if (ci >= 0 && ci < (int)sizes.size() && ph >= 0 && ph < GFD_NUM_PHASES)
          (*per)[ci][ph] += ms;
      }
    }
    return cudaSuccess;
  };
  auto fail = [&](cudaError_t e) {
    c->tune = saved;
    drop_plan(c);
    return map_err(e);
  };
  // one shape at a time: every class takes each candidate together; each
  // class keeps its fastest over the phases the shape affects
  struct Axis {
    int ClassTune::*field;
    std::vector<int> cand;
    std::vector<int> phases;
  };
  const std::vector<Axis> axes = {
      {&ClassTune::col_threads, {64, 128, 256},
       {GFD_PHASE_ROW_FWD, GFD_PHASE_COL_FWD_LAMBDA, GFD_PHASE_LAMBDA_PASS, GFD_PHASE_COL_SOLVE_INV,
        GFD_PHASE_ROW_INV}},
      {&ClassTune::row_threads, {64, 128, 256},
       {GFD_PHASE_ROW_FWD, GFD_PHASE_COL_FWD_LAMBDA, GFD_PHASE_ROW_INV}},
      {&ClassTune::gf_rows, {16, 32, 64}, {GFD_PHASE_GUIDED_FILTER}}};
  for (const Axis& ax : axes) {
    std::vector<double> best(sizes.size(), 1e300);
    std::vector<int> pick(sizes.size(), 0);
    for (size_t ci = 0; ci < sizes.size(); ++ci) pick[ci] = cur.get(sizes[ci].first, sizes[ci].second).*(ax.field);
    for (int v : ax.cand) {
      for (const auto& sz : sizes) {
        ClassTune t = cur.get(sz.first, sz.second);
        t.*(ax.field) = v;
        cur.set(t);
      }
      std::vector<std::vector<double>> per;
      const cudaError_t e = measure(&per);
      if (e != cudaSuccess) return fail(e);
      for (size_t ci = 0; ci < sizes.size(); ++ci) {
        double ms = 0.0;
        for (int ph : ax.phases) ms += per[ci][ph];
        if (ms < best[ci]) {
          best[ci] = ms;
          pick[ci] = v;
        }
      }
    }
    for (size_t ci = 0; ci < sizes.size(); ++ci) {
      ClassTune t = cur.get(sizes[ci].first, sizes[ci].second);
      t.*(ax.field) = pick[ci];
      cur.set(t);
    }
  }
  // concurrent chains of the captured solve: graph replays timed on `s`
  if (c->opts.use_graphs) {
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaError_t e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    double best = 1e300;
    int pick = cur.chains;
    for (int q = 1; q <= CHAINS && e == cudaSuccess; ++q) {
      cur.chains = q;
      c->tune = cur;
      drop_plan(c);
      const int r = solve_batched_dev(c, n, imgs, iters, s);  // builds and captures
      if (r != GFD_OK) {
        e = g_last_cuda_error == cudaSuccess ? cudaErrorUnknown : g_last_cuda_error;
        break;
      }
      if ((e = cudaEventRecord(e0, s)) != cudaSuccess) break;
      for (int k = 0; k < 3 && e == cudaSuccess; ++k) e = cudaGraphLaunch(c->plan.exec, s);
      if (e == cudaSuccess) e = cudaEventRecord(e1, s);
      if (e == cudaSuccess) e = cudaEventSynchronize(e1);
      float ms = 0.0f;
      if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
      if (e == cudaSuccess && ms < best) {
        best = ms;
        pick = q;
      }
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (e != cudaSuccess) return fail(e);
    cur.chains = pick;
  }
  c->tune = cur;
  drop_plan(c);
  if (path && path[0] && !save_tune(path, cur)) return GFD_ERR_INVALID_ARG;
  return GFD_OK;
}

int gfdeconv_tune_read(const char* path, int* chains, int* n_classes, int* shapes,
                       int max_classes) {
  if (!path) return GFD_ERR_INVALID_ARG;
  TuneTable t;
  if (!load_tune(path, &t)) return GFD_ERR_INVALID_ARG;
  if (chains) *chains = t.chains;
  if (n_classes) *n_classes = (int)t.cls.size();
  for (int i = 0; shapes && i < max_classes && i < (int)t.cls.size(); ++i) {
    const ClassTune& c = t.cls[i];
    const int v[5] = {c.M, c.N, c.col_threads, c.row_threads, c.gf_rows};
    std::memcpy(shapes + 5 * i, v, sizeof v);
  }
  return GFD_OK;
}

int gfdeconv_tune_get(gfdeconv_ctx* c, int M, int N, int* col_threads, int* row_threads,
                      int* gf_rows, int* chains) {
  if (!c) return GFD_ERR_INVALID_ARG;
  const ClassTune t = c->tune.get(M, N);
  if (col_threads) *col_threads = t.col_threads;
  if (row_threads) *row_threads = t.row_threads;
  if (gf_rows) *gf_rows = t.gf_rows;
  if (chains) *chains = c->tune.chains;
  return GFD_OK;
}

int gfdeconv_solve_batched_timed(gfdeconv_ctx* c, int n, const gfdeconv_image* imgs, int iters,
                                 void* stream, double* phase_ms, long long* phase_launches) {
  if (!c || !imgs || n <= 0 || !phase_ms || !phase_launches) return GFD_ERR_INVALID_ARG;
  for (int i = 0; i < n; ++i) {
    int r = validate_image(imgs[i], iters);
    if (r == GFD_OK) r = validate_device_planes(imgs[i]);
    if (r != GFD_OK) return r;
  }
  if (cudaSetDevice(c->device) != cudaSuccess) return GFD_ERR_CUDA;
  cudaStream_t s = (cudaStream_t)stream;
  // plan as the graph path would (the cached graph, if any, stays valid)
  std::vector<unsigned char> key = make_key(c, n, imgs, iters);
  if (!(c->have_plan && c->plan.key == key)) {
    cudaError_t e = cudaDeviceSynchronize();
    if (e != cudaSuccess) return map_err(e);
    drop_plan(c);
    if ((e = build_plan(c, n, imgs, iters)) != cudaSuccess) {
      drop_plan(c);
      return map_err(e);
    }
    c->plan.key.swap(key);
    c->have_plan = true;
  }
  Timer tm;
  cudaError_t e = record(c, c->plan, s, &tm);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return map_err(e);
  for (size_t i = 0; i < tm.used; ++i) {
    float ms = 0.0f;
    if ((e = cudaEventElapsedTime(&ms, tm.ev[2 * i], tm.ev[2 * i + 1])) != cudaSuccess)
      return map_err(e);
    const int ph = tm.phase[i];
    if (ph >= 0 && ph < GFD_NUM_PHASES) {
      phase_ms[ph] += ms;
      phase_launches[ph] += 1;
    }
  }
  c->last_stream = s;
  c->last_launches = c->plan.launches;
  return GFD_OK;
}

int gfdeconv_backward_batched(gfdeconv_ctx* c, int n, const gfdeconv_image* imgs,
                              const gfdeconv_grad* grads, int iters, void* stream) {
  if (!c || !imgs || !grads || n <= 0 || iters < 1) return GFD_ERR_INVALID_ARG;
  if (c->opts.boundary != GFD_BOUNDARY_PERIODIC) return GFD_ERR_INVALID_ARG;
  const int M = imgs[0].M, N = imgs[0].N;
  int max_psf = 1;
  for (int i = 0; i < n; ++i) {
    int r = validate_image(imgs[i], iters);
    if (r == GFD_OK) r = validate_device_planes(imgs[i]);
    if (r != GFD_OK) return r;
    if (imgs[i].M != M || imgs[i].N != N || !imgs[i].u_iters || !imgs[i].lambda_out)
      return GFD_ERR_INVALID_ARG;
    const gfdeconv_grad& g = grads[i];
    if (!g.g_u || !g.g_y || !g.g_h || !g.g_eps || !aligned16(g.g_u) || !aligned16(g.g_y))
      return GFD_ERR_INVALID_ARG;
    max_psf = std::max(max_psf, imgs[i].kh * imgs[i].kw);
  }
  if (cudaSetDevice(c->device) != cudaSuccess) return GFD_ERR_CUDA;
  cudaStream_t s = (cudaStream_t)stream;
  const size_t P = (size_t)M * N;
  // per image: 17 real planes (16 of the adjoint, u_E^k) and 11 spectra (10
  // of the adjoint, the FFT scratch) of P floats each, 12 doubles (lambda,
  // g_eps, the sums)
  const int n_real = 17, n_spec = 11, n_dbl = 12;
  const size_t plane = align256(P * sizeof(float));
  const size_t per_img = (n_real + n_spec) * plane + align256(n_dbl * sizeof(double));
  const size_t descs_bytes = align256(sizeof(AdjDesc) * n);
  // ImgDesc arrays of the DFTs below: 11 of n entries, then 2 of 2n that
  // transform two planes of every image in one launch
  const int n_fft = 13;
  const size_t fft_bytes = align256(sizeof(ImgDesc) * 2 * n) * n_fft;
  const size_t need = per_img * n + descs_bytes + fft_bytes;
  cudaError_t e;
  if (need > c->adj_ws_bytes) {
    if ((e = cudaDeviceSynchronize()) != cudaSuccess) return map_err(e);
    if (c->adj_ws) cudaFree(c->adj_ws);
    c->adj_ws = nullptr;
    c->adj_ws_bytes = 0;
    if ((e = cudaMalloc(&c->adj_ws, need)) != cudaSuccess) return map_err(e);
    c->adj_ws_bytes = need;
  }
  char* cur = c->adj_ws;
  AdjDesc* d_desc = reinterpret_cast<AdjDesc*>(cur);
  cur += descs_bytes;
  ImgDesc* d_fft = reinterpret_cast<ImgDesc*>(cur);
  const size_t fft_stride = align256(sizeof(ImgDesc) * 2 * n) / sizeof(ImgDesc);
  cur += fft_bytes;
  std::vector<AdjDesc> ad(n);
  std::vector<float*> uEcur(n), hc(n), scratch(n);
  std::vector<std::vector<ImgDesc>> fd(n_fft, std::vector<ImgDesc>(n));
  for (int i = 0; i < n; ++i) {
    char* b = cur + per_img * i;
    auto realp = [&](int k) { return reinterpret_cast<float*>(b + plane * k); };
    auto specp = [&](int k) { return reinterpret_cast<float2*>(b + plane * (n_real + k)); };
    double* dbl = reinterpret_cast<double*>(b + plane * (n_real + n_spec));
    AdjDesc& a = ad[i];
    a = AdjDesc{};
    a.y = imgs[i].y;
    a.h = imgs[i].h;
    a.kh = imgs[i].kh;
    a.kw = imgs[i].kw;
    a.sigma = imgs[i].sigma;
    a.eps = imgs[i].eps;
    a.rho_fixed = c->opts.rho;
    float* uIp = realp(0);
    float* upp = realp(1);
    a.uI = uIp;
    a.up = upp;
    a.gu = realp(2);
    a.A = realp(3);
    a.MU = realp(4);
    a.PB = realp(5);
    a.VE = realp(6);
    a.GI0 = realp(7);
    a.GCOV = realp(8);
    a.GVAR = realp(9);
    a.GMU = realp(10);
    a.GPB = realp(11);
    a.guI = realp(12);
    a.gup = realp(13);
    a.gtmp = realp(14);
    a.gtmp2 = realp(15);
    uEcur[i] = realp(16);
    a.H = specp(0);
    a.Y = specp(1);
    a.UE = specp(2);
    a.UI = specp(3);
    a.Up = specp(4);
    a.GUI = specp(5);
    a.GUp = specp(6);
    a.gUE = specp(7);
    a.gH = specp(8);
    a.gY = specp(9);
    scratch[i] = reinterpret_cast<float*>(specp(10));
    hc[i] = a.gtmp2;  // the embedded PSF, transformed before gtmp2 is needed
    a.lam_hist = imgs[i].lambda_out;
    a.lam = dbl;
    a.g_eps = dbl + 1;
    a.acc = dbl + 2;  // ADJ_ACC (9) doubles
    a.g_eps_out = grads[i].g_eps;
    a.gy_out = grads[i].g_y;
    a.gh_out = grads[i].g_h;
    // DFT descriptors: r2c(src -> dst) uses u, S, Y; c2r(src -> dst) uses QI, uI
    auto r2c = [&](int op, const float* src, float2* dst, float2* rows) {
      ImgDesc& q = fd[op][i];
      q = ImgDesc{};
      q.u = const_cast<float*>(src);
      q.S = rows;  // the row pass's intermediate
      q.Y = dst;
    };
    float2* const scr = reinterpret_cast<float2*>(scratch[i]);
    auto c2r = [&](int op, float2* src, float* dst) {
      ImgDesc& q = fd[op][i];
      q = ImgDesc{};
      q.QI = src;
      q.uI = dst;
    };
    r2c(0, uEcur[i], a.UE, scr);
    c2r(1, a.UI, uIp);  // the recomputed step: U_I, U_p -> u_I, u_p
    c2r(2, a.Up, upp);
    // g_uI, g_up are transformed in one launch (op 12), each through its own
    // intermediate: the spectra U_I, U_p are free by then (the spectral
    // adjoint re-forms them from U_E)
    r2c(3, a.guI, a.GUI, a.UI);
    r2c(4, a.gup, a.GUp, a.Up);
    r2c(5, hc[i], a.H, scr);
    r2c(6, imgs[i].y, a.Y, scr);
    c2r(7, a.gUE, a.gtmp);
    c2r(8, a.gY, a.gtmp);
    c2r(9, a.gH, a.gtmp2);
    ImgDesc& q = fd[10][i];  // the PSF embedding writes q.uI
    q = ImgDesc{};
    q.h = imgs[i].h;
    q.kh = imgs[i].kh;
    q.kw = imgs[i].kw;
    q.uI = hc[i];
  }
  if ((e = cudaMemcpyAsync(d_desc, ad.data(), sizeof(AdjDesc) * n, cudaMemcpyHostToDevice, s)) !=
      cudaSuccess)
    return map_err(e);
  // paired transforms: u_I and u_p (inverse), g_uI and g_up (forward)
  fd[11] = fd[1];
  fd[11].insert(fd[11].end(), fd[2].begin(), fd[2].end());
  fd[12] = fd[3];
  fd[12].insert(fd[12].end(), fd[4].begin(), fd[4].end());
  for (int op = 0; op < n_fft; ++op)
    if ((e = cudaMemcpyAsync(d_fft + fft_stride * op, fd[op].data(), sizeof(ImgDesc) * fd[op].size(),
                             cudaMemcpyHostToDevice, s)) != cudaSuccess)
      return map_err(e);
  const Tables t{c->tw, c->d2, c->twdf};
  auto cls = [&](int op) {
    ClassLaunch cl{};
    cl.cd = ClassDesc{M, N, (int)fd[op].size(), 0, N / 2};
    cl.imgs = d_fft + fft_stride * op;
    cl.st = nullptr;
    return cl;
  };
  auto fwd = [&](int op) -> cudaError_t {
    const ClassLaunch cl = cls(op);
    cudaError_t r = launch_row_r2c(cl, t, SEL_U, SEL_S, false, s);
    if (r == cudaSuccess) r = launch_col_plain(cl, t, SEL_S, SEL_YS, false, s);
    return r;
  };
  // scale * F^H of a packed Hermitian spectrum (in place on the spectrum):
  // scale 1 is the adjoint DFT, 1/P the inverse
  auto adj = [&](int op, float scale) -> cudaError_t {
    const ClassLaunch cl = cls(op);
    cudaError_t r = launch_col_plain(cl, t, SEL_QI, SEL_QI, true, s);
    if (r == cudaSuccess) r = launch_row_c2r(cl, t, SEL_QI, -1, SEL_UI, -1, scale, s);
    return r;
  };
  const float invP = 1.0f / (float)P;
#define GFD_ADJ_CK(x)                    \
  do {                                   \
    if ((e = (x)) != cudaSuccess) return map_err(e); \
  } while (0)
  // setup: H, Y, the sums of Eq. 12; zeroed accumulators; g_u of u^K
  for (int i = 0; i < n; ++i) {
    GFD_ADJ_CK(cudaMemsetAsync(ad[i].gH, 0, P * sizeof(float), s));
    GFD_ADJ_CK(cudaMemsetAsync(ad[i].gY, 0, P * sizeof(float), s));
    GFD_ADJ_CK(cudaMemsetAsync(const_cast<double*>(ad[i].lam), 0, n_dbl * sizeof(double), s));
    GFD_ADJ_CK(cudaMemcpyAsync(ad[i].gu, grads[i].g_u, P * sizeof(float),
                               cudaMemcpyDeviceToDevice, s));
  }
  GFD_ADJ_CK(launch_embed_psf(cls(10), SEL_UI, s));
  GFD_ADJ_CK(fwd(5));
  GFD_ADJ_CK(fwd(6));
  GFD_ADJ_CK(launch_adj_stats(d_desc, n, M, N, s));
  // the steps, last first
  for (int k = iters - 1; k >= 0; --k) {
    // recompute the step from u_E^k and the forward's lambda_k: U_E, then
    // U_I, U_p (Eq. 8-9) and u_I, u_p
    for (int i = 0; i < n; ++i)
      GFD_ADJ_CK(cudaMemcpyAsync(uEcur[i], imgs[i].u_iters + (size_t)k * P, P * sizeof(float),
                                 cudaMemcpyDeviceToDevice, s));
    GFD_ADJ_CK(fwd(0));
    GFD_ADJ_CK(launch_adj_recompute(d_desc, n, M, N, k, c->d2, s));
    GFD_ADJ_CK(adj(11, invP));  // u_I and u_p
    for (int i0 = 0; i0 < n;) {  // guided-filter adjoint, one launch per run of equal w
      int i1 = i0 + 1;
      while (i1 < n && imgs[i1].w == imgs[i0].w) ++i1;
      GFD_ADJ_CK(launch_adj_guided_filter(d_desc + i0, i1 - i0, M, N, (imgs[i0].w - 1) / 2, s));
      i0 = i1;
    }
    GFD_ADJ_CK(fwd(12));  // G_UI and G_Up
    GFD_ADJ_CK(launch_adj_spectral(d_desc, n, M, N, c->d2, s));
    GFD_ADJ_CK(adj(7, 1.0f));
    GFD_ADJ_CK(launch_adj_next(d_desc, n, M, N, s));
  }
  GFD_ADJ_CK(adj(8, 1.0f));
  GFD_ADJ_CK(adj(9, 1.0f));
  GFD_ADJ_CK(launch_adj_final(d_desc, n, M, N, max_psf, s));
#undef GFD_ADJ_CK
  c->last_stream = s;
  return GFD_OK;
}

int gfdeconv_solve(gfdeconv_ctx* c, const float* y, int M, int N, const float* h, int kh, int kw,
                   double sigma, int w, double eps, int iters, float* u_out, double* lambda_out,
                   double* isnr_out, const float* u_orig, const float* u_init, void* stream) {
  gfdeconv_image im{};
  im.y = y;
  im.M = M;
  im.N = N;
  im.h = h;
  im.kh = kh;
  im.kw = kw;
  im.sigma = sigma;
  im.w = w;
  im.eps = eps;
  im.u_out = u_out;
  im.lambda_out = lambda_out;
  im.isnr_out = isnr_out;
  im.u_orig = u_orig;
  im.u_init = u_init;
  return gfdeconv_solve_batched(c, 1, &im, iters, stream);
}

int gfdeconv_solve_batched_host(gfdeconv_ctx* c, int n, const gfdeconv_image* imgs, int iters,
                                void* stream) {
  if (!c || !imgs || n <= 0) return GFD_ERR_INVALID_ARG;
  for (int i = 0; i < n; ++i) {
    const int r = validate_image(imgs[i], iters);
    if (r != GFD_OK) return r;
  }
  if (cudaSetDevice(c->device) != cudaSuccess) return GFD_ERR_CUDA;
  cudaStream_t s = (cudaStream_t)stream;
  // device staging, one area per field, images back to back in user order
  std::vector<size_t> off_y(n), off_h(n), off_uo(n), off_ui(n), off_u(n), off_l(n), off_is(n),
      off_r(n), off_I(n), off_p(n);
  size_t cur = 0;
  auto take = [&](size_t bytes) {
    const size_t o = cur;
    cur += align256(bytes);
    return o;
  };
  for (int i = 0; i < n; ++i) {
    const gfdeconv_image& im = imgs[i];
    const size_t P = (size_t)im.M * im.N * sizeof(float);
    off_y[i] = take(P);
    off_uo[i] = im.u_orig ? take(P) : 0;
    off_ui[i] = im.u_init ? take(P) : 0;
    off_u[i] = take(P);
    off_I[i] = im.uI_out ? take(P) : 0;
    off_p[i] = im.up_out ? take(P) : 0;
  }
  // the small arrays back to back: all PSFs, then lambda / ISNR / res of
  // each image in turn (each pack is one contiguous run on the device)
  for (int i = 0; i < n; ++i) {
    off_h[i] = cur;
    cur += (size_t)imgs[i].kh * imgs[i].kw * sizeof(float);
  }
  cur = align256(cur);
  const size_t itb = sizeof(double) * (size_t)std::max(iters, 1);
  for (int i = 0; i < n; ++i) {
    const gfdeconv_image& im = imgs[i];
    off_l[i] = im.lambda_out ? (cur += itb) - itb : 0;
    off_is[i] = im.isnr_out ? (cur += itb) - itb : 0;
    off_r[i] = im.res_out ? (cur += itb) - itb : 0;
  }
  cur = align256(cur);
  if (cur > c->stage_bytes) {
    cudaError_t e = cudaDeviceSynchronize();
    if (e != cudaSuccess) return map_err(e);
    if (c->stage) cudaFree(c->stage);
  if (c->adj_ws) cudaFree(c->adj_ws);
    c->stage = nullptr;
    c->stage_bytes = 0;
    if ((e = cudaMalloc(&c->stage, cur)) != cudaSuccess) return map_err(e);
    c->stage_bytes = cur;
  }
  char* base = c->stage;
  std::vector<gfdeconv_image> dev(imgs, imgs + n);
  // The PSFs (in) and the per-iteration lambda / ISNR / residual arrays (out)
  // are small: they travel packed, one copy each way through pinned host
  // staging, instead of one copy per image and field.
  size_t in_small = 0, out_small = 0;
  const size_t it = sizeof(double) * (size_t)iters;
  for (int i = 0; i < n; ++i) {
    in_small += (size_t)imgs[i].kh * imgs[i].kw * sizeof(float);
    out_small += it * ((imgs[i].lambda_out ? 1 : 0) + (imgs[i].isnr_out ? 1 : 0) + (imgs[i].res_out ? 1 : 0));
  }
  const size_t hneed = in_small + out_small;
  if (hneed > c->hstage_bytes) {
    if (c->hstage) cudaFreeHost(c->hstage);
    c->hstage = nullptr;
    c->hstage_bytes = 0;
    const cudaError_t e = cudaHostAlloc(&c->hstage, hneed, cudaHostAllocDefault);
    if (e != cudaSuccess) return map_err(e);
    c->hstage_bytes = hneed;
  }
  // device side of the packs: the h area and the lambda/ISNR/res areas of
  // the staging are laid out back to back (offsets from the layout above)
  struct Cp {
    char* dst;
    const char* src;
    size_t bytes;
  };
  std::vector<Cp> unpack;  // host pack -> user arrays
  // One copy per caller buffer: buffers that happen to be adjacent in host
  // memory may still be separate allocations, and one copy must not span two.
  auto add = [](std::vector<Cp>& v, char* dst, const char* src, size_t bytes) {
    v.push_back(Cp{dst, src, bytes});
  };
  // runs inside this library's own staging (both sides) are merged
  auto add_run = [](std::vector<Cp>& v, char* dst, const char* src, size_t bytes) {
    if (!v.empty() && v.back().dst + v.back().bytes == dst && v.back().src + v.back().bytes == src)
      v.back().bytes += bytes;
    else
      v.push_back(Cp{dst, src, bytes});
  };
  char* hin = c->hstage;
  char* hout = c->hstage + in_small;
  size_t pin = 0, pout = 0;
  std::vector<Cp> small_in_d, small_out_d;  // device areas of the packs, in pack order
  std::vector<std::vector<Cp>> h2d_img(n), d2h_img(n);  // per image (user order)
  std::vector<Cp> d2h_late;  // u_I, u_p: copied from the staging after the solve's last copies
  std::vector<Cp> init_in;   // u_init: copied before any of the solve's work
  for (int i = 0; i < n; ++i) {
    const gfdeconv_image& im = imgs[i];
    const size_t P = (size_t)im.M * im.N * sizeof(float);
    const size_t hb = (size_t)im.kh * im.kw * sizeof(float);
    dev[i].y = (const float*)(base + off_y[i]);
    add(h2d_img[i], base + off_y[i], (const char*)im.y, P);
    std::memcpy(hin + pin, im.h, hb);
    dev[i].h = (const float*)(base + off_h[i]);
    small_in_d.push_back(Cp{base + off_h[i], hin + pin, hb});
    pin += hb;
    if (im.u_orig) {
      dev[i].u_orig = (const float*)(base + off_uo[i]);
      add(h2d_img[i], base + off_uo[i], (const char*)im.u_orig, P);
    }
    if (im.u_init) {
      dev[i].u_init = (const float*)(base + off_ui[i]);
      // before the solve's first work: the start values are copied into u
      // ahead of every chain
      init_in.push_back(Cp{base + off_ui[i], (const char*)im.u_init, P});
    }
    dev[i].u_iters = nullptr;  // checkpoints are a device-buffer feature
    dev[i].u_out = (float*)(base + off_u[i]);
    add(d2h_img[i], (char*)im.u_out, base + off_u[i], P);
    double* const outs[3] = {im.lambda_out, im.isnr_out, im.res_out};
    const size_t offs[3] = {off_l[i], off_is[i], off_r[i]};
    double** const douts[3] = {&dev[i].lambda_out, &dev[i].isnr_out, &dev[i].res_out};
    for (int f = 0; f < 3; ++f) {
      if (!outs[f]) continue;
      *douts[f] = (double*)(base + offs[f]);
      if (it) {
        small_out_d.push_back(Cp{hout + pout, base + offs[f], it});
        unpack.push_back(Cp{(char*)outs[f], hout + pout, it});
        pout += it;
      }
    }
    if (im.uI_out) {
      dev[i].uI_out = (float*)(base + off_I[i]);
      add(d2h_late, (char*)im.uI_out, base + off_I[i], P);
    }
    if (im.up_out) {
      dev[i].up_out = (float*)(base + off_p[i]);
      add(d2h_late, (char*)im.up_out, base + off_p[i], P);
    }
  }
  // the device areas of each pack are consecutive in the staging layout
  // (h, then lambda / ISNR / res of each image), so each pack moves in runs
  std::vector<Cp> h2d_small, d2h_small;
  for (const Cp& cp : small_in_d) add_run(h2d_small, cp.dst, cp.src, cp.bytes);
  for (const Cp& cp : small_out_d) add_run(d2h_small, cp.dst, cp.src, cp.bytes);
  // With every caller buffer in page-locked memory the copies go into the
  // solve's graph: each chain of the solve copies its own images in and out,
  // overlapping the other chains' work.  Otherwise they run before and after.
  bool pinned = true;
  for (int i = 0; i < n && pinned; ++i) {
    const gfdeconv_image& im = imgs[i];
    const void* bufs[6] = {im.y, im.u_orig, im.u_init, im.u_out, im.uI_out, im.up_out};
    for (const void* b : bufs) {
      if (!b) continue;
      cudaPointerAttributes a{};
      if (cudaPointerGetAttributes(&a, b) != cudaSuccess || a.type != cudaMemoryTypeHost) {
        cudaGetLastError();
        pinned = false;
        break;
      }
    }
  }
  HostCopies hc;
  hc.in.resize(n);
  hc.out.resize(n);
  for (const Cp& cp : h2d_small) hc.pre.push_back(HostCopy{cp.dst, cp.src, cp.bytes, cudaMemcpyHostToDevice});
  for (const Cp& cp : init_in) hc.pre.push_back(HostCopy{cp.dst, cp.src, cp.bytes, cudaMemcpyHostToDevice});
  for (const Cp& cp : d2h_small) hc.post.push_back(HostCopy{cp.dst, cp.src, cp.bytes, cudaMemcpyDeviceToHost});
  for (int i = 0; i < n; ++i) {
    for (const Cp& cp : h2d_img[i]) hc.in[i].push_back(HostCopy{cp.dst, cp.src, cp.bytes, cudaMemcpyHostToDevice});
    for (const Cp& cp : d2h_img[i]) hc.out[i].push_back(HostCopy{cp.dst, cp.src, cp.bytes, cudaMemcpyDeviceToHost});
  }
  for (const Cp& cp : d2h_late) hc.post.push_back(HostCopy{cp.dst, cp.src, cp.bytes, cudaMemcpyDeviceToHost});
  if (pinned) {
    const int r = solve_batched_dev(c, n, dev.data(), iters, s, &hc);
    if (r != GFD_OK) return r;
  } else {
    auto run = [&](const std::vector<HostCopy>& v) -> cudaError_t {
      for (const HostCopy& cp : v) {
        const cudaError_t e = cudaMemcpyAsync(cp.dst, cp.src, cp.bytes, cp.kind, s);
        if (e != cudaSuccess) return e;
      }
      return cudaSuccess;
    };
    cudaError_t e = run(hc.pre);
    for (int i = 0; i < n && e == cudaSuccess; ++i) e = run(hc.in[i]);
    if (e != cudaSuccess) return map_err(e);
    const int r = solve_batched_dev(c, n, dev.data(), iters, s);
    if (r != GFD_OK) return r;
    for (int i = 0; i < n && e == cudaSuccess; ++i) e = run(hc.out[i]);
    if (e == cudaSuccess) e = run(hc.post);
    if (e != cudaSuccess) return map_err(e);
  }
  const cudaError_t e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return map_err(e);
  for (const Cp& cp : unpack) std::memcpy(cp.dst, cp.src, cp.bytes);
  return GFD_OK;
}

int gfdeconv_guidfilter(gfdeconv_ctx* c, const float* I, const float* p, int M, int N, int w,
                        double eps, float* u_out, void* stream) {
  if (!c || !I || !p || !u_out) return GFD_ERR_INVALID_ARG;
  if (!aligned16(I) || !aligned16(p) || !aligned16(u_out)) return GFD_ERR_INVALID_ARG;
  if (!pow2_in(M, 8, 4096) || !pow2_in(N, 8, 4096)) return GFD_ERR_UNSUPPORTED_SIZE;
  if (!std::isfinite(eps)) return GFD_ERR_NONFINITE_INPUT;
  if (!(eps > 0.0) || w < 1 || w > 17 || !(w & 1)) return GFD_ERR_INVALID_ARG;
  if (cudaSetDevice(c->device) != cudaSuccess) return GFD_ERR_CUDA;
  cudaStream_t s = (cudaStream_t)stream;
  AuxSlot* a = nullptr;
  cudaError_t e = aux_slot(c, 0, &a);
  if (e != cudaSuccess) return map_err(e);
  ImgDesc d{};
  d.uI = const_cast<float*>(I);
  d.up = const_cast<float*>(p);
  d.u = u_out;
  d.w = w;
  d.eps = eps;
  if ((e = aux_upload(a, d, s)) != cudaSuccess) return map_err(e);
  ClassLaunch cl{};
  cl.cd = ClassDesc{M, N, 1, 0, N / 2};
  cl.imgs = a->d_img;
  cl.st = c->aux_st;
  cl.max_rad = (w - 1) / 2;
  cl.n_rad_groups = 1;
  cl.rad_groups[0] = RadGroup{0, 1, (w - 1) / 2};
  if (c->opts.var_precision == GFD_VAR_COMPENSATED) {  // the split sums' bound
    if ((e = cudaMemsetAsync(c->aux_st->absmax, 0, sizeof(c->aux_st->absmax), s)) != cudaSuccess ||
        (e = launch_plane_absmax(cl, s)) != cudaSuccess)
      return map_err(e);
  }
  if ((e = launch_guided_filter(cl, -1, c->opts.var_precision, c->opts.boundary, s)) != cudaSuccess)
    return map_err(e);
  return map_err(aux_finish(a, s));
}

int gfdeconv_pad_symmetric(gfdeconv_ctx* c, const float* y, int m, int n, float* y_canvas, int M,
                           int N, void* stream) {
  if (!c || !y || !y_canvas) return GFD_ERR_INVALID_ARG;
  if (!pow2_in(M, 8, 4096) || !pow2_in(N, 8, 4096)) return GFD_ERR_UNSUPPORTED_SIZE;
  if (m < 1 || n < 1 || m > M || n > N) return GFD_ERR_INVALID_ARG;
  if (cudaSetDevice(c->device) != cudaSuccess) return GFD_ERR_CUDA;
  return map_err(launch_pad_symmetric(y, m, n, y_canvas, M, N, (cudaStream_t)stream));
}

int gfdeconv_crop(gfdeconv_ctx* c, const float* u_canvas, int M, int N, float* u, int m, int n,
                  void* stream) {
  if (!c || !u_canvas || !u) return GFD_ERR_INVALID_ARG;
  if (!pow2_in(M, 8, 4096) || !pow2_in(N, 8, 4096)) return GFD_ERR_UNSUPPORTED_SIZE;
  if (m < 1 || n < 1 || m > M || n > N) return GFD_ERR_INVALID_ARG;
  if (cudaSetDevice(c->device) != cudaSuccess) return GFD_ERR_CUDA;
  return map_err(launch_crop(u_canvas, N, u, m, n, (cudaStream_t)stream));
}

int gfdeconv_guidfilter_color(gfdeconv_ctx* c, const float* I, const float* p, int M, int N,
                              int w, double eps, float* u_out, void* stream) {
  if (!c || !I || !p || !u_out) return GFD_ERR_INVALID_ARG;
  if (!aligned16(I) || !aligned16(p) || !aligned16(u_out)) return GFD_ERR_INVALID_ARG;
  if (!pow2_in(M, 8, 4096) || !pow2_in(N, 8, 4096)) return GFD_ERR_UNSUPPORTED_SIZE;
  if (!std::isfinite(eps)) return GFD_ERR_NONFINITE_INPUT;
  if (!(eps > 0.0) || w < 1 || w > 17 || !(w & 1)) return GFD_ERR_INVALID_ARG;
  if (cudaSetDevice(c->device) != cudaSuccess) return GFD_ERR_CUDA;
  cudaStream_t s = (cudaStream_t)stream;
  AuxSlot* a = nullptr;
  cudaError_t e = aux_slot(c, (size_t)4 * M * N * sizeof(float), &a);
  if (e != cudaSuccess) return map_err(e);
  if ((e = launch_guided_filter_color(I, p, M, N, w, eps, c->opts.boundary,
                                      reinterpret_cast<float*>(a->ws), u_out, s)) != cudaSuccess)
    return map_err(e);
  return map_err(aux_finish(a, s));
}

int gfdeconv_fft2_r2c(gfdeconv_ctx* c, const float* x, int M, int N, float* X, void* stream) {
  if (!c || !x || !X) return GFD_ERR_INVALID_ARG;
  if (!aligned16(x) || !aligned16(X)) return GFD_ERR_INVALID_ARG;
  if (!pow2_in(M, 8, 4096) || !pow2_in(N, 8, 4096)) return GFD_ERR_UNSUPPORTED_SIZE;
  if (cudaSetDevice(c->device) != cudaSuccess) return GFD_ERR_CUDA;
  cudaStream_t s = (cudaStream_t)stream;
  const size_t P = (size_t)M * N;
  AuxSlot* a = nullptr;
  cudaError_t e = aux_slot(c, P * sizeof(float), &a);
  if (e != cudaSuccess) return map_err(e);
  ImgDesc d{};
  d.u = const_cast<float*>(x);
  d.S = reinterpret_cast<float2*>(a->ws);
  d.Y = reinterpret_cast<float2*>(X);
  if ((e = aux_upload(a, d, s)) != cudaSuccess) return map_err(e);
  ClassLaunch cl{};
  cl.cd = ClassDesc{M, N, 1, 0, N / 2};
  cl.imgs = a->d_img;
  cl.st = c->aux_st;
  const Tables t{c->tw, c->d2, c->twdf};
  if ((e = launch_row_r2c(cl, t, SEL_U, SEL_S, false, s)) != cudaSuccess) return map_err(e);
  if ((e = launch_col_plain(cl, t, SEL_S, SEL_YS, false, s)) != cudaSuccess) return map_err(e);
  return map_err(aux_finish(a, s));
}

int gfdeconv_fft2_c2r(gfdeconv_ctx* c, const float* X, int M, int N, float* x, void* stream) {
  if (!c || !x || !X) return GFD_ERR_INVALID_ARG;
  if (!aligned16(x) || !aligned16(X)) return GFD_ERR_INVALID_ARG;
  if (!pow2_in(M, 8, 4096) || !pow2_in(N, 8, 4096)) return GFD_ERR_UNSUPPORTED_SIZE;
  if (cudaSetDevice(c->device) != cudaSuccess) return GFD_ERR_CUDA;
  cudaStream_t s = (cudaStream_t)stream;
  const size_t P = (size_t)M * N;
  AuxSlot* a = nullptr;
  cudaError_t e = aux_slot(c, P * sizeof(float), &a);
  if (e != cudaSuccess) return map_err(e);
  ImgDesc d{};
  d.QI = reinterpret_cast<float2*>(a->ws);
  d.uI = x;
  if ((e = aux_upload(a, d, s)) != cudaSuccess) return map_err(e);
  if ((e = cudaMemcpyAsync(a->ws, X, P * sizeof(float), cudaMemcpyDeviceToDevice, s)) != cudaSuccess)
    return map_err(e);
  ClassLaunch cl{};
  cl.cd = ClassDesc{M, N, 1, 0, N / 2};
  cl.imgs = a->d_img;
  cl.st = c->aux_st;
  const Tables t{c->tw, c->d2, c->twdf};
  if ((e = launch_col_plain(cl, t, SEL_QI, SEL_QI, true, s)) != cudaSuccess) return map_err(e);
  if ((e = launch_row_c2r(cl, t, SEL_QI, -1, SEL_UI, -1, 1.0f / ((float)M * (float)N), s)) !=
      cudaSuccess)
    return map_err(e);
  return map_err(aux_finish(a, s));
}

int gfdeconv_status(gfdeconv_ctx* c, int* per_image_status, int n) {
  if (!c || !per_image_status || n < 0) return GFD_ERR_INVALID_ARG;
  if (!c->have_plan) return GFD_ERR_INVALID_ARG;
  if (n > c->plan.n) return GFD_ERR_INVALID_ARG;
  if (cudaSetDevice(c->device) != cudaSuccess) return GFD_ERR_CUDA;
  cudaError_t e = cudaStreamSynchronize(c->last_stream);
  if (e != cudaSuccess) return map_err(e);
  std::vector<ImgState> st(c->plan.n);
  e = cudaMemcpy(st.data(), c->d_st, sizeof(ImgState) * c->plan.n, cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return map_err(e);
  std::vector<int> by_user(c->plan.n, 0);
  for (int i = 0; i < c->plan.n; ++i) by_user[c->plan.order[i]] = st[i].status;
  for (int i = 0; i < n; ++i) per_image_status[i] = by_user[i];
  return GFD_OK;
}

long long gfdeconv_last_launch_count(gfdeconv_ctx* c) { return c ? c->last_launches : -1; }

const char* gfdeconv_last_cuda_error(void) {
  return g_last_cuda_error == cudaSuccess ? "no error" : cudaGetErrorString(g_last_cuda_error);
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Allocation-free 2-D real DFT (no counterpart in the paper).  The descriptor
// and the packed row-pass plane live in a static device array; the descriptor
// is written by a one-thread kernel from its by-value argument, so no host
// buffer is involved either.
namespace gfd {
namespace {

static_assert(sizeof(ImgDesc) <= 256, "descriptor slot");
static __device__ __align__(256) unsigned char g_noalloc_scratch[GFD_NOALLOC_SCRATCH_BYTES];

constexpr int NOALLOC_MAX_DEVICES = 64;
// Device address of g_noalloc_scratch per device (null until looked up).
// Atomic: host threads making their first call on a device at the same time
// both look the address up and store the same value.
std::atomic<void*> g_noalloc_addr[NOALLOC_MAX_DEVICES];

__global__ void k_store_desc(ImgDesc d, ImgDesc* dst) { *dst = d; }

}  // namespace
}  // namespace gfd

int gfdeconv_fft2_r2c_noalloc(gfdeconv_ctx* c, const float* x, int M, int N, float* X,
                              void* stream) {
  using namespace gfd;
  if (!c || !x || !X) return GFD_ERR_INVALID_ARG;
  if (!aligned16(x) || !aligned16(X)) return GFD_ERR_INVALID_ARG;
  if (!pow2_in(M, 8, 4096) || !pow2_in(N, 8, 4096)) return GFD_ERR_UNSUPPORTED_SIZE;
  if ((long long)M * N > GFD_NOALLOC_MAX_PIXELS) return GFD_ERR_SCRATCH_LIMIT;
  if (c->device < 0 || c->device >= NOALLOC_MAX_DEVICES) return GFD_ERR_INVALID_ARG;
  if (cudaSetDevice(c->device) != cudaSuccess) return GFD_ERR_CUDA;
  cudaError_t e;
  void* addr = g_noalloc_addr[c->device].load(std::memory_order_acquire);
  if (!addr) {
    if ((e = cudaGetSymbolAddress(&addr, g_noalloc_scratch)) != cudaSuccess) return map_err(e);
    g_noalloc_addr[c->device].store(addr, std::memory_order_release);
  }
  char* base = static_cast<char*>(addr);
  cudaStream_t s = (cudaStream_t)stream;
  ImgDesc d{};
  d.u = const_cast<float*>(x);
  d.S = reinterpret_cast<float2*>(base + 256);
  d.Y = reinterpret_cast<float2*>(X);
  ImgDesc* d_desc = reinterpret_cast<ImgDesc*>(base);
  k_store_desc<<<1, 1, 0, s>>>(d, d_desc);
  if ((e = cudaGetLastError()) != cudaSuccess) return map_err(e);
  ClassLaunch cl{};
  cl.cd = ClassDesc{M, N, 1, 0, N / 2};
  cl.imgs = d_desc;
  cl.st = nullptr;  // the plain passes keep no per-image state
  const Tables t{c->tw, c->d2, c->twdf};
  if ((e = launch_row_r2c(cl, t, SEL_U, SEL_S, false, s)) != cudaSuccess) return map_err(e);
  if ((e = launch_col_plain(cl, t, SEL_S, SEL_YS, false, s)) != cudaSuccess) return map_err(e);
  return GFD_OK;
}

int gfdeconv_device_arch(int cuda_device, int* binary_version, int* device_cc) {
  using namespace gfd;
  cudaError_t e = cudaSetDevice(cuda_device);
  if (e != cudaSuccess) return map_err(e);
  cudaFuncAttributes a{};
  if ((e = cudaFuncGetAttributes(&a, (const void*)k_store_desc)) != cudaSuccess) return map_err(e);
  int major = 0, minor = 0;
  if ((e = cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, cuda_device)) !=
          cudaSuccess ||
      (e = cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, cuda_device)) !=
          cudaSuccess)
    return map_err(e);
  if (binary_version) *binary_version = a.binaryVersion;
  if (device_cc) *device_cc = major * 10 + minor;
  return GFD_OK;
}
