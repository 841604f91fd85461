"""Guided-filter non-blind deconvolution (arXiv 1609.01839) on one GB300 GPU.

Thin ctypes binding over the C-ABI library ``libgfdeconv.so`` (declared in
``include/gfdeconv.h``).  This module only marshals arguments: every step of
the method runs in the library's CUDA kernels.  PyTorch supplies device
memory and the current CUDA stream.  There is no CPU fallback: importing the
binding without the built library, or passing CPU tensors where device
buffers are required, raises.
"""
from __future__ import annotations

import ctypes
import os
import re

__all__ = [
    "Context", "GfdError", "lib", "library_path", "header_functions",
    "STATUS_NONCONVERGED", "STATUS_NONFINITE", "STATUS_BAD_PSF", "STATUS_BAD_RHO",
    "STATUS_PASSES_EXHAUSTED", "STATUS_COPY_TIMEOUT", "VAR_COMPENSATED", "VAR_FP64", "VAR_FP32", "VAR_FP32_RAW",
    "VAR_DOUBLE_FLOAT",
    "BOUNDARY_PERIODIC", "BOUNDARY_TRUNCATED",
]

_HERE = os.path.dirname(os.path.abspath(__file__))
_ROOT = os.path.dirname(_HERE)
HEADER = os.path.join(_ROOT, "include", "gfdeconv.h")
library_path = os.path.join(_HERE, "libgfdeconv.so")

STATUS_NONCONVERGED = 1
STATUS_NONFINITE = 2
STATUS_BAD_PSF = 4
STATUS_BAD_RHO = 8
STATUS_PASSES_EXHAUSTED = 16
STATUS_COPY_TIMEOUT = 32
# window-statistics arithmetic of the guided filter (gfdeconv_opts.var_precision)
VAR_COMPENSATED = 0
VAR_FP64 = 1
VAR_FP32 = 2
VAR_FP32_RAW = 3
VAR_DOUBLE_FLOAT = 4
VAR_NAMES = {VAR_COMPENSATED: "compensated_split", VAR_FP64: "fp64", VAR_FP32: "fp32_shifted",
             VAR_FP32_RAW: "fp32_raw", VAR_DOUBLE_FLOAT: "double_float"}
# guided-filter window boundary (gfdeconv_opts.boundary)
BOUNDARY_PERIODIC = 0
BOUNDARY_TRUNCATED = 1
ERR_INVALID_ARG = -1    # argument errors, returned before any launch
ERR_SCRATCH_LIMIT = -8  # gfdeconv_fft2_r2c_noalloc: M*N above its static scratch
NUM_PHASES = 8
PHASES = ("setup", "row_fwd", "col_fwd_lambda", "lambda_pass", "col_solve_inv", "row_inv",
          "guided_filter", "copy")


def header_functions() -> list[str]:
    """Names of the functions declared in include/gfdeconv.h."""
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(gfdeconv_\w+)\s*\(", text)))


class GfdError(RuntimeError):
    def __init__(self, code: int, what: str = ""):
        msg = _lib.gfdeconv_strerror(code).decode() if _lib is not None else str(code)
        if _lib is not None and code in (-4, -5):
            msg += " [" + _lib.gfdeconv_last_cuda_error().decode() + "]"
        super().__init__(f"{what}: {msg} ({code})" if what else f"{msg} ({code})")
        self.code = code


class Image(ctypes.Structure):
    """Mirror of gfdeconv_image."""
    _fields_ = [
        ("y", ctypes.c_void_p), ("M", ctypes.c_int), ("N", ctypes.c_int),
        ("h", ctypes.c_void_p), ("kh", ctypes.c_int), ("kw", ctypes.c_int),
        ("sigma", ctypes.c_double), ("w", ctypes.c_int), ("eps", ctypes.c_double),
        ("u_out", ctypes.c_void_p), ("lambda_out", ctypes.c_void_p),
        ("isnr_out", ctypes.c_void_p), ("res_out", ctypes.c_void_p),
        ("u_orig", ctypes.c_void_p), ("u_init", ctypes.c_void_p),
        ("uI_out", ctypes.c_void_p), ("up_out", ctypes.c_void_p),
        ("u_iters", ctypes.c_void_p),
    ]


class Grad(ctypes.Structure):
    """Mirror of gfdeconv_grad."""
    _fields_ = [("g_u", ctypes.c_void_p), ("g_y", ctypes.c_void_p), ("g_h", ctypes.c_void_p),
                ("g_eps", ctypes.c_void_p)]


class Opts(ctypes.Structure):
    """Mirror of gfdeconv_opts."""
    _fields_ = [("var_precision", ctypes.c_int), ("rho", ctypes.c_double),
                ("use_graphs", ctypes.c_int), ("lambda_max_passes", ctypes.c_int),
                ("lambda_rtol", ctypes.c_double), ("boundary", ctypes.c_int),
                ("tune_cache", ctypes.c_char_p)]


def _load():
    if not os.path.exists(library_path):
        raise ImportError(
            f"{library_path} is missing: build it with "
            "`python -c 'import __graft_entry__ as g; g.build()'` (needs nvcc)")
    L = ctypes.CDLL(library_path)
    vp, ci, cd = ctypes.c_void_p, ctypes.c_int, ctypes.c_double
    sigs = {
        "gfdeconv_create": (ci, [ctypes.POINTER(vp), ci, ctypes.POINTER(Opts)]),
        "gfdeconv_destroy": (None, [vp]),
        "gfdeconv_solve": (ci, [vp, vp, ci, ci, vp, ci, ci, cd, ci, cd, ci, vp, vp, vp, vp, vp, vp]),
        "gfdeconv_solve_batched": (ci, [vp, ci, ctypes.POINTER(Image), ci, vp]),
        "gfdeconv_solve_batched_host": (ci, [vp, ci, ctypes.POINTER(Image), ci, vp]),
        "gfdeconv_guidfilter": (ci, [vp, vp, vp, ci, ci, ci, cd, vp, vp]),
        "gfdeconv_guidfilter_color": (ci, [vp, vp, vp, ci, ci, ci, cd, vp, vp]),
        "gfdeconv_pad_symmetric": (ci, [vp, vp, ci, ci, vp, ci, ci, vp]),
        "gfdeconv_crop": (ci, [vp, vp, ci, ci, vp, ci, ci, vp]),
        "gfdeconv_fft2_r2c": (ci, [vp, vp, ci, ci, vp, vp]),
        "gfdeconv_fft2_c2r": (ci, [vp, vp, ci, ci, vp, vp]),
        "gfdeconv_fft2_r2c_noalloc": (ci, [vp, vp, ci, ci, vp, vp]),
        "gfdeconv_solve_batched_timed": (ci, [vp, ci, ctypes.POINTER(Image), ci, vp,
                                              ctypes.POINTER(cd), ctypes.POINTER(ctypes.c_longlong)]),
        "gfdeconv_status": (ci, [vp, ctypes.POINTER(ci), ci]),
        "gfdeconv_last_launch_count": (ctypes.c_longlong, [vp]),
        "gfdeconv_strerror": (ctypes.c_char_p, [ci]),
        "gfdeconv_last_cuda_error": (ctypes.c_char_p, []),
        "gfdeconv_device_arch": (ci, [ci, ctypes.POINTER(ci), ctypes.POINTER(ci)]),
        "gfdeconv_autotune": (ci, [vp, ci, ctypes.POINTER(Image), ci, ctypes.c_char_p, vp]),
        "gfdeconv_backward_batched": (ci, [vp, ci, ctypes.POINTER(Image), ctypes.POINTER(Grad), ci,
                                           vp]),
        "gfdeconv_tune_read": (ci, [ctypes.c_char_p, ctypes.POINTER(ci), ctypes.POINTER(ci),
                                    ctypes.POINTER(ci), ci]),
        "gfdeconv_tune_get": (ci, [vp, ci, ci, ctypes.POINTER(ci), ctypes.POINTER(ci),
                                   ctypes.POINTER(ci), ctypes.POINTER(ci)]),
    }
    for name, (res, args) in sigs.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args
    return L


_lib = _load()
lib = _lib


def tune_read(path: str):
    """Contents of a tile-shape file (host only): (chains, {(M, N):
    (col_threads, row_threads, gf_rows)})."""
    ch, n = ctypes.c_int(0), ctypes.c_int(0)
    rc = _lib.gfdeconv_tune_read(path.encode(), ctypes.byref(ch), ctypes.byref(n), None, 0)
    if rc != 0:
        raise GfdError(rc, "gfdeconv_tune_read")
    buf = (ctypes.c_int * (5 * max(n.value, 1)))()
    rc = _lib.gfdeconv_tune_read(path.encode(), ctypes.byref(ch), ctypes.byref(n), buf, n.value)
    if rc != 0:
        raise GfdError(rc, "gfdeconv_tune_read")
    return ch.value, {(buf[5 * i], buf[5 * i + 1]): tuple(buf[5 * i + 2:5 * i + 5])
                      for i in range(n.value)}


def device_arch(device: int = 0) -> tuple[int, int]:
    """(compute capability the library's kernels were built for, as loaded on
    `device`; the device's compute capability), each major * 10 + minor."""
    b, d = ctypes.c_int(0), ctypes.c_int(0)
    rc = _lib.gfdeconv_device_arch(int(device), ctypes.byref(b), ctypes.byref(d))
    if rc != 0:
        raise GfdError(rc, "gfdeconv_device_arch")
    return b.value, d.value


def _ptr(t, what, dtype=None, numel=None):
    import torch
    if t is None:
        return None
    if not isinstance(t, torch.Tensor):
        raise TypeError(f"{what} must be a torch.Tensor")
    if not t.is_cuda:
        raise ValueError(f"{what} must be a CUDA tensor (there is no CPU path)")
    if not t.is_contiguous():
        raise ValueError(f"{what} must be contiguous")
    if dtype is not None and t.dtype != dtype:
        raise TypeError(f"{what} must be {dtype}, got {t.dtype}")
    if numel is not None and t.numel() != numel:
        raise ValueError(f"{what} must have {numel} elements, got {t.numel()}")
    return t.data_ptr()


def _hptr(t, what, dtype=None, numel=None):
    import torch
    if t is None:
        return None
    if not isinstance(t, torch.Tensor) or t.is_cuda or not t.is_contiguous():
        raise ValueError(f"{what} must be a contiguous host (CPU) tensor")
    if dtype is not None and t.dtype != dtype:
        raise TypeError(f"{what} must be {dtype}, got {t.dtype}")
    if numel is not None and t.numel() != numel:
        raise ValueError(f"{what} must have {numel} elements")
    return t.data_ptr()


def _stream(stream):
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


class Context:
    """A library context on one CUDA device (owns workspaces and cached
    CUDA graphs).  Not thread-safe."""

    def __init__(self, device: int = 0, var_precision: int = VAR_COMPENSATED, rho: float = 0.0,
                 use_graphs: bool = True, lambda_max_passes: int = 0, lambda_rtol: float = 0.0,
                 boundary: int = BOUNDARY_PERIODIC, tune_cache: str | None = None):
        import torch
        torch.cuda.init()
        self.device = device
        self._h = ctypes.c_void_p()
        opts = Opts(int(var_precision), float(rho), 1 if use_graphs else 0, int(lambda_max_passes),
                    float(lambda_rtol), int(boundary),
                    tune_cache.encode() if tune_cache else None)
        with torch.cuda.device(device):
            rc = _lib.gfdeconv_create(ctypes.byref(self._h), device, ctypes.byref(opts))
        if rc != 0:
            raise GfdError(rc, "gfdeconv_create")

    def close(self):
        if self._h:
            _lib.gfdeconv_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    # -- entry points --------------------------------------------------------
    def solve(self, y, h, sigma, w, eps, iters, u_orig=None, u_init=None, stream=None,
              with_lambda=True, u_out=None):
        """One image: returns (u, lambda[iters] float64, isnr[iters] or None)."""
        import torch
        M, N = y.shape
        kh, kw = h.shape
        u = torch.empty((M, N), dtype=torch.float32, device=y.device) if u_out is None else u_out
        lam = torch.empty(max(iters, 1), dtype=torch.float64, device=y.device) if with_lambda else None
        isnr = (torch.empty(max(iters, 1), dtype=torch.float64, device=y.device)
                if u_orig is not None else None)
        rc = _lib.gfdeconv_solve(
            self._h, _ptr(y, "y", torch.float32), M, N, _ptr(h, "h", torch.float32), kh, kw,
            float(sigma), int(w), float(eps), int(iters), _ptr(u, "u_out", torch.float32, M * N),
            _ptr(lam, "lambda"), _ptr(isnr, "isnr"), _ptr(u_orig, "u_orig", torch.float32, M * N),
            _ptr(u_init, "u_init", torch.float32, M * N), _stream(stream))
        if rc != 0:
            raise GfdError(rc, "gfdeconv_solve")
        return u, lam, isnr

    def make_images(self, items, iters, want_res=False, want_uIp=False, want_checkpoints=False):
        """Descriptors for solve_batched from dicts with CUDA tensors
        y, h, sigma, w, eps and optional u_orig, u_init.  Allocates u (and
        lambda / isnr / res / u_I / u_p / the per-iteration checkpoints
        u_iters) and stores them in each dict."""
        import torch
        arr = (Image * len(items))()
        for i, it in enumerate(items):
            y, h = it["y"], it["h"]
            M, N = y.shape
            dev = y.device
            it["u"] = it.get("u") if it.get("u") is not None else torch.empty((M, N), dtype=torch.float32, device=dev)
            it["lam"] = torch.empty(max(iters, 1), dtype=torch.float64, device=dev)
            it["isnr"] = (torch.empty(max(iters, 1), dtype=torch.float64, device=dev)
                          if it.get("u_orig") is not None else None)
            it["res"] = torch.empty(max(iters, 1), dtype=torch.float64, device=dev) if want_res else None
            if want_uIp:
                it["uI"] = torch.empty((M, N), dtype=torch.float32, device=dev)
                it["up"] = torch.empty((M, N), dtype=torch.float32, device=dev)
            if want_checkpoints:
                it["u_iters"] = torch.empty((max(iters, 1), M, N), dtype=torch.float32, device=dev)
            a = arr[i]
            a.y = _ptr(y, "y", torch.float32)
            a.M, a.N = M, N
            a.h = _ptr(h, "h", torch.float32)
            a.kh, a.kw = h.shape
            a.sigma = float(it["sigma"])
            a.w = int(it["w"])
            a.eps = float(it["eps"])
            a.u_out = _ptr(it["u"], "u", torch.float32, M * N)
            a.lambda_out = _ptr(it["lam"], "lambda")
            a.isnr_out = _ptr(it["isnr"], "isnr")
            a.res_out = _ptr(it["res"], "res")
            a.u_orig = _ptr(it.get("u_orig"), "u_orig", torch.float32, M * N)
            a.u_init = _ptr(it.get("u_init"), "u_init", torch.float32, M * N)
            a.uI_out = _ptr(it.get("uI"), "uI", torch.float32, M * N)
            a.up_out = _ptr(it.get("up"), "up", torch.float32, M * N)
            a.u_iters = _ptr(it.get("u_iters"), "u_iters", torch.float32)
        return arr

    def solve_batched_images(self, arr, iters, stream=None):
        rc = _lib.gfdeconv_solve_batched(self._h, len(arr), arr, int(iters), _stream(stream))
        if rc != 0:
            raise GfdError(rc, "gfdeconv_solve_batched")

    def solve_batched(self, items, iters, stream=None, want_res=False, want_uIp=False,
                      want_checkpoints=False):
        """Batched solve of dicts (see make_images); results land in the dicts."""
        arr = self.make_images(items, iters, want_res, want_uIp, want_checkpoints)
        self.solve_batched_images(arr, iters, stream)
        return items

    def backward_batched(self, items, iters, g_us, stream=None):
        """gfdeconv_backward_batched: items are the dicts of a solve_batched
        call made with want_checkpoints=True, g_us the gradients dL/du of their
        results.  Returns [(g_y, g_h, g_eps)] (CUDA tensors; g_eps float64)."""
        import torch
        arr = (Image * len(items))()
        grads = (Grad * len(items))()
        out = []
        for i, (it, gu) in enumerate(zip(items, g_us)):
            y, h = it["y"], it["h"]
            M, N = y.shape
            a = arr[i]
            a.y = _ptr(y, "y", torch.float32)
            a.M, a.N = M, N
            a.h = _ptr(h, "h", torch.float32)
            a.kh, a.kw = h.shape
            a.sigma, a.w, a.eps = float(it["sigma"]), int(it["w"]), float(it["eps"])
            a.u_out = _ptr(it["u"], "u", torch.float32, M * N)
            a.u_iters = _ptr(it["u_iters"], "u_iters", torch.float32)
            a.lambda_out = _ptr(it["lam"], "lambda")
            gy = torch.empty_like(y)
            gh = torch.empty_like(h)
            ge = torch.empty((), dtype=torch.float64, device=y.device)
            g = grads[i]
            g.g_u = _ptr(gu, "g_u", torch.float32, M * N)
            g.g_y, g.g_h, g.g_eps = gy.data_ptr(), gh.data_ptr(), ge.data_ptr()
            out.append((gy, gh, ge))
        rc = _lib.gfdeconv_backward_batched(self._h, len(items), arr, grads, int(iters),
                                            _stream(stream))
        if rc != 0:
            raise GfdError(rc, "gfdeconv_backward_batched")
        return out

    def deconv(self, y, h, eps, sigma, w, iters, stream=None):
        """Differentiable solve: u^iters of a batch (y: (B, M, N) or (M, N);
        h: (B, kh, kw) or (kh, kw); eps: a tensor of B values or one value;
        sigma: a float or B floats; w one odd window).  Gradients with respect
        to y, h and eps come from gfdeconv_backward_batched (the library's
        hand-written adjoint), through torch.autograd."""
        return _Deconv.apply(y, h, eps, self, sigma, int(w), int(iters), stream)


    def make_host_images(self, items, iters):
        """Descriptors for solve_batched_host from dicts of pinned CPU tensors
        y, h (+ u_orig, u_init); allocates pinned outputs u, lam, isnr in the dicts."""
        import torch
        arr = (Image * len(items))()
        for i, it in enumerate(items):
            y, h = it["y"], it["h"]
            M, N = y.shape
            if it.get("u") is None:
                it["u"] = torch.empty((M, N), dtype=torch.float32).pin_memory()
            it["lam"] = torch.empty(max(iters, 1), dtype=torch.float64).pin_memory()
            it["isnr"] = (torch.empty(max(iters, 1), dtype=torch.float64).pin_memory()
                          if it.get("u_orig") is not None else None)
            a = arr[i]
            a.y = _hptr(y, "y", torch.float32)
            a.M, a.N = M, N
            a.h = _hptr(h, "h", torch.float32)
            a.kh, a.kw = h.shape
            a.sigma = float(it["sigma"])
            a.w = int(it["w"])
            a.eps = float(it["eps"])
            a.u_out = _hptr(it["u"], "u", torch.float32)
            a.lambda_out = _hptr(it["lam"], "lambda")
            a.isnr_out = _hptr(it["isnr"], "isnr")
            a.u_orig = _hptr(it.get("u_orig"), "u_orig", torch.float32)
            a.u_init = _hptr(it.get("u_init"), "u_init", torch.float32)
        return arr

    def solve_batched_timed(self, arr, iters, stream=None):
        """Direct-launch solve with an event pair around every launch; returns
        (phase_ms[8], phase_launches[8]) summed over the solve."""
        ms = (ctypes.c_double * NUM_PHASES)()
        nl = (ctypes.c_longlong * NUM_PHASES)()
        rc = _lib.gfdeconv_solve_batched_timed(self._h, len(arr), arr, int(iters), _stream(stream),
                                               ms, nl)
        if rc != 0:
            raise GfdError(rc, "gfdeconv_solve_batched_timed")
        return list(ms), list(nl)

    def solve_batched_host_images(self, arr, iters, stream=None):
        rc = _lib.gfdeconv_solve_batched_host(self._h, len(arr), arr, int(iters), _stream(stream))
        if rc != 0:
            raise GfdError(rc, "gfdeconv_solve_batched_host")

    def guidfilter(self, I, p, w, eps, stream=None, out=None):
        import torch
        M, N = I.shape
        u = torch.empty_like(I) if out is None else out
        rc = _lib.gfdeconv_guidfilter(self._h, _ptr(I, "I", torch.float32), _ptr(p, "p", torch.float32, M * N),
                                      M, N, int(w), float(eps), _ptr(u, "u", torch.float32, M * N),
                                      _stream(stream))
        if rc != 0:
            raise GfdError(rc, "gfdeconv_guidfilter")
        return u

    def pad_symmetric(self, y, M, N, stream=None):
        """(m, n) CUDA tensor -> (M, N) canvas by symmetric reflection."""
        import torch
        m, n = y.shape
        out = torch.empty((M, N), dtype=torch.float32, device=y.device)
        rc = _lib.gfdeconv_pad_symmetric(self._h, _ptr(y, "y", torch.float32), m, n,
                                         out.data_ptr(), int(M), int(N), _stream(stream))
        if rc != 0:
            raise GfdError(rc, "gfdeconv_pad_symmetric")
        return out

    def crop(self, u_canvas, m, n, stream=None):
        import torch
        M, N = u_canvas.shape
        out = torch.empty((m, n), dtype=torch.float32, device=u_canvas.device)
        rc = _lib.gfdeconv_crop(self._h, _ptr(u_canvas, "u_canvas", torch.float32), M, N,
                                out.data_ptr(), int(m), int(n), _stream(stream))
        if rc != 0:
            raise GfdError(rc, "gfdeconv_crop")
        return out

    def solve_padded(self, y, h, sigma, w, eps, iters, stream=None):
        """An observation of any size up to 4096 x 4096: padded to the next
        power-of-two canvas (gfdeconv_pad_symmetric), solved there, cropped
        back.  Returns (u (m, n), lambda[iters])."""
        m, n = y.shape
        M, N = 1 << max(3, (m - 1).bit_length()), 1 << max(3, (n - 1).bit_length())
        yc = self.pad_symmetric(y, M, N, stream)
        uc, lam, _ = self.solve(yc, h, sigma, w, eps, iters, stream=stream)
        return self.crop(uc, m, n, stream), lam

    def guidfilter_color(self, I, p, w, eps, stream=None, out=None):
        """Colour guidance: I is a (3, M, N) float32 CUDA tensor, p (M, N)."""
        import torch
        C, M, N = I.shape
        if C != 3:
            raise ValueError("I must have 3 channels (3, M, N)")
        u = torch.empty((M, N), dtype=torch.float32, device=p.device) if out is None else out
        rc = _lib.gfdeconv_guidfilter_color(self._h, _ptr(I, "I", torch.float32),
                                            _ptr(p, "p", torch.float32, M * N), M, N, int(w),
                                            float(eps), _ptr(u, "u", torch.float32, M * N),
                                            _stream(stream))
        if rc != 0:
            raise GfdError(rc, "gfdeconv_guidfilter_color")
        return u

    def fft2_r2c(self, x, stream=None):
        """Packed half spectrum as a complex64 (M, N/2) tensor."""
        import torch
        M, N = x.shape
        X = torch.empty((M, N // 2), dtype=torch.complex64, device=x.device)
        rc = _lib.gfdeconv_fft2_r2c(self._h, _ptr(x, "x", torch.float32), M, N, X.data_ptr(),
                                    _stream(stream))
        if rc != 0:
            raise GfdError(rc, "gfdeconv_fft2_r2c")
        return X

    def fft2_r2c_noalloc(self, x, X, stream=None):
        """gfdeconv_fft2_r2c_noalloc into the caller's complex64 (M, N/2)
        tensor X (the library allocates nothing; M*N <= 1024*1024)."""
        import torch
        M, N = x.shape
        rc = _lib.gfdeconv_fft2_r2c_noalloc(self._h, _ptr(x, "x", torch.float32), M, N,
                                            _ptr(X, "X", torch.complex64, M * (N // 2)),
                                            _stream(stream))
        if rc != 0:
            raise GfdError(rc, "gfdeconv_fft2_r2c_noalloc")
        return X

    def fft2_c2r(self, X, stream=None):
        import torch
        M, L = X.shape
        x = torch.empty((M, 2 * L), dtype=torch.float32, device=X.device)
        rc = _lib.gfdeconv_fft2_c2r(self._h, _ptr(X, "X", torch.complex64), M, 2 * L, x.data_ptr(),
                                    _stream(stream))
        if rc != 0:
            raise GfdError(rc, "gfdeconv_fft2_c2r")
        return x

    def autotune(self, arr, iters, path=None, stream=None):
        """gfdeconv_autotune over the descriptors `arr` (see make_images)."""
        rc = _lib.gfdeconv_autotune(self._h, len(arr), arr, int(iters),
                                    path.encode() if path else None, _stream(stream))
        if rc != 0:
            raise GfdError(rc, "gfdeconv_autotune")

    def tune_get(self, M, N):
        """(col_threads, row_threads, gf_rows, chains) used for an M x N canvas."""
        v = [ctypes.c_int(0) for _ in range(4)]
        rc = _lib.gfdeconv_tune_get(self._h, int(M), int(N), *[ctypes.byref(x) for x in v])
        if rc != 0:
            raise GfdError(rc, "gfdeconv_tune_get")
        return tuple(x.value for x in v)

    def status(self, n):
        arr = (ctypes.c_int * n)()
        rc = _lib.gfdeconv_status(self._h, arr, n)
        if rc != 0:
            raise GfdError(rc, "gfdeconv_status")
        return list(arr)

    def last_launch_count(self) -> int:
        return int(_lib.gfdeconv_last_launch_count(self._h))


def _autograd_function():
    import torch

    class Deconv(torch.autograd.Function):
        @staticmethod
        def forward(fctx, y, h, eps, lib, sigma, w, iters, stream):
            single = y.dim() == 2
            Y = y.detach().reshape((-1,) + tuple(y.shape[-2:])).contiguous().float()
            Hh = h.detach().reshape((-1,) + tuple(h.shape[-2:])).contiguous().float()
            B = Y.shape[0]
            if Hh.shape[0] == 1 and B > 1:
                Hh = Hh.expand(B, -1, -1).contiguous()
            E = torch.as_tensor(eps, dtype=torch.float64).reshape(-1)
            if E.numel() == 1 and B > 1:
                E = E.expand(B)
            sig = [float(sigma)] * B if not hasattr(sigma, "__len__") else [float(s) for s in sigma]
            items = [{"y": Y[b], "h": Hh[b], "sigma": sig[b], "w": w, "eps": float(E[b])}
                     for b in range(B)]
            lib.solve_batched(items, iters, stream=stream, want_checkpoints=True)
            fctx.lib, fctx.items, fctx.iters, fctx.stream = lib, items, iters, stream
            fctx.shapes = (y.shape, h.shape, torch.as_tensor(eps).shape, single, Hh.shape[0] != h.reshape((-1,) + tuple(h.shape[-2:])).shape[0])
            fctx.eps_dtype = torch.as_tensor(eps).dtype
            u = torch.stack([it["u"] for it in items])
            return u[0] if single else u

        @staticmethod
        def backward(fctx, g_u):
            import torch as T
            G = g_u.reshape((-1,) + tuple(g_u.shape[-2:])).contiguous().float()
            res = fctx.lib.backward_batched(fctx.items, fctx.iters, [G[b] for b in range(G.shape[0])],
                                            fctx.stream)
            y_shape, h_shape, e_shape, single, h_expanded = fctx.shapes
            gy = T.stack([r[0] for r in res]).reshape(y_shape)
            gh = T.stack([r[1] for r in res])
            gh = gh.sum(0) if h_expanded else gh
            gh = gh.reshape(h_shape)
            ge = T.stack([r[2] for r in res])
            ge = (ge.sum() if len(e_shape) == 0 or T.Size(e_shape).numel() == 1 else ge).reshape(e_shape)
            return gy, gh, ge.to(fctx.eps_dtype), None, None, None, None, None

    return Deconv


class _LazyDeconv:
    fn = None

    @classmethod
    def apply(cls, *args):
        if cls.fn is None:
            cls.fn = _autograd_function()
        return cls.fn.apply(*args)


_Deconv = _LazyDeconv
