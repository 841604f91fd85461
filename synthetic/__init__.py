"""Seeded synthetic inputs for the guided-filter deconvolution workloads.

This module only *makes inputs*: clean images, point-spread functions and the
degraded observation of the paper's forward model y = h*u_orig + gamma
(Sec. 1, Eq. 1: circular convolution plus i.i.d. zero-mean Gaussian noise of
variance sigma^2).  It holds none of the deconvolution method's arithmetic
(no spectral solve, no guided filter, no regularisation-parameter choice), so
both the FP64 oracle and the GPU path may consume it.

Every array handed to a solver is rounded to float32 exactly once here, so the
oracle (which promotes to float64) and the GPU see identical bits.

The paper's test images (Cameraman, House; Sec. 4) are not available, so the
workloads below are synthetic stand-ins with the structure the configurations
describe: piecewise-constant or piecewise-smooth content with hard edges.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

__all__ = [
    "Problem", "pixel_grid", "image_rects_disks", "image_polygons",
    "psf_uniform", "psf_inv_quadratic", "psf_gaussian", "psf_binomial5",
    "psf_motion", "blur_circular", "sigma_from_bsnr", "mirror_extend",
    "config_c0", "config_c1", "config_c2_image", "config_c2", "config_c4",
    "config_c4_image", "config_table1", "config_c3_image", "table1_psf", "next_pow2",
]


# ----------------------------------------------------------------------------
# images
# ----------------------------------------------------------------------------

def pixel_grid(M: int, N: int, lo: float, hi: float):
    """Pixel-centre coordinates (row-major): returns (x, y), each M x N,
    mapped so that the canvas spans [lo, hi] in both axes."""
    xs = lo + (hi - lo) * (np.arange(N) + 0.5) / N
    ys = lo + (hi - lo) * (np.arange(M) + 0.5) / M
    return np.meshgrid(xs, ys)


def image_rects_disks(seed: int, M: int = 256, N: int = 256,
                      n_rect: int = 20, n_disk: int = 10) -> np.ndarray:
    """Piecewise-constant test image: a linear-gradient background
    g0 + gx*x + gy*y (x, y in [0, 1]; g0 ~ U[0.2, 0.6], gx, gy ~ U[-0.2, 0.2]),
    then ``n_rect`` axis-aligned rectangles (sides U[8, 96] px) and ``n_disk``
    disks (radius U[4, 40] px), each with an intensity ~ U[0, 1], painted in
    that order with hard edges and pixel-centre sampling.  float64."""
    rng = np.random.default_rng(seed)
    g0 = rng.uniform(0.2, 0.6)
    gx, gy = rng.uniform(-0.2, 0.2, size=2)
    x, y = pixel_grid(M, N, 0.0, 1.0)
    u = g0 + gx * x + gy * y
    for _ in range(n_rect):
        h = int(rng.integers(8, 97))
        w = int(rng.integers(8, 97))
        top = int(rng.integers(0, max(1, M - h + 1)))
        left = int(rng.integers(0, max(1, N - w + 1)))
        u[top:top + h, left:left + w] = rng.uniform(0.0, 1.0)
    ii, jj = np.meshgrid(np.arange(M) + 0.5, np.arange(N) + 0.5, indexing="ij")
    for _ in range(n_disk):
        rad = rng.uniform(4.0, 40.0)
        cy = rng.uniform(0.0, M)
        cx = rng.uniform(0.0, N)
        val = rng.uniform(0.0, 1.0)
        u[(ii - cy) ** 2 + (jj - cx) ** 2 <= rad * rad] = val
    return u


def _inside_polygon(px: np.ndarray, py: np.ndarray, vx: np.ndarray,
                    vy: np.ndarray) -> np.ndarray:
    """Even-odd ray-casting point-in-polygon test, vectorised over points."""
    inside = np.zeros(px.shape, dtype=bool)
    n = len(vx)
    for k in range(n):
        x1, y1 = vx[k], vy[k]
        x2, y2 = vx[(k + 1) % n], vy[(k + 1) % n]
        if y1 == y2:
            continue
        crosses = (y1 > py) != (y2 > py)
        xint = x1 + (py - y1) * (x2 - x1) / (y2 - y1)
        inside ^= crosses & (px < xint)
    return inside


def _gaussian_lowpass_periodic(a: np.ndarray, sigma_px: float) -> np.ndarray:
    """Periodic Gaussian low-pass of a field (texture synthesis only)."""
    M, N = a.shape
    fy = np.fft.fftfreq(M)[:, None]
    fx = np.fft.fftfreq(N)[None, :]
    g = np.exp(-2.0 * (math.pi * sigma_px) ** 2 * (fx * fx + fy * fy))
    return np.real(np.fft.ifft2(np.fft.fft2(a) * g))


def image_polygons(seed: int, M: int, N: int, n_poly: int = 30,
                   texture_std: float = 0.02, texture_sigma_px: float = 1.5,
                   rng: np.random.Generator | None = None) -> np.ndarray:
    """Piecewise-smooth test image (float64, clipped to [0, 1]).

    ``n_poly`` random polygons (3..8 vertices at sorted random angles, radius
    U[0.05, 0.3]*size with a per-vertex jitter U[0.5, 1]) are painted over a
    background region.  Each region (the background included) carries its own
    quadratic shading c + g.(x, y) + quadratic terms, with c ~ U[0.1, 0.9] and
    the linear and quadratic coefficients ~ U[-0.2, 0.2], x, y in [-1, 1].
    A texture field (white Gaussian noise low-passed by a Gaussian of
    ``texture_sigma_px`` px, rescaled to std ``texture_std``) is added and the
    result is clipped to [0, 1]."""
    if rng is None:
        rng = np.random.default_rng(seed)
    x, y = pixel_grid(M, N, -1.0, 1.0)

    def shading():
        c = rng.uniform(0.1, 0.9)
        gx, gy, qxx, qxy, qyy = rng.uniform(-0.2, 0.2, size=5)
        return c, gx, gy, qxx, qxy, qyy

    def paint(mask, coef):
        c, gx, gy, qxx, qxy, qyy = coef
        xs, ys = x[mask], y[mask]
        u[mask] = c + gx * xs + gy * ys + qxx * xs * xs + qxy * xs * ys + qyy * ys * ys

    u = np.empty((M, N))
    paint(np.ones((M, N), dtype=bool), shading())
    size = min(M, N)
    for _ in range(n_poly):
        nv = int(rng.integers(3, 9))
        ang = np.sort(rng.uniform(0.0, 2.0 * math.pi, size=nv))
        rad = rng.uniform(0.05, 0.3) * size
        jit = rng.uniform(0.5, 1.0, size=nv)
        cx = rng.uniform(0.0, N)
        cy = rng.uniform(0.0, M)
        vx = cx + rad * jit * np.cos(ang)
        vy = cy + rad * jit * np.sin(ang)
        coef = shading()
        r0 = max(0, int(math.floor(vy.min())))
        r1 = min(M, int(math.ceil(vy.max())) + 1)
        c0 = max(0, int(math.floor(vx.min())))
        c1 = min(N, int(math.ceil(vx.max())) + 1)
        if r1 <= r0 or c1 <= c0:
            continue
        jj, ii = np.meshgrid(np.arange(c0, c1) + 0.5, np.arange(r0, r1) + 0.5)
        sub = _inside_polygon(jj, ii, vx, vy)
        mask = np.zeros((M, N), dtype=bool)
        mask[r0:r1, c0:c1] = sub
        paint(mask, coef)
    tex = _gaussian_lowpass_periodic(rng.standard_normal((M, N)), texture_sigma_px)
    tex *= texture_std / tex.std()
    return np.clip(u + tex, 0.0, 1.0)


# ----------------------------------------------------------------------------
# point-spread functions (all odd-sized, centred, float64, summing to 1)
# ----------------------------------------------------------------------------

def psf_uniform(k: int) -> np.ndarray:
    """k x k boxcar (Table 1, test 3 uses k = 9)."""
    return np.full((k, k), 1.0 / (k * k))


def psf_inv_quadratic(k: int = 15) -> np.ndarray:
    """h(i, j) = 1 / (1 + i^2 + j^2) for i, j = -(k-1)/2 .. (k-1)/2
    (Table 1, tests 1-2, k = 15), normalised to sum 1."""
    r = (k - 1) // 2
    i = np.arange(-r, r + 1)
    h = 1.0 / (1.0 + i[:, None] ** 2 + i[None, :] ** 2)
    return h / h.sum()


def psf_gaussian(k: int, sigma: float) -> np.ndarray:
    """k x k sampled Gaussian of standard deviation ``sigma`` px, sum 1
    (Table 1, test 5: sigma = 1.6; the support is not stated there)."""
    r = (k - 1) // 2
    i = np.arange(-r, r + 1)
    h = np.exp(-(i[:, None] ** 2 + i[None, :] ** 2) / (2.0 * sigma * sigma))
    return h / h.sum()


def psf_binomial5() -> np.ndarray:
    """[1 4 6 4 1]^T [1 4 6 4 1] / 256 (Table 1, test 4)."""
    v = np.array([1.0, 4.0, 6.0, 4.0, 1.0])
    return np.outer(v, v) / 256.0


def psf_motion(k: int = 31, length: float = 21.0, angle_deg: float = 30.0,
               samples_per_px: int = 100) -> np.ndarray:
    """Linear motion blur: a segment of ``length`` px through the kernel
    centre at ``angle_deg`` counter-clockwise from +x (y pointing up),
    sampled at ``samples_per_px`` points per pixel of length, each sample
    splatted bilinearly onto the grid, then normalised to sum 1."""
    c = (k - 1) / 2.0
    n = int(math.ceil(samples_per_px * length))
    t = (np.arange(n) + 0.5) / n * length - length / 2.0
    th = math.radians(angle_deg)
    col = c + t * math.cos(th)
    row = c - t * math.sin(th)
    h = np.zeros((k, k))
    r0 = np.floor(row).astype(int)
    c0 = np.floor(col).astype(int)
    fr = row - r0
    fc = col - c0
    for dr, dc, wt in ((0, 0, (1 - fr) * (1 - fc)), (0, 1, (1 - fr) * fc),
                       (1, 0, fr * (1 - fc)), (1, 1, fr * fc)):
        rr = r0 + dr
        cc = c0 + dc
        ok = (rr >= 0) & (rr < k) & (cc >= 0) & (cc < k)
        np.add.at(h, (rr[ok], cc[ok]), wt[ok])
    return h / h.sum()


def table1_psf(test: int) -> np.ndarray:
    """The five PSFs of the paper's Table 1 (tests 1..5).  Test 5's Gaussian
    support is unstated; 25 x 25 is used."""
    if test in (1, 2):
        return psf_inv_quadratic(15)
    if test == 3:
        return psf_uniform(9)
    if test == 4:
        return psf_binomial5()
    if test == 5:
        return psf_gaussian(25, 1.6)
    raise ValueError(test)


# Table 1 noise variances, on the [0, 255] intensity scale (Table 1 caption).
TABLE1_SIGMA2_255 = {1: 2.0, 2: 8.0, 3: 0.308, 4: 49.0, 5: 4.0}


# ----------------------------------------------------------------------------
# forward model (Eq. 1) -- data synthesis only
# ----------------------------------------------------------------------------

def blur_circular(u: np.ndarray, h: np.ndarray) -> np.ndarray:
    """h * u with periodic boundaries on the canvas of u: the PSF offset
    (i, j) (kernel centre = (0, 0)) is placed at canvas index (i mod M,
    j mod N).  Used to synthesise observations."""
    M, N = u.shape
    kh, kw = h.shape
    canvas = np.zeros((M, N))
    rh, rw = kh // 2, kw // 2
    for a in range(kh):
        for b in range(kw):
            canvas[(a - rh) % M, (b - rw) % N] += h[a, b]
    return np.real(np.fft.ifft2(np.fft.fft2(u) * np.fft.fft2(canvas)))


def sigma_from_bsnr(blurred: np.ndarray, bsnr_db: float) -> float:
    """Noise std for a blurred-signal-to-noise ratio
    BSNR = 10 log10(var(h*u) / sigma^2), var = mean-removed energy / pixels."""
    var = float(np.mean((blurred - blurred.mean()) ** 2))
    return math.sqrt(var / (10.0 ** (bsnr_db / 10.0)))


def mirror_extend(u: np.ndarray, M: int, N: int) -> np.ndarray:
    """Symmetric (mirror) extension of u at its bottom and right edges to an
    M x N canvas."""
    m, n = u.shape
    return np.pad(u, ((0, M - m), (0, N - n)), mode="symmetric")


def next_pow2(n: int) -> int:
    return 1 << (int(n) - 1).bit_length()


# ----------------------------------------------------------------------------
# workloads
# ----------------------------------------------------------------------------

@dataclass
class Problem:
    """One deconvolution problem on an M x N power-of-two canvas.

    y, h, u_orig are float32 (the exact bits both solvers see); sigma is the
    noise standard deviation on the [0, 1] scale."""
    y: np.ndarray
    h: np.ndarray
    sigma: float
    w: int
    eps: float
    iters: int
    u_orig: np.ndarray
    true_shape: tuple = (0, 0)
    meta: dict = field(default_factory=dict)

    @property
    def shape(self):
        return self.y.shape


def _degrade(u_canvas: np.ndarray, h: np.ndarray, rng: np.random.Generator,
             sigma: float | None = None, bsnr_db: float | None = None):
    hu = blur_circular(u_canvas, h)
    if sigma is None:
        sigma = sigma_from_bsnr(hu, bsnr_db)
    y = hu + sigma * rng.standard_normal(u_canvas.shape)
    return y, float(sigma)


def _f32(a):
    return np.ascontiguousarray(a, dtype=np.float32)


def config_c0(seed: int = 0, M: int = 256, N: int = 256) -> Problem:
    """Plain method, 256 x 256: rectangles and disks over a gradient, 9 x 9
    uniform PSF, AWGN at BSNR 40 dB, w = 5, eps = 1e-3, 10 iterations."""
    u = image_rects_disks(seed, M, N)
    h = psf_uniform(9)
    rng = np.random.default_rng(seed + 7919)
    y, sigma = _degrade(u, h, rng, bsnr_db=40.0)
    return Problem(_f32(y), _f32(h), sigma, 5, 1e-3, 10, _f32(u), (M, N),
                   {"name": "c0_256_uniform9_bsnr40"})


def config_c1(seed: int = 1, M: int = 512, N: int = 512) -> Problem:
    """Plain method, 512 x 512 piecewise-smooth, 15 x 15 1/(1+x^2+y^2) PSF,
    AWGN sigma = 2/255, w = 7, eps = 1e-3, 20 iterations."""
    u = image_polygons(seed, M, N, n_poly=30, texture_std=0.02)
    h = psf_inv_quadratic(15)
    rng = np.random.default_rng(seed + 7919)
    y, sigma = _degrade(u, h, rng, sigma=2.0 / 255.0)
    return Problem(_f32(y), _f32(h), sigma, 7, 1e-3, 20, _f32(u), (M, N),
                   {"name": "c1_512_invquad15_sigma2"})


C2_SIZES = ((256, 256), (384, 384), (512, 512), (768, 1024))  # (rows, cols)


def config_c2_image(i: int, iters: int = 15) -> Problem:
    """Image i of the 256-image uneven batch (seed 1000 + i): size uniform
    over {256^2, 384^2 -> 512^2, 512^2, 1024 x 768 -> 1024^2}, content as in
    the 512^2 workload, PSF uniform over {9 x 9 uniform, 25 x 25 Gaussian
    sigma ~ U[1, 3], 15 x 15 1/(1+x^2+y^2)}, BSNR ~ U[30, 40] dB,
    w in {5, 7, 9}, eps = 1e-3.  Padded sizes are mirror-extended clean
    images, blurred circularly on the canvas, with noise over the whole
    canvas."""
    rng = np.random.default_rng(1000 + i)
    m, n = C2_SIZES[int(rng.integers(0, 4))]
    kind = int(rng.integers(0, 3))
    gsig = rng.uniform(1.0, 3.0)
    bsnr = rng.uniform(30.0, 40.0)
    w = (5, 7, 9)[int(rng.integers(0, 3))]
    if kind == 0:
        h = psf_uniform(9)
    elif kind == 1:
        h = psf_gaussian(25, gsig)
    else:
        h = psf_inv_quadratic(15)
    M, N = next_pow2(m), next_pow2(n)
    u = image_polygons(1000 + i, m, n, n_poly=30, texture_std=0.02, rng=rng)
    uc = mirror_extend(u, M, N)
    y, sigma = _degrade(uc, h, rng, bsnr_db=bsnr)
    return Problem(_f32(y), _f32(h), sigma, w, 1e-3, iters, _f32(uc), (m, n),
                   {"name": f"c2_{i}", "psf": ("uniform9", "gauss25", "invquad15")[kind],
                    "gauss_sigma": gsig, "bsnr": bsnr})


def config_c2(n_images: int = 256, iters: int = 15):
    return [config_c2_image(i, iters) for i in range(n_images)]


def config_c4_image(j: int, size: int = 4096, iters: int = 30) -> Problem:
    """Large-image bandwidth stress (seed 4000 + j): piecewise-smooth content
    with texture std 0.03, 31 x 31 motion blur (length 21 px, 30 degrees),
    BSNR 35 dB, w = 9, eps = 1e-4, 30 iterations."""
    seed = 4000 + j
    rng = np.random.default_rng(seed)
    u = image_polygons(seed, size, size, n_poly=30, texture_std=0.03, rng=rng)
    h = psf_motion(31, 21.0, 30.0)
    y, sigma = _degrade(u, h, rng, bsnr_db=35.0)
    return Problem(_f32(y), _f32(h), sigma, 9, 1e-4, iters, _f32(u), (size, size),
                   {"name": f"c4_{j}"})


def config_c3_image(i: int, size: int = 512, iters: int = 10) -> Problem:
    """Differentiation workload, image i (seed 3000 + i): piecewise-smooth
    content as in the 512^2 workload, 25 x 25 Gaussian PSF with sigma 1.6,
    AWGN sigma = 1/255, w = 7, eps = 1e-3, 10 iterations; the loss is the MSE
    of u^10 against the clean image."""
    seed = 3000 + i
    rng = np.random.default_rng(seed)
    u = image_polygons(seed, size, size, n_poly=30, texture_std=0.02, rng=rng)
    h = psf_gaussian(25, 1.6)
    y, sigma = _degrade(u, h, rng, sigma=1.0 / 255.0)
    return Problem(_f32(y), _f32(h), sigma, 7, 1e-3, iters, _f32(u), (size, size),
                   {"name": f"c3_{i}"})


def config_table1(test: int, seed: int = 0, M: int = 256, N: int = 256,
                  iters: int = 30) -> Problem:
    """One of the paper's five experiment settings (Sec. 4, Table 1: PSF and
    noise variance on the [0, 255] scale) on a synthetic 256 x 256 stand-in
    for its test images (rectangles and disks over a gradient, as in the
    256^2 workload), with the paper's hand-tuned eps = 7.5e-4 and w = 3
    (Sec. 4) and about 30 iterations (Sec. 4's timing)."""
    u = image_rects_disks(seed, M, N)
    h = table1_psf(test)
    sigma = math.sqrt(TABLE1_SIGMA2_255[test]) / 255.0
    rng = np.random.default_rng(seed + 104729 * test)
    y, sigma = _degrade(u, h, rng, sigma=sigma)
    return Problem(_f32(y), _f32(h), sigma, 3, 7.5e-4, iters, _f32(u), (M, N),
                   {"name": f"table1_test{test}", "test": test})


def config_c4(batch: int = 4, size: int = 4096, iters: int = 30):
    return [config_c4_image(j, size, iters) for j in range(batch)]
