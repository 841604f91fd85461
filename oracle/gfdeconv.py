"""FP64 oracle: the paper's method step by step (test infrastructure only).

Notation follows the paper: y observed image, h PSF, sigma noise std,
u_E pre-estimate, u_I guidance image, u_p filtering input, w window size,
eps guided-filter regulariser, lambda deblurring regulariser, rho the
discrepancy factor.  The canvas is M x N (the paper writes N^2 for the pixel
count; reading: P = M*N).
"""
from __future__ import annotations

import math

import numpy as np

NONCONVERGED = 1          # flag: the root of Eq. 11 lies below LAMBDA_LO
LAMBDA_LO = 1e-14         # reading: lower end of the bisection bracket
LAMBDA_RTOL = 1e-13       # reading: bisection stops at this relative width


# ---------------------------------------------------------------------------
# Degradation model and Fourier diagonalisation (Sec. 1 Eq. 1; Sec. 3.1)
# ---------------------------------------------------------------------------

def embed_psf(h, M, N):
    """Circular embedding of a centred odd-sized PSF into an M x N canvas:
    offset (i, j) from the kernel centre goes to (i mod M, j mod N), so that
    the DFT product is the circular convolution h*u of Eq. 1 (the FFT
    diagonalisation of Sec. 3.1 assumes periodic boundaries)."""
    h = np.asarray(h, dtype=np.float64)
    kh, kw = h.shape
    if kh % 2 == 0 or kw % 2 == 0:
        raise ValueError("PSF sizes must be odd")
    rh, rw = kh // 2, kw // 2
    canvas = np.zeros((M, N))
    for a in range(kh):
        for b in range(kw):
            canvas[(a - rh) % M, (b - rw) % N] += h[a, b]
    return canvas


def psf_spectrum(h, M, N):
    """F(h): full M x N DFT of the embedded PSF (Sec. 3.1, Eq. 8-9)."""
    return np.fft.fft2(embed_psf(h, M, N))


def grad_weight(M, N):
    """|F(nabla)|^2 = |F(d_x)|^2 + |F(d_y)|^2 (Sec. 3.1, below Eq. 9).
    reading: periodic forward differences, whose DFT magnitudes squared are
    4 sin^2(pi k / M) (vertical) and 4 sin^2(pi l / N) (horizontal)."""
    k = np.arange(M)[:, None]
    l = np.arange(N)[None, :]
    return 4.0 * np.sin(np.pi * k / M) ** 2 + 4.0 * np.sin(np.pi * l / N) ** 2


# ---------------------------------------------------------------------------
# Discrepancy principle (Sec. 3.2, Eq. 10-12)
# ---------------------------------------------------------------------------

def rho_eq12(y, h, sigma):
    """rho = sqrt(1 - (||y - mu(y)||^2 - N^2 sigma^2) / (||h||_1^2 ||y||^2))
    (Sec. 3.2, Eq. 12).  reading: N^2 is the pixel count P; rho is clamped
    to 1 when the radicand exceeds 1, as 0 < rho <= 1 is required by the
    feasible set K (Sec. 3.2).  A non-positive radicand is an invalid input."""
    y = np.asarray(y, dtype=np.float64)
    h = np.asarray(h, dtype=np.float64)
    P = y.size
    num = np.sum((y - y.mean()) ** 2) - P * sigma * sigma
    den = np.sum(np.abs(h)) ** 2 * np.sum(y * y)
    rad = 1.0 - num / den
    if not rad > 0.0:
        raise ValueError("Eq. 12 radicand is not positive")
    return min(1.0, math.sqrt(rad))


def discrepancy_target(y, h, sigma, rho=None):
    """Right-hand side of K's bound: rho * N^2 * sigma^2 (Sec. 3.2)."""
    if rho is None:
        rho = rho_eq12(y, h, sigma)
    return rho * np.asarray(y).size * sigma * sigma


def residual_norm2(H, Y, UE):
    """||h*u_E - y||^2 computed by Parseval from the full spectra:
    (1/P) sum |H U_E - Y|^2 (right-hand side of Eq. 10; reading: the 1/P of
    the unnormalised DFT that the paper omits)."""
    return float(np.sum(np.abs(H * UE - Y) ** 2) / H.size)


def f_lambda(lam, a, r, P):
    """Left-hand side of Eq. 11: || lambda (F(h)F(u_E) - F(y)) /
    (|F(h)|^2 + lambda) ||^2, i.e. (1/P) sum lambda^2 r / (a + lambda)^2 with
    a = |F(h)|^2 and r = |F(h)F(u_E) - F(y)|^2 (Sec. 3.2, Eq. 10-11)."""
    return float(np.sum(lam * lam * r / (a + lam) ** 2) / P)


def solve_lambda(H, Y, UE, T):
    """lambda for one iteration (Sec. 3.2).

    If ||h*u_E - y||^2 <= T, u_E lies in K and lambda = inf (the branch after
    Eq. 10; a tie counts as inside K since K uses "<=").  Otherwise the root of
    Eq. 11 is found by bisection, as the paper says (the left-hand side is
    increasing in lambda).  reading: the bisection runs in log(lambda) from
    [LAMBDA_LO, hi], hi doubled from 1 until f(hi) >= T, until the relative
    width is <= LAMBDA_RTOL; the result is the geometric midpoint.  If even
    f(LAMBDA_LO) > T the result is LAMBDA_LO with the NONCONVERGED flag.

    Returns (lambda, res_inf, flag)."""
    P = H.size
    a = np.abs(H) ** 2
    r = np.abs(H * UE - Y) ** 2
    res = float(np.sum(r) / P)
    if res <= T:
        return math.inf, res, 0
    lo = LAMBDA_LO
    if f_lambda(lo, a, r, P) > T:
        return lo, res, NONCONVERGED
    hi = 1.0
    while f_lambda(hi, a, r, P) < T:
        hi *= 2.0
        if hi > 1e300:
            break
    while hi / lo - 1.0 > LAMBDA_RTOL:
        mid = math.sqrt(lo * hi)
        if f_lambda(mid, a, r, P) < T:
            lo = mid
        else:
            hi = mid
    return math.sqrt(lo * hi), res, 0


# ---------------------------------------------------------------------------
# Deblurring step: the two Fourier-domain solves (Sec. 3.1, Eq. 6-9)
# ---------------------------------------------------------------------------

def deblur(H, Y, UE, lam, D2):
    """u_I from Eq. 8 (minimiser of Eq. 6) and u_p from Eq. 9 (minimiser of
    Eq. 7), with component-wise arithmetic on the full spectra.  reading: one
    lambda serves both solves.  lambda = inf gives u_I = u_p = u_E (Sec. 3.2).
    Returns (u_I, u_p) as real images."""
    if math.isinf(lam):
        uE = np.real(np.fft.ifft2(UE))
        return uE.copy(), uE.copy()
    HY = np.conj(H) * Y
    a = np.abs(H) ** 2
    UI = (HY + lam * D2 * UE) / (a + lam * D2)
    Up = (HY + lam * UE) / (a + lam)
    return np.real(np.fft.ifft2(UI)), np.real(np.fft.ifft2(Up))


# ---------------------------------------------------------------------------
# Denoising step: the guided filter (Sec. 2, Eq. 2-5)
# ---------------------------------------------------------------------------

def box_mean(x, w):
    """(1/w^2) sum over the w x w window centred at each pixel.
    reading: periodic windows (the normalisation 1/w^2 of Eq. 3 and Eq. 5 is a
    true mean only if every window holds w^2 pixels).  Written as the nested
    sum over the window's row offsets of the sum over its column offsets."""
    if w % 2 != 1 or w < 1:
        raise ValueError("w must be odd and positive")
    rad = (w - 1) // 2
    inner = np.zeros_like(x, dtype=np.float64)
    for dx in range(-rad, rad + 1):
        inner += np.roll(x, dx, axis=1)
    outer = np.zeros_like(inner)
    for dy in range(-rad, rad + 1):
        outer += np.roll(inner, dy, axis=0)
    return outer / (w * w)


def box_mean_truncated(x, w):
    """Window mean with the w x w window cut at the canvas edge: the sum of
    the window's pixels that lie inside the canvas divided by their number.
    reading: the non-periodic boundary of He et al.'s box filter, which the
    paper cites for its O(N^2) guided filter (Sec. 3.1); an opt-in variant of
    the periodic windows above.  Written as the sum over the window's
    offsets of the zero-extended image, divided by the same sum of ones."""
    if w % 2 != 1 or w < 1:
        raise ValueError("w must be odd and positive")
    rad = (w - 1) // 2
    x = np.asarray(x, dtype=np.float64)
    M, N = x.shape
    xz = np.pad(x, rad)                       # zero outside the canvas
    oz = np.pad(np.ones((M, N)), rad)
    total = np.zeros((M, N))
    count = np.zeros((M, N))
    for dy in range(-rad, rad + 1):
        for dx in range(-rad, rad + 1):
            total += xz[rad + dy:rad + dy + M, rad + dx:rad + dx + N]
            count += oz[rad + dy:rad + dy + M, rad + dx:rad + dx + N]
    return total / count


BOX_MEANS = {"periodic": box_mean, "truncated": box_mean_truncated}


def guided_filter(uI, up, w, eps, boundary="periodic"):
    """u = guidfilter(u_I, u_p, w, eps) (Sec. 2):
    a_k = (mean_w(u_I u_p) - mu_k pbar_k) / (sigma_k^2 + eps)   (Eq. 3)
    b_k = pbar_k - a_k mu_k                                      (Eq. 4)
    u(i) = abar_i u_I(i) + bbar_i                                (Eq. 5)
    with mu_k, pbar_k the window means of u_I, u_p and sigma_k^2 the window
    (population) variance of u_I (reading of "mean and variance").
    The filter output averages a and b over the windows covering each pixel
    (reading of Eq. 5's garbled index: the window centred at i).
    ``boundary`` selects periodic windows (default) or windows truncated at
    the canvas edge (box_mean_truncated); Eq. 3-5 are the same for both."""
    box = BOX_MEANS[boundary]
    uI = np.asarray(uI, dtype=np.float64)
    up = np.asarray(up, dtype=np.float64)
    mu = box(uI, w)
    pbar = box(up, w)
    var = box(uI * uI, w) - mu * mu
    a = (box(uI * up, w) - mu * pbar) / (var + eps)
    b = pbar - a * mu
    return box(a, w) * uI + box(b, w)


def guided_filter_color(I, p, w, eps, boundary="periodic"):
    """Guided filter with a colour guidance image (Sec. 3.1 remarks that the
    guided filter applies to colour as well as grey-scale images): I is
    M x N x 3, p is M x N.  reading: the local linear model of Eq. 2 with a
    3-vector slope, u(i) = a_k . I(i) + b_k, whose least-squares solution over
    window k with the regulariser eps |a_k|^2 of Eq. 3 is
        a_k = (Sigma_k + eps U)^-1 (mean_k(I p) - mu_k pbar_k)
        b_k = pbar_k - a_k . mu_k                                  (Eq. 4)
    with mu_k the window mean of I (3-vector), Sigma_k its window covariance
    (3 x 3, population), U the identity; the output averages a and b over the
    windows covering each pixel as in Eq. 5: u = abar . I + bbar.  The 3 x 3
    systems are solved with numpy.linalg.solve (a library primitive)."""
    box = BOX_MEANS[boundary]
    I = np.asarray(I, dtype=np.float64)
    p = np.asarray(p, dtype=np.float64)
    M, N, C = I.shape
    mu = np.stack([box(I[:, :, c], w) for c in range(C)], axis=-1)
    pbar = box(p, w)
    cov_Ip = np.stack([box(I[:, :, c] * p, w) for c in range(C)], axis=-1) - mu * pbar[..., None]
    Sigma = np.empty((M, N, C, C))
    for c in range(C):
        for d in range(C):
            Sigma[:, :, c, d] = box(I[:, :, c] * I[:, :, d], w) - mu[:, :, c] * mu[:, :, d]
    a = np.linalg.solve(Sigma + eps * np.eye(C), cov_Ip[..., None])[..., 0]
    b = pbar - np.sum(a * mu, axis=-1)
    abar = np.stack([box(a[:, :, c], w) for c in range(C)], axis=-1)
    return np.sum(abar * I, axis=-1) + box(b, w)


# ---------------------------------------------------------------------------
# Observation padded to a power-of-two canvas (reading of the paper's silence
# on image sizes; the variant that pads only y)
# ---------------------------------------------------------------------------

def pad_symmetric(y, M, N):
    """y (m x n) extended to M x N by symmetric reflection at its bottom and
    right edges (the edge sample repeats: ... c b a | a b c ...), so that the
    circular model of the canvas sees no jump where the canvas wraps.
    reading: the problem is posed on the true size and only the observation
    is extended; the solve runs on the canvas and its result is cropped."""
    y = np.asarray(y, dtype=np.float64)
    m, n = y.shape
    return np.pad(y, ((0, M - m), (0, N - n)), mode="symmetric")


def crop(u, m, n):
    """The top-left m x n part of a canvas-sized result."""
    return np.asarray(u)[:m, :n].copy()


# ---------------------------------------------------------------------------
# Evaluation (Sec. 4)
# ---------------------------------------------------------------------------

def isnr(y, u_orig, u):
    """Improvement in SNR (dB): 10 log10(||y - u_orig||^2 / ||u - u_orig||^2).
    reading: the standard definition; the paper uses ISNR without defining
    it (Sec. 4, Tables 2-3)."""
    y = np.asarray(y, dtype=np.float64)
    uo = np.asarray(u_orig, dtype=np.float64)
    u = np.asarray(u, dtype=np.float64)
    return 10.0 * math.log10(np.sum((y - uo) ** 2) / np.sum((u - uo) ** 2))


# ---------------------------------------------------------------------------
# The algorithm (Sec. 3.1 Steps 0-3, Sec. 3.2)
# ---------------------------------------------------------------------------

def iterate(H, Y, D2, uE, T, w, eps, boundary="periodic"):
    """One pass of Steps 1-2: lambda by the discrepancy principle, the two
    deblurring solves, then the guided filter.  Returns a dict with the new
    iterate u and the step's intermediates (lambda, res = ||h*u_E - y||^2,
    flag, u_I, u_p)."""
    UE = np.fft.fft2(uE)
    lam, res, flag = solve_lambda(H, Y, UE, T)
    uI, up = deblur(H, Y, UE, lam, D2)
    u = guided_filter(uI, up, w, eps, boundary)
    return {"u": u, "lam": lam, "res": res, "flag": flag, "uI": uI, "up": up}


def solve(y, h, sigma, w, eps, iters, u_orig=None, u_init=None, rho=None,
          trace=False, boundary="periodic"):
    """The whole method (Sec. 3.1 Steps 0-3 with Sec. 3.2's lambda).

    Step 0 sets u_E = 0 (or ``u_init``, for resuming).  Each iteration k runs
    Steps 1-2 and records lambda_k, res_k = ||h*u_E^k - y||^2, the flag, and,
    if ``u_orig`` is given, ISNR_k of u^{k+1}.  Step 3 sets u_E = u^{k+1}.

    Returns a dict: u (float64 final iterate), lam, res, flag, isnr (lists),
    rho, T, and with ``trace`` the per-iteration u_E, u_I, u_p, u."""
    y = np.asarray(y, dtype=np.float64)
    M, N = y.shape
    H = psf_spectrum(h, M, N)
    Y = np.fft.fft2(y)
    D2 = grad_weight(M, N)
    if rho is None:
        rho = rho_eq12(y, h, sigma)
    T = rho * y.size * sigma * sigma
    uE = np.zeros((M, N)) if u_init is None else np.asarray(u_init, dtype=np.float64)
    out = {"lam": [], "res": [], "flag": [], "isnr": [], "rho": rho, "T": T}
    if trace:
        out.update({"uE": [], "uI": [], "up": [], "u_k": []})
    for _ in range(iters):
        st = iterate(H, Y, D2, uE, T, w, eps, boundary)
        out["lam"].append(st["lam"])
        out["res"].append(st["res"])
        out["flag"].append(st["flag"])
        if u_orig is not None:
            out["isnr"].append(isnr(y, u_orig, st["u"]))
        if trace:
            out["uE"].append(uE)
            out["uI"].append(st["uI"])
            out["up"].append(st["up"])
            out["u_k"].append(st["u"])
        uE = st["u"]
    out["u"] = uE
    return out
