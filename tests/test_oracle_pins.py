"""Pins for the FP64 oracle against things other than itself: brute force on
tiny inputs, closed forms, exact rational arithmetic and invariants that the
paper's equations imply.  CPU only."""
import math
from fractions import Fraction

import numpy as np
import pytest

import oracle as O
import synthetic as S

RNG = np.random.default_rng(12345)


# ---------------------------------------------------------------------------
# independent brute-force helpers (no oracle code)
# ---------------------------------------------------------------------------

def conv_direct(u, h):
    """(h*u)(i,j) = sum_{a,b} h(a,b) u(i-a, j-b), offsets relative to the
    kernel centre, periodic: the circular convolution of Eq. 1 by loops."""
    M, N = u.shape
    kh, kw = h.shape
    rh, rw = kh // 2, kw // 2
    out = np.zeros((M, N))
    for i in range(M):
        for j in range(N):
            s = 0.0
            for a in range(kh):
                for b in range(kw):
                    s += h[a, b] * u[(i - (a - rh)) % M, (j - (b - rw)) % N]
            out[i, j] = s
    return out


def corr_direct(v, h):
    """Adjoint of conv_direct: (h^T * v)(i,j) = sum h(a,b) v(i+a, j+b)."""
    M, N = v.shape
    kh, kw = h.shape
    rh, rw = kh // 2, kw // 2
    out = np.zeros((M, N))
    for i in range(M):
        for j in range(N):
            s = 0.0
            for a in range(kh):
                for b in range(kw):
                    s += h[a, b] * v[(i + (a - rh)) % M, (j + (b - rw)) % N]
            out[i, j] = s
    return out


def dft2_direct(x):
    """O(P^2) 2-D DFT, X(k,l) = sum x(i,j) exp(-2 pi i (ki/M + lj/N))."""
    M, N = x.shape
    i = np.arange(M)
    j = np.arange(N)
    Fm = np.exp(-2j * np.pi * np.outer(i, i) / M)
    Fn = np.exp(-2j * np.pi * np.outer(j, j) / N)
    X = np.zeros((M, N), dtype=complex)
    for k in range(M):
        for l in range(N):
            X[k, l] = np.sum(x * Fm[k][:, None] * Fn[l][None, :])
    return X


def gtg(u):
    """nabla^T nabla u for periodic forward differences, by stencils."""
    dx = np.roll(u, -1, axis=1) - u
    dy = np.roll(u, -1, axis=0) - u
    return (np.roll(dx, 1, axis=1) - dx) + (np.roll(dy, 1, axis=0) - dy)


def gf_bruteforce(I, p, w, eps):
    """Per-pixel loops over periodic windows, Eq. 3-5 written out."""
    M, N = I.shape
    r = (w - 1) // 2
    a = np.zeros((M, N))
    b = np.zeros((M, N))
    for ky in range(M):
        for kx in range(N):
            Iv, pv = [], []
            for dy in range(-r, r + 1):
                for dx in range(-r, r + 1):
                    Iv.append(I[(ky + dy) % M, (kx + dx) % N])
                    pv.append(p[(ky + dy) % M, (kx + dx) % N])
            Iv = np.array(Iv)
            pv = np.array(pv)
            mu = Iv.mean()
            pb = pv.mean()
            var = np.mean((Iv - mu) ** 2)
            cov = np.mean(Iv * pv) - mu * pb
            a[ky, kx] = cov / (var + eps)
            b[ky, kx] = pb - a[ky, kx] * mu
    u = np.zeros((M, N))
    for iy in range(M):
        for ix in range(N):
            sa = sb = 0.0
            for dy in range(-r, r + 1):
                for dx in range(-r, r + 1):
                    sa += a[(iy + dy) % M, (ix + dx) % N]
                    sb += b[(iy + dy) % M, (ix + dx) % N]
            u[iy, ix] = sa / (w * w) * I[iy, ix] + sb / (w * w)
    return u


# ---------------------------------------------------------------------------
# Fourier diagonalisation (Sec. 3.1) and the forward model (Eq. 1)
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("M,N", [(8, 8), (16, 16), (8, 32)])
def test_psf_spectrum_matches_direct_dft(M, N):
    h = RNG.random((3, 5))
    H = O.psf_spectrum(h, M, N)
    X = dft2_direct(O.embed_psf(h, M, N))
    assert np.abs(H - X).max() < 1e-12


def test_fft_convolution_equals_direct_circular_convolution():
    # asymmetric PSF pins the embedding orientation (convolution, not correlation)
    M, N = 12, 16
    u = RNG.random((M, N))
    h = RNG.random((5, 3))
    via_fft = np.real(np.fft.ifft2(np.fft.fft2(u) * O.psf_spectrum(h, M, N)))
    assert np.abs(via_fft - conv_direct(u, h)).max() < 1e-12


def test_embed_psf_wraps_large_kernel():
    # a 5x5 kernel on a 4x4 canvas: offsets -2 and +2 both land on index 2
    h = np.arange(1.0, 26.0).reshape(5, 5)
    c = O.embed_psf(h, 4, 4)
    assert abs(c.sum() - h.sum()) < 1e-12
    assert c[0, 0] == h[2, 2]                       # kernel centre at (0, 0)
    assert c[0, 1] == h[2, 3] and c[1, 0] == h[3, 2]
    assert c[2, 2] == h[0, 0] + h[0, 4] + h[4, 0] + h[4, 4]


def test_grad_weight_is_dft_of_forward_difference_stencils():
    M, N = 8, 16
    sx = np.zeros((M, N))
    sx[0, 0] = -1.0
    sx[0, 1] = 1.0
    sy = np.zeros((M, N))
    sy[0, 0] = -1.0
    sy[1, 0] = 1.0
    D2 = np.abs(dft2_direct(sx)) ** 2 + np.abs(dft2_direct(sy)) ** 2
    assert np.abs(O.grad_weight(M, N) - D2).max() < 1e-12


def test_grad_weight_parseval_against_gradient_energy():
    M, N = 16, 8
    u = RNG.random((M, N))
    dx = np.roll(u, -1, axis=1) - u
    dy = np.roll(u, -1, axis=0) - u
    energy = np.sum(dx * dx + dy * dy)
    spec = np.sum(O.grad_weight(M, N) * np.abs(np.fft.fft2(u)) ** 2) / (M * N)
    assert abs(energy - spec) < 1e-11 * energy


# ---------------------------------------------------------------------------
# Deblurring solves (Eq. 6-9): spatial normal equations by direct stencils
# ---------------------------------------------------------------------------

@pytest.fixture(scope="module")
def small_problem():
    M, N = 16, 12
    u0 = RNG.random((M, N))
    h = RNG.random((3, 5))
    h /= h.sum()
    y = conv_direct(u0, h) + 0.01 * RNG.standard_normal((M, N))
    uE = RNG.random((M, N))
    return M, N, y, h, uE


def test_up_satisfies_normal_equations_of_eq7(small_problem):
    M, N, y, h, uE = small_problem
    lam = 0.037
    H = O.psf_spectrum(h, M, N)
    _, up = O.deblur(H, np.fft.fft2(y), np.fft.fft2(uE), lam, O.grad_weight(M, N))
    g = corr_direct(conv_direct(up, h) - y, h) + lam * (up - uE)
    assert np.abs(g).max() < 1e-10


def test_uI_satisfies_normal_equations_of_eq6(small_problem):
    M, N, y, h, uE = small_problem
    lam = 0.21
    H = O.psf_spectrum(h, M, N)
    uI, _ = O.deblur(H, np.fft.fft2(y), np.fft.fft2(uE), lam, O.grad_weight(M, N))
    g = corr_direct(conv_direct(uI, h) - y, h) + lam * gtg(uI - uE)
    assert np.abs(g).max() < 1e-10


def test_deblur_limits(small_problem):
    M, N, y, h, uE = small_problem
    H = O.psf_spectrum(h, M, N)
    Y, UE, D2 = np.fft.fft2(y), np.fft.fft2(uE), O.grad_weight(M, N)
    # lambda -> inf: both solutions tend to u_E; lambda = inf is the branch
    uI, up = O.deblur(H, Y, UE, 1e12, D2)
    assert np.abs(up - uE).max() < 1e-9
    uI, up = O.deblur(H, Y, UE, math.inf, D2)
    assert np.abs(up - uE).max() < 1e-14 and np.abs(uI - uE).max() < 1e-14
    # invertible H and lambda -> 0: h*u_p reproduces y
    hi = np.array([[0.05, 0.1, 0.05], [0.1, 1.0, 0.1], [0.05, 0.1, 0.05]])
    Hi = O.psf_spectrum(hi, M, N)
    assert np.abs(Hi).min() > 0.3
    _, up = O.deblur(Hi, Y, UE, 1e-13, D2)
    assert np.abs(conv_direct(up, hi) - y).max() < 1e-10


# ---------------------------------------------------------------------------
# Discrepancy principle (Sec. 3.2, Eq. 10-12)
# ---------------------------------------------------------------------------

def test_residual_norm2_is_spatial_residual(small_problem):
    M, N, y, h, uE = small_problem
    H = O.psf_spectrum(h, M, N)
    res = O.residual_norm2(H, np.fft.fft2(y), np.fft.fft2(uE))
    direct = np.sum((conv_direct(uE, h) - y) ** 2)
    assert abs(res - direct) < 1e-11 * direct


def test_lambda_root_meets_target_and_eq10(small_problem):
    M, N, y, h, uE = small_problem
    H = O.psf_spectrum(h, M, N)
    Y, UE, D2 = np.fft.fft2(y), np.fft.fft2(uE), O.grad_weight(M, N)
    resE = np.sum((conv_direct(uE, h) - y) ** 2)
    T = 0.3 * resE
    lam, res, flag = O.solve_lambda(H, Y, UE, T)
    assert flag == 0 and math.isfinite(lam)
    assert abs(res - resE) < 1e-11 * resE
    _, up = O.deblur(H, Y, UE, lam, D2)
    resp = np.sum((conv_direct(up, h) - y) ** 2)
    assert abs(resp - T) < 1e-9 * T          # Eq. 11 reached, measured spatially
    assert resp <= resE                        # Eq. 10 inequality


def test_f_lambda_monotone_and_limits(small_problem):
    M, N, y, h, uE = small_problem
    H = O.psf_spectrum(h, M, N)
    a = np.abs(H) ** 2
    r = np.abs(H * np.fft.fft2(uE) - np.fft.fft2(y)) ** 2
    lams = np.geomspace(1e-8, 1e8, 200)
    f = np.array([O.f_lambda(l, a, r, M * N) for l in lams])
    assert np.all(np.diff(f) > 0)
    assert f[-1] == pytest.approx(r.sum() / (M * N), rel=1e-7)
    assert f[0] < 1e-10 * f[-1]


def test_lambda_branch_when_uE_in_K(small_problem):
    M, N, y, h, uE = small_problem
    H = O.psf_spectrum(h, M, N)
    Y, UE = np.fft.fft2(y), np.fft.fft2(uE)
    res = O.residual_norm2(H, Y, UE)
    lam, _, _ = O.solve_lambda(H, Y, UE, res)        # tie counts as inside K
    assert math.isinf(lam)
    lam, _, _ = O.solve_lambda(H, Y, UE, 2 * res)
    assert math.isinf(lam)


def test_lambda_below_bracket_flags_nonconverged():
    M, N = 8, 8
    H = np.ones((M, N), dtype=complex)   # a = 1 everywhere
    Y = np.ones((M, N), dtype=complex)
    UE = np.zeros((M, N), dtype=complex)
    # f(lambda) = lambda^2/(1+lambda)^2 * 1; demand T below f(1e-14)
    lam, res, flag = O.solve_lambda(H, Y, UE, 1e-30)
    assert flag == O.NONCONVERGED and lam == O.LAMBDA_LO


def test_lambda_closed_form_single_level():
    # a and r constant: f = r lam^2/(a+lam)^2 = T  =>  lam = a t/(1-t), t = sqrt(T/r)
    M, N = 8, 4
    H = np.full((M, N), 0.5 + 0.0j)
    Y = np.full((M, N), 2.0 + 1.0j)
    UE = np.zeros((M, N), dtype=complex)
    a = 0.25
    r = 5.0
    T = 0.2 * r
    lam, res, _ = O.solve_lambda(H, Y, UE, T)
    t = math.sqrt(T / r)
    assert lam == pytest.approx(a * t / (1 - t), rel=1e-12)
    assert res == pytest.approx(r, rel=1e-14)


def test_rho_eq12_hand_computed():
    # 4x4 checkerboard of 0/1: mean 0.5, ||y-mu||^2 = 4, ||y||^2 = 8
    y = (np.indices((4, 4)).sum(axis=0) % 2).astype(float)
    h = np.array([[1.0]])
    sigma = 0.1
    rho = O.rho_eq12(y, h, sigma)
    assert rho == pytest.approx(math.sqrt(1 - (4 - 16 * 0.01) / 8), rel=1e-14)
    # ||h||_1 = 2 scales the denominator by 4
    rho2 = O.rho_eq12(y, 2.0 * h, sigma)
    assert rho2 == pytest.approx(math.sqrt(1 - (4 - 0.16) / 32), rel=1e-14)
    # a constant image has radicand > 1: clamped to 1
    assert O.rho_eq12(np.full((4, 4), 0.7), h, sigma) == 1.0
    assert O.discrepancy_target(y, h, sigma) == pytest.approx(rho * 16 * 0.01)


# ---------------------------------------------------------------------------
# Guided filter (Sec. 2, Eq. 2-5)
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("shape,w", [((7, 9), 1), ((7, 9), 3), ((7, 9), 5),
                                     ((16, 16), 7), ((5, 6), 7), ((4, 4), 9)])
def test_guided_filter_matches_bruteforce(shape, w):
    I = RNG.random(shape)
    p = I + 0.1 * RNG.standard_normal(shape)
    eps = 1e-3
    assert np.abs(O.guided_filter(I, p, w, eps) - gf_bruteforce(I, p, w, eps)).max() < 1e-12


def test_box_mean_matches_window_loops():
    x = RNG.random((6, 10))
    for w in (1, 3, 5, 7, 11):
        r = (w - 1) // 2
        ref = np.zeros_like(x)
        for i in range(6):
            for j in range(10):
                ref[i, j] = np.mean([x[(i + dy) % 6, (j + dx) % 10]
                                     for dy in range(-r, r + 1) for dx in range(-r, r + 1)])
        assert np.abs(O.box_mean(x, w) - ref).max() < 1e-14


def test_guided_filter_exact_rationals():
    """Eq. 3-5 in exact rational arithmetic on a 5x5 image, w = 3."""
    M = N = 5
    w, r = 3, 1
    Iq = [[Fraction(int(v), 8) for v in row] for row in (np.arange(25).reshape(5, 5) * 7 % 9)]
    pq = [[Fraction(int(v), 16) for v in row] for row in (np.arange(25).reshape(5, 5) * 5 % 11)]
    epsq = Fraction(1, 100)

    def win(A, i, j):
        return [A[(i + dy) % M][(j + dx) % N] for dy in range(-r, r + 1) for dx in range(-r, r + 1)]

    a = [[None] * N for _ in range(M)]
    b = [[None] * N for _ in range(M)]
    for i in range(M):
        for j in range(N):
            Iv, pv = win(Iq, i, j), win(pq, i, j)
            mu = sum(Iv) / 9
            pb = sum(pv) / 9
            var = sum(v * v for v in Iv) / 9 - mu * mu
            cov = sum(x * y for x, y in zip(Iv, pv)) / 9 - mu * pb
            a[i][j] = cov / (var + epsq)
            b[i][j] = pb - a[i][j] * mu
    u = np.zeros((M, N))
    for i in range(M):
        for j in range(N):
            u[i, j] = float(sum(win(a, i, j)) / 9 * Iq[i][j] + sum(win(b, i, j)) / 9)
    got = O.guided_filter(np.array(Iq, dtype=float), np.array(pq, dtype=float), w, 0.01)
    assert np.abs(got - u).max() < 1e-14


def test_guided_filter_invariants():
    I = RNG.random((12, 10))
    p = RNG.random((12, 10))
    w, eps = 5, 1e-3
    g = O.guided_filter(I, p, w, eps)
    # constant image is a fixed point
    c = np.full((12, 10), 0.3)
    assert np.abs(O.guided_filter(c, c, w, eps) - 0.3).max() < 1e-14
    # eps -> inf: a -> 0, b -> pbar, output -> box(box(p))
    big = O.guided_filter(I, p, w, 1e12)
    assert np.abs(big - O.box_mean(O.box_mean(p, w), w)).max() < 1e-10
    # I = p, eps -> 0: identity where the local variance is positive
    ident = O.guided_filter(I, I, w, 1e-14)
    assert np.abs(ident - I).max() < 1e-9
    # w = 1: one-pixel windows have zero variance and covariance -> output p
    assert np.abs(O.guided_filter(I, p, 1, eps) - p).max() < 1e-14
    # affine in p
    assert np.abs(O.guided_filter(I, 2.5 * p - 0.7, w, eps) - (2.5 * g - 0.7)).max() < 1e-12
    # invariant to I -> I + c
    assert np.abs(O.guided_filter(I + 3.0, p, w, eps) - g).max() < 1e-10
    # scaling I by s with eps by s^2
    assert np.abs(O.guided_filter(4.0 * I, p, w, 16.0 * eps) - g).max() < 1e-11
    # commutes with circular shifts
    sh = O.guided_filter(np.roll(I, (3, -2), (0, 1)), np.roll(p, (3, -2), (0, 1)), w, eps)
    assert np.abs(sh - np.roll(g, (3, -2), (0, 1))).max() < 1e-13


# ---------------------------------------------------------------------------
# Guided filter with windows truncated at the canvas edge (He et al.'s box
# filter, cited in Sec. 3.1): every mean over the window's in-canvas pixels
# ---------------------------------------------------------------------------

def gf_bruteforce_truncated(I, p, w, eps):
    """Per-pixel loops over the in-canvas part of every window, Eq. 3-5
    written out with the pixel count of each window as its normaliser."""
    M, N = I.shape
    r = (w - 1) // 2

    def window(A, i, j):
        return np.array([A[y, x] for y in range(max(0, i - r), min(M, i + r + 1))
                         for x in range(max(0, j - r), min(N, j + r + 1))])

    a = np.zeros((M, N))
    b = np.zeros((M, N))
    for i in range(M):
        for j in range(N):
            Iv, pv = window(I, i, j), window(p, i, j)
            mu, pb = Iv.mean(), pv.mean()
            a[i, j] = (np.mean(Iv * pv) - mu * pb) / (np.mean((Iv - mu) ** 2) + eps)
            b[i, j] = pb - a[i, j] * mu
    u = np.zeros((M, N))
    for i in range(M):
        for j in range(N):
            u[i, j] = window(a, i, j).mean() * I[i, j] + window(b, i, j).mean()
    return u


def test_box_mean_truncated_matches_window_loops():
    x = RNG.random((6, 10))
    for w in (1, 3, 5, 9, 13):
        r = (w - 1) // 2
        ref = np.zeros_like(x)
        for i in range(6):
            for j in range(10):
                ref[i, j] = x[max(0, i - r):i + r + 1, max(0, j - r):j + r + 1].mean()
        assert np.abs(O.box_mean_truncated(x, w) - ref).max() < 1e-14


@pytest.mark.parametrize("shape,w", [((7, 9), 3), ((7, 9), 5), ((5, 6), 7), ((12, 8), 9)])
def test_guided_filter_truncated_matches_bruteforce(shape, w):
    I = RNG.random(shape)
    p = I + 0.1 * RNG.standard_normal(shape)
    got = O.guided_filter(I, p, w, 1e-3, boundary="truncated")
    assert np.abs(got - gf_bruteforce_truncated(I, p, w, 1e-3)).max() < 1e-12


def test_guided_filter_truncated_special_cases():
    I = RNG.random((11, 13))
    p = RNG.random((11, 13))
    eps = 1e-3
    # constant image is a fixed point; w = 1 returns p
    c = np.full((11, 13), 0.6)
    assert np.abs(O.guided_filter(c, c, 5, eps, "truncated") - 0.6).max() < 1e-14
    assert np.abs(O.guided_filter(I, p, 1, eps, "truncated") - p).max() < 1e-14
    # a window reaching past every edge holds the whole canvas everywhere:
    # one global linear regression of p on I (closed form)
    w = 2 * 13 + 1
    a = (np.mean(I * p) - I.mean() * p.mean()) / (np.var(I) + eps)
    b = p.mean() - a * I.mean()
    assert np.abs(O.guided_filter(I, p, w, eps, "truncated") - (a * I + b)).max() < 1e-12
    # pixels at least 2r from every edge see only in-canvas windows: there the
    # truncated and periodic filters agree
    w, r = 3, 1
    t = O.guided_filter(I, p, w, eps, "truncated")
    g = O.guided_filter(I, p, w, eps, "periodic")
    assert np.abs(t[2 * r:-2 * r, 2 * r:-2 * r] - g[2 * r:-2 * r, 2 * r:-2 * r]).max() < 1e-13
    # and they differ next to the edge (the windows there wrap or are cut)
    assert np.abs(t[0] - g[0]).max() > 1e-6


# ---------------------------------------------------------------------------
# Colour guidance (3-channel I, 3 x 3 window covariance)
# ---------------------------------------------------------------------------

def gf_color_bruteforce(I, p, w, eps):
    """Per-pixel loops over periodic windows: the least-squares fit of
    p ~ a . I + b in each window with penalty eps |a|^2, solved by an explicit
    3 x 3 Cramer's rule, then the averages of a and b over covering windows."""
    M, N, C = I.shape
    r = (w - 1) // 2
    a = np.zeros((M, N, C))
    b = np.zeros((M, N))
    for i in range(M):
        for j in range(N):
            X = np.array([I[(i + dy) % M, (j + dx) % N] for dy in range(-r, r + 1)
                          for dx in range(-r, r + 1)])
            y = np.array([p[(i + dy) % M, (j + dx) % N] for dy in range(-r, r + 1)
                          for dx in range(-r, r + 1)])
            mu, pb = X.mean(axis=0), y.mean()
            Xc = X - mu
            A = Xc.T @ Xc / len(y) + eps * np.eye(C)
            rhs = Xc.T @ (y - pb) / len(y)
            det = np.linalg.det(A)
            for c in range(C):
                Ac = A.copy()
                Ac[:, c] = rhs
                a[i, j, c] = np.linalg.det(Ac) / det
            b[i, j] = pb - a[i, j] @ mu
    u = np.zeros((M, N))
    for i in range(M):
        for j in range(N):
            sa = np.zeros(C)
            sb = 0.0
            for dy in range(-r, r + 1):
                for dx in range(-r, r + 1):
                    sa += a[(i + dy) % M, (j + dx) % N]
                    sb += b[(i + dy) % M, (j + dx) % N]
            u[i, j] = sa @ I[i, j] / (w * w) + sb / (w * w)
    return u


@pytest.mark.parametrize("shape,w", [((6, 7), 3), ((5, 5), 5), ((8, 6), 1)])
def test_guided_filter_color_matches_bruteforce(shape, w):
    I = RNG.random(shape + (3,))
    p = I.mean(axis=-1) + 0.1 * RNG.standard_normal(shape)
    got = O.guided_filter_color(I, p, w, 1e-2)
    assert np.abs(got - gf_color_bruteforce(I, p, w, 1e-2)).max() < 1e-11


def test_guided_filter_color_special_cases():
    I = RNG.random((12, 10, 3))
    p = RNG.random((12, 10))
    w, eps = 5, 1e-3
    g = O.guided_filter_color(I, p, w, eps)
    # three equal channels: Sigma = var * ones, a = alpha (1, 1, 1) with
    # (3 var + eps) alpha = cov, i.e. the grey-scale filter with eps / 3
    G = RNG.random((12, 10))
    same = O.guided_filter_color(np.stack([G, G, G], axis=-1), p, w, eps)
    assert np.abs(same - O.guided_filter(G, p, w, eps / 3.0)).max() < 1e-11
    # constant guidance and input: fixed point; eps -> inf: box(box(p))
    c = np.full((12, 10), 0.4)
    assert np.abs(O.guided_filter_color(np.full((12, 10, 3), 0.7), c, w, eps) - 0.4).max() < 1e-13
    big = O.guided_filter_color(I, p, w, 1e12)
    assert np.abs(big - O.box_mean(O.box_mean(p, w), w)).max() < 1e-10
    # affine in p, invariant to a constant added to each guidance channel
    assert np.abs(O.guided_filter_color(I, 2.0 * p + 0.3, w, eps) - (2.0 * g + 0.3)).max() < 1e-11
    shift = I + np.array([1.0, -2.0, 0.5])
    assert np.abs(O.guided_filter_color(shift, p, w, eps) - g).max() < 1e-9
    # p equal to one guidance channel and eps -> 0: that channel is reproduced
    ident = O.guided_filter_color(I, I[:, :, 1], w, 1e-13)
    assert np.abs(ident - I[:, :, 1]).max() < 1e-7


# ---------------------------------------------------------------------------
# Padding only the observation to the canvas
# ---------------------------------------------------------------------------

def test_pad_symmetric_matches_index_reflection():
    y = RNG.random((5, 7))
    for M, N in ((8, 8), (5, 16), (16, 7), (32, 32)):
        got = O.pad_symmetric(y, M, N)
        ref = np.zeros((M, N))
        for i in range(M):
            for j in range(N):
                ti, tj = i % (2 * 5), j % (2 * 7)        # reflection period 2m
                si = ti if ti < 5 else 2 * 5 - 1 - ti
                sj = tj if tj < 7 else 2 * 7 - 1 - tj
                ref[i, j] = y[si, sj]
        assert np.array_equal(got, ref), (M, N)
    assert np.array_equal(O.pad_symmetric(y, 5, 7), y)
    assert np.array_equal(O.crop(O.pad_symmetric(y, 16, 16), 5, 7), y)


# ---------------------------------------------------------------------------
# ISNR (Sec. 4) and the whole iteration
# ---------------------------------------------------------------------------

def test_isnr_closed_form():
    uo = RNG.random((8, 8))
    y = uo + RNG.standard_normal((8, 8))
    assert O.isnr(y, uo, y) == pytest.approx(0.0, abs=1e-12)
    u = uo + (y - uo) / 10.0
    assert O.isnr(y, uo, u) == pytest.approx(20.0, rel=1e-12)


def test_solve_iterations_reach_target_and_decrease_residual():
    """Each non-branch iteration's u_p meets Eq. 11 exactly (checked by direct
    spatial convolution) and obeys Eq. 10's inequality."""
    M, N = 16, 16
    u0 = S.image_rects_disks(3, M, N, n_rect=3, n_disk=2)
    h = S.psf_uniform(3)
    rng = np.random.default_rng(5)
    y = conv_direct(u0, h) + 0.01 * rng.standard_normal((M, N))
    out = O.solve(y, h, 0.01, 3, 1e-3, 4, u_orig=u0, trace=True)
    H = O.psf_spectrum(h, M, N)
    for k in range(4):
        resE = np.sum((conv_direct(out["uE"][k], h) - y) ** 2)
        assert out["res"][k] == pytest.approx(resE, rel=1e-10)
        if math.isfinite(out["lam"][k]):
            resp = np.sum((conv_direct(out["up"][k], h) - y) ** 2)
            assert resp == pytest.approx(out["T"], rel=1e-9)
            assert resp <= resE
        u_next = O.guided_filter(out["uI"][k], out["up"][k], 3, 1e-3)
        assert np.abs(u_next - out["u_k"][k]).max() == 0.0
    assert H.shape == (M, N)


def test_step0_starts_from_zero():
    M, N = 16, 16
    y = RNG.random((M, N))
    h = S.psf_uniform(3)
    out = O.solve(y, h, 0.01, 3, 1e-3, 1, trace=True)
    assert np.all(out["uE"][0] == 0.0)
    # with u_E = 0 the residual is ||y||^2
    assert out["res"][0] == pytest.approx(np.sum(y * y), rel=1e-12)


# ---------------------------------------------------------------------------
# Table 1 PSFs (paper's printed settings, tests/golden/table1_settings.txt)
# ---------------------------------------------------------------------------

def test_table1_psfs_match_printed_definitions():
    import os
    path = os.path.join(os.path.dirname(__file__), "golden", "table1_settings.txt")
    rows = [l for l in open(path) if l.strip() and not l.startswith("#")]
    assert len(rows) == 5
    sig = {int(r.split("|")[0]): float(r.split("|")[2]) for r in rows}
    assert sig == S.TABLE1_SIGMA2_255
    b = S.psf_binomial5()
    assert b[2, 2] == 36 / 256 and b[0, 0] == 1 / 256 and b[0, 2] == 6 / 256
    iq = S.psf_inv_quadratic(15)
    raw = 1.0 / (1.0 + np.arange(-7, 8)[:, None] ** 2 + np.arange(-7, 8)[None, :] ** 2)
    assert np.allclose(iq, raw / raw.sum(), rtol=0, atol=1e-17)
    assert iq[7, 7] / iq[7, 8] == pytest.approx(2.0)
    assert np.all(S.psf_uniform(9) == 1 / 81)
    g = S.psf_gaussian(25, 1.6)
    assert g[12, 13] / g[12, 12] == pytest.approx(math.exp(-1 / (2 * 1.6 ** 2)))
