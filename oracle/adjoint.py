"""FP64 gradient of the unrolled method (test infrastructure only).

The method's K iterations (Sec. 3.1 Steps 0-3 with Sec. 3.2's lambda) are a
function of the observation y, the PSF h and the guided filter's eps; with the
loss L = mean((u^K - u_clean)^2) this module computes dL/dh, dL/deps and dL/dy
by reverse-mode differentiation, one step of the method at a time, from the
iterates u_E^k kept as checkpoints (every intermediate of a step is recomputed
from its u_E^k).  Each backward step is the chain rule applied to the forward
step it undoes (gfdeconv.py), in reverse order:

  guided filter (Eq. 3-5)  ->  inverse DFT  ->  spectral solves (Eq. 8-9)
  ->  lambda, the root of Eq. 11 (implicit function: dlambda = -(df - dT) / f')
  ->  DFT of u_E  ->  u_E = u^k of the previous step,

with H = DFT(embedded h), Y = DFT(y) and T = rho(y, h) P sigma^2 (Eq. 12)
collecting their gradients over all steps.  Where lambda = inf (u_E already
in the feasible set, Sec. 3.2) lambda is a constant (the branch has no
derivative) and u_I = u_p = u_E.  Windows are periodic (the box mean is then
its own adjoint).

Complex gradients: for a real L of a complex z, g_z = dL/dRe z + i dL/dIm z,
so that dL = Re(conj(g_z) dz).  With the unnormalised DFT U = F u of a real u,
g_u = Re(F^H g_U) = P Re(ifft2(g_U)); for u = Re(F^-1 U), g_U = fft2(g_u) / P.
"""
from __future__ import annotations

import math

import numpy as np

from . import gfdeconv as G


def _forward_step(H, Y, D2, uE, T, w, eps):
    """Steps 1-2 from u_E with every intermediate the backward step needs."""
    UE = np.fft.fft2(uE)
    lam, res, flag = G.solve_lambda(H, Y, UE, T)
    st = {"UE": UE, "lam": lam}
    if math.isinf(lam):
        uI = np.real(np.fft.ifft2(UE))
        up = uI.copy()
    else:
        a = np.abs(H) ** 2
        HY = np.conj(H) * Y
        DI = a + lam * D2
        Dp = a + lam
        UI = (HY + lam * D2 * UE) / DI
        Up = (HY + lam * UE) / Dp
        st.update(UI=UI, Up=Up, DI=DI, Dp=Dp)
        uI = np.real(np.fft.ifft2(UI))
        up = np.real(np.fft.ifft2(Up))
    st["uI"], st["up"] = uI, up
    st["u"] = G.guided_filter(uI, up, w, eps)
    return st


def guided_filter_backward(I, p, w, eps, g_u):
    """Reverse of u = guidfilter(I, p, w, eps) (Eq. 3-5): returns
    (g_I, g_p, g_eps) for the output gradient g_u."""
    box = G.box_mean
    mu, pbar = box(I, w), box(p, w)
    var = box(I * I, w) - mu * mu
    cov = box(I * p, w) - mu * pbar
    a = cov / (var + eps)
    b = pbar - a * mu
    abar = box(a, w)
    # u = abar I + bbar
    g_I = g_u * abar
    g_a = box(g_u * I, w)          # adjoint of abar = box(a)
    g_b = box(g_u, w)              # adjoint of bbar = box(b)
    # b = pbar - a mu
    g_pbar = g_b.copy()
    g_a = g_a - mu * g_b
    g_mu = -a * g_b
    # a = cov / (var + eps)
    g_cov = g_a / (var + eps)
    g_var = -g_a * a / (var + eps)
    g_eps = float(np.sum(-g_a * a / (var + eps)))
    # cov = box(I p) - mu pbar ;  var = box(I^2) - mu^2
    g_mIp = g_cov
    g_mu = g_mu - pbar * g_cov - 2.0 * mu * g_var
    g_pbar = g_pbar - mu * g_cov
    t = box(g_mIp, w)
    g_I = g_I + p * t
    g_p = I * t
    g_I = g_I + 2.0 * I * box(g_var, w)
    g_I = g_I + box(g_mu, w)
    g_p = g_p + box(g_pbar, w)
    return g_I, g_p, g_eps


def _rho_parts(y, h, sigma):
    """rho of Eq. 12 with the pieces its derivative needs."""
    y = np.asarray(y, dtype=np.float64)
    P = y.size
    Sy, Syy = float(np.sum(y)), float(np.sum(y * y))
    h1 = float(np.sum(np.abs(h)))
    num = Syy - Sy * Sy / P - P * sigma * sigma
    den = h1 * h1 * Syy
    rad = 1.0 - num / den
    return {"P": P, "Sy": Sy, "Syy": Syy, "h1": h1, "num": num, "den": den, "rad": rad,
            "rho": min(1.0, math.sqrt(rad)), "clamped": math.sqrt(rad) >= 1.0}


def solve_with_grad(y, h, sigma, w, eps, iters, u_clean, u_init=None):
    """L = mean((u^K - u_clean)^2) after `iters` iterations from u_E = 0 (or
    the constant start u_init) and its gradient.  Returns a dict: loss, g_h
    (kh x kw), g_eps, g_y (M x N), lam (the forward lambdas), u (u^K)."""
    y = np.asarray(y, dtype=np.float64)
    h = np.asarray(h, dtype=np.float64)
    u_clean = np.asarray(u_clean, dtype=np.float64)
    M, N = y.shape
    P = M * N
    H = G.psf_spectrum(h, M, N)
    Y = np.fft.fft2(y)
    D2 = G.grad_weight(M, N)
    rp = _rho_parts(y, h, sigma)
    T = rp["rho"] * P * sigma * sigma
    # forward, keeping the checkpoints u_E^k
    checkpoints, lams = [], []
    uE = np.zeros((M, N)) if u_init is None else np.asarray(u_init, dtype=np.float64)
    for _ in range(iters):
        checkpoints.append(uE)
        st = _forward_step(H, Y, D2, uE, T, w, eps)
        lams.append(st["lam"])
        uE = st["u"]
    u = uE
    loss = float(np.mean((u - u_clean) ** 2))
    # backward
    g_u = 2.0 * (u - u_clean) / P
    g_H = np.zeros((M, N), dtype=complex)
    g_Y = np.zeros((M, N), dtype=complex)
    g_T = 0.0
    g_eps = 0.0
    a = np.abs(H) ** 2
    for k in range(iters - 1, -1, -1):
        st = _forward_step(H, Y, D2, checkpoints[k], T, w, eps)
        g_uI, g_up, ge = guided_filter_backward(st["uI"], st["up"], w, eps, g_u)
        g_eps += ge
        lam = st["lam"]
        if math.isinf(lam):       # u_I = u_p = u_E, lambda constant
            g_u = g_uI + g_up
            continue
        UE = st["UE"]
        g_UI = np.fft.fft2(g_uI) / P
        g_Up = np.fft.fft2(g_up) / P
        # Eq. 9: U_p = (conj(H) Y + lam U_E) / (a + lam)
        g_Np = g_Up / st["Dp"]
        g_Dp = -np.real(np.conj(g_Up) * st["Up"]) / st["Dp"]
        # Eq. 8: U_I = (conj(H) Y + lam D2 U_E) / (a + lam D2)
        g_NI = g_UI / st["DI"]
        g_DI = -np.real(np.conj(g_UI) * st["UI"]) / st["DI"]
        g_N = g_Np + g_NI
        g_Y += H * g_N
        g_H += np.conj(g_N) * Y + 2.0 * (g_Dp + g_DI) * H
        g_UE = lam * g_Np + lam * D2 * g_NI
        g_lam = float(np.sum(np.real(np.conj(g_Np) * UE) + g_Dp)
                      + np.sum(np.real(np.conj(g_NI) * D2 * UE) + D2 * g_DI))
        # Eq. 11: f(lam; U_E, H, Y) = T, f = (1/P) sum lam^2 |e|^2 / (a + lam)^2,
        # e = H U_E - Y; dlam = -(df - dT) / f'(lam)
        e = H * UE - Y
        r = np.abs(e) ** 2
        fprime = float(np.sum(r * 2.0 * lam * a / (a + lam) ** 3) / P)
        c = -g_lam / fprime
        g_T += -c
        g_e = c * (lam * lam / (a + lam) ** 2) * 2.0 * e / P
        g_a = c * (-2.0 * lam * lam * r / (a + lam) ** 3) / P
        g_UE += np.conj(H) * g_e
        g_H += np.conj(UE) * g_e + 2.0 * g_a * H
        g_Y += -g_e
        # U_E = F u_E
        g_u = P * np.real(np.fft.ifft2(g_UE))
    # Y = F y; H = F embed(h)
    g_y = P * np.real(np.fft.ifft2(g_Y))
    g_hc = P * np.real(np.fft.ifft2(g_H))
    kh, kw = h.shape
    rh, rw = kh // 2, kw // 2
    g_h = np.zeros_like(h)
    for i in range(kh):
        for j in range(kw):
            g_h[i, j] = g_hc[(i - rh) % M, (j - rw) % N]
    # T = rho P sigma^2, rho = sqrt(1 - num / den) (Eq. 12) unless clamped to 1
    if not rp["clamped"]:
        g_rad = g_T * P * sigma * sigma / (2.0 * rp["rho"])
        g_num = -g_rad / rp["den"]
        g_den = g_rad * rp["num"] / rp["den"] ** 2
        g_y += g_num * (2.0 * y - 2.0 * rp["Sy"] / P) + g_den * rp["h1"] ** 2 * 2.0 * y
        g_h += g_den * 2.0 * rp["h1"] * rp["Syy"] * np.sign(h)
    return {"loss": loss, "g_h": g_h, "g_eps": g_eps, "g_y": g_y, "lam": lams, "u": u}


def loss_only(y, h, sigma, w, eps, iters, u_clean, u_init=None):
    """L = mean((u^K - u_clean)^2) of the oracle's solve (for finite differences)."""
    r = G.solve(np.asarray(y, dtype=np.float64), np.asarray(h, dtype=np.float64), sigma, w, eps,
                iters, u_init=u_init)
    return float(np.mean((r["u"] - np.asarray(u_clean, dtype=np.float64)) ** 2))
