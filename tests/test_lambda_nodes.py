"""Accuracy of the node layout the GPU lambda procedure relies on (Sec. 3.2,
Eq. 10-11), checked on the CPU in FP64.

The GPU evaluates f(lambda) = sum_b lambda^2 r_b / (a_b + lambda)^2 at 12
nodes of a bracket and, for brackets of ratio <= 4, takes the root of the
degree-11 interpolant in t = ln(lambda) through Chebyshev-Lobatto nodes in t
as the answer (8 nodes, degree 7, on the ratio-1.56 first brackets of later
iterations).  These tests restate that layout (not the GPU code) and check
the claim it rests on: in t the poles of f sit at Im t = pi for every
spectrum, so the interpolated root is within ~1e-10 of the true one on ratio
4, whereas the same nodes in lambda (poles at lambda = -a_b, close to the
bracket when a_b -> 0) are not accurate enough there.
"""
import numpy as np
import pytest
from scipy.optimize import brentq

K = 12  # nodes per spectral pass


def f(lam, a, r):
    return np.sum(lam * lam * r / (a + lam) ** 2)


def lobatto(lo, hi):
    """Chebyshev-Lobatto points of [lo, hi], ascending."""
    return 0.5 * (lo + hi) - 0.5 * (hi - lo) * np.cos(np.pi * np.arange(K) / (K - 1))


def interp_root(x, g):
    """Root of the polynomial interpolant through (x, g) between the nodes that
    straddle 0 (barycentric form with exact weights)."""
    w = np.array([1.0 / np.prod([x[m] - x[n] for n in range(K) if n != m]) for m in range(K)])

    def p(t):
        d = t - x
        if np.any(d == 0.0):
            return g[np.argmin(np.abs(d))]
        q = w / d
        return np.sum(q * g) / np.sum(q)

    j = int(np.max(np.nonzero(g < 0.0)[0]))
    return brentq(p, x[j], x[j + 1], xtol=1e-15, rtol=1e-15)


def spectra(kind, rng, n=4000):
    """|H_b|^2 spread over many decades (heavy blur), with zero bins, or narrow."""
    if kind == "wide":
        a = 10.0 ** rng.uniform(-12, 0, n)
    elif kind == "zeros":
        a = np.concatenate([np.zeros(n // 10), 10.0 ** rng.uniform(-8, 0, n)])
    else:
        a = 10.0 ** rng.uniform(-3, -2, n)
    return a, rng.exponential(1.0, a.size)


def worst_root_error(kind, ratio, log_space, trials=12, seed=0):
    rng = np.random.default_rng(seed)
    a, r = spectra(kind, rng)
    worst = 0.0
    for _ in range(trials):
        c = 10.0 ** rng.uniform(-9, -1)
        lo, hi = c / np.sqrt(ratio), c * np.sqrt(ratio)
        root = np.exp(rng.uniform(np.log(lo), np.log(hi)))
        T = f(root, a, r)  # the target that makes `root` the answer
        if log_space:
            t = lobatto(np.log(lo), np.log(hi))
            g = np.array([f(np.exp(v), a, r) / T - 1.0 for v in t])
            est = np.exp(interp_root(t, g))
        else:
            x = lobatto(lo, hi)
            g = np.array([f(v, a, r) / T - 1.0 for v in x])
            est = interp_root(x, g)
        worst = max(worst, abs(est / root - 1.0))
    return worst


@pytest.mark.parametrize("kind", ["wide", "zeros", "narrow"])
def test_log_space_nodes_resolve_ratio_4_brackets(kind):
    # the interpolated brackets of the GPU procedure: ratio <= 4
    assert worst_root_error(kind, 4.0, log_space=True) < 1e-9


@pytest.mark.parametrize("kind", ["wide", "zeros"])
def test_lambda_space_nodes_do_not(kind):
    # the same 12 nodes placed in lambda fall far short of the 1e-6 tolerance
    # on ratio 4 (poles of f at lambda = -|H_b|^2 next to the bracket)
    assert worst_root_error(kind, 4.0, log_space=False) > 1e-7


@pytest.mark.parametrize("kind", ["wide", "zeros", "narrow"])
def test_eight_nodes_resolve_the_narrow_first_brackets(kind):
    # from the sixth iteration on the first pass of an iteration takes 8
    # nodes on [c / 1.25, 1.25 c] (ratio 1.56) about the extrapolated lambda
    global K
    saved, K = K, 8
    try:
        assert worst_root_error(kind, 1.5625, log_space=True, trials=30) < 1e-9
    finally:
        K = saved


def test_log_space_error_shrinks_with_the_bracket():
    e4 = worst_root_error("zeros", 4.0, log_space=True)
    e16 = worst_root_error("zeros", 16.0, log_space=True)
    assert e4 < e16
