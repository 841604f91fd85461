"""Pins of the oracle's gradient of the unrolled method (oracle/adjoint.py)
against FP64 central finite differences of the oracle's own forward solve
(a different computation: no chain rule, no implicit derivative of lambda)."""
import numpy as np
import pytest

import oracle as O
import synthetic as S
from oracle import adjoint as A

RTOL = 1e-4  # configs' gradient check: relative error <= 1e-4


def fd(fun, x0, v, delta):
    return (fun(x0 + delta * v) - fun(x0 - delta * v)) / (2.0 * delta)


def problem(M, k, psf_sigma, noise, w, eps, iters, seed):
    rng = np.random.default_rng(seed)
    u0 = S.image_polygons(seed, M, M, n_poly=6, texture_std=0.02, rng=rng)
    h = S.psf_gaussian(k, psf_sigma)
    y = S.blur_circular(u0, h) + noise * rng.standard_normal((M, M))
    return y, h, noise, w, eps, iters, u0


def test_guided_filter_backward_matches_finite_differences():
    rng = np.random.default_rng(1)
    I = rng.random((9, 8))
    p = I + 0.1 * rng.standard_normal((9, 8))
    gu = rng.standard_normal((9, 8))
    w, eps = 3, 1e-2

    def L(I_, p_, e_):
        return float(np.sum(gu * O.guided_filter(I_, p_, w, e_)))

    gI, gp, geps = A.guided_filter_backward(I, p, w, eps, gu)
    vI, vp = rng.standard_normal(I.shape), rng.standard_normal(p.shape)
    assert np.sum(gI * vI) == pytest.approx(fd(lambda x: L(x, p, eps), I, vI, 1e-6), rel=1e-7)
    assert np.sum(gp * vp) == pytest.approx(fd(lambda x: L(I, x, eps), p, vp, 1e-6), rel=1e-7)
    assert geps == pytest.approx(fd(lambda e: L(I, p, e), eps, 1.0, 1e-7), rel=1e-6)


@pytest.fixture(scope="module")
def small():
    """16 x 16, 5 x 5 Gaussian PSF, 3 iterations (lambda finite throughout)."""
    args = problem(16, 5, 1.0, 0.01, 3, 1e-3, 3, 5)
    r = A.solve_with_grad(*args)
    assert all(np.isfinite(r["lam"]))
    return args, r


def test_gradient_eps_small(small):
    (y, h, s, w, eps, K, uc), r = small
    num = fd(lambda e: A.loss_only(y, h, s, w, e, K, uc), eps, 1.0, 1e-7)
    assert r["g_eps"] == pytest.approx(num, rel=1e-6)


def test_gradient_every_psf_entry_small(small):
    (y, h, s, w, eps, K, uc), r = small
    for i in range(h.shape[0]):
        for j in range(h.shape[1]):
            e = np.zeros_like(h)
            e[i, j] = 1.0
            num = fd(lambda x: A.loss_only(y, x, s, w, eps, K, uc), h, e, 1e-7)
            assert r["g_h"][i, j] == pytest.approx(num, rel=1e-5, abs=1e-12), (i, j)


def test_gradient_observation_directions_small(small):
    (y, h, s, w, eps, K, uc), r = small
    rng = np.random.default_rng(2)
    for _ in range(3):
        v = rng.standard_normal(y.shape)
        num = fd(lambda x: A.loss_only(x, h, s, w, eps, K, uc), y, v, 1e-6)
        assert np.sum(r["g_y"] * v) == pytest.approx(num, rel=1e-6)


def test_gradient_64_crop_of_the_differentiation_workload():
    """The differentiation workload's settings on a 64 x 64 crop: 25 x 25
    Gaussian PSF (sigma 1.6), noise 1/255, w = 7, eps = 1e-3, 10 iterations;
    eps, 5 PSF entries and 3 observation directions to 1e-4 relative."""
    y, h, s, w, eps, K, uc = problem(64, 25, 1.6, 1.0 / 255.0, 7, 1e-3, 10, 11)
    r = A.solve_with_grad(y, h, s, w, eps, K, uc)
    assert all(np.isfinite(r["lam"]))
    num = fd(lambda e: A.loss_only(y, h, s, w, e, K, uc), eps, 1.0, 1e-7)
    assert r["g_eps"] == pytest.approx(num, rel=RTOL)
    # entries well above the step (|h| has no derivative at 0, where Eq. 12 uses sum |h|)
    for (i, j) in ((12, 12), (12, 13), (10, 15), (8, 12), (16, 9)):
        e = np.zeros_like(h)
        e[i, j] = 1.0
        num = fd(lambda x: A.loss_only(y, x, s, w, eps, K, uc), h, e, 1e-7)
        assert r["g_h"][i, j] == pytest.approx(num, rel=RTOL, abs=1e-10), (i, j)
    rng = np.random.default_rng(3)
    for _ in range(3):
        v = rng.standard_normal(y.shape)
        num = fd(lambda x: A.loss_only(x, h, s, w, eps, K, uc), y, v, 1e-6)
        assert np.sum(r["g_y"] * v) == pytest.approx(num, rel=RTOL)


def test_gradient_through_the_infinite_lambda_branch():
    """A trajectory whose first two steps take the lambda = inf branch (u_E
    starts at the clean image, in the feasible set for sigma twice the noise)
    and whose later steps solve Eq. 11: the branch steps pass the gradient
    through the guided filter only."""
    y, h, s, w, eps, K, uc = problem(64, 25, 1.6, 1.0 / 255.0, 7, 1e-3, 4, 11)
    s2 = 2.0 * s
    r = A.solve_with_grad(y, h, s2, w, eps, K, uc, u_init=uc)
    assert np.isinf(r["lam"][0]) and np.isinf(r["lam"][1]) and np.isfinite(r["lam"][2])
    num = fd(lambda e: A.loss_only(y, h, s2, w, e, K, uc, u_init=uc), eps, 1.0, 1e-7)
    assert r["g_eps"] == pytest.approx(num, rel=RTOL)
    rng = np.random.default_rng(4)
    v = rng.standard_normal(y.shape)
    num = fd(lambda x: A.loss_only(x, h, s2, w, eps, K, uc, u_init=uc), y, v, 1e-6)
    assert np.sum(r["g_y"] * v) == pytest.approx(num, rel=RTOL)
    e = np.zeros_like(h)
    e[12, 12] = 1.0
    num = fd(lambda x: A.loss_only(y, x, s2, w, eps, K, uc, u_init=uc), h, e, 1e-7)
    assert r["g_h"][12, 12] == pytest.approx(num, rel=RTOL)
