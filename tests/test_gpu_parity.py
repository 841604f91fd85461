"""GPU parity: every step of the CUDA path, called through the C-ABI, against
the FP64 oracle on the same seeded inputs.

Tolerances:
  u          max-abs 2e-5 on [0, 1] images, per iteration
  lambda     1e-6 relative on a teacher-forced step (the GPU step fed the
             oracle's own u_E^k); along a free trajectory the GPU's u_E drifts
             from the oracle's by up to ~1e-6, which moves lambda by more, so
             free-trajectory lambda is held to 1e-4 relative
  ISNR       0.01 dB
  FFT        relative rms error 1e-6 of the spectrum's norm
  residual   ||h*u_E - y||^2 to 1e-5 relative: it is a noise-level quantity
             (about sigma^2 per pixel) formed from FP32 spectra whose absolute
             error is about eps32 * sqrt(log2 P) * ||u_E||, so a few 1e-6 of
             it is the FP32 floor
Measured errors are appended to parity_metrics.jsonl in the run's output folder.
"""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import oracle as O  # noqa: E402
import synthetic as S  # noqa: E402
import paper_1609_01839_gb300 as gfd  # noqa: E402

DEV = torch.device("cuda:0")
RES_TOL = 1e-5
U_TOL = 2e-5
LAM_TOL_TF = 1e-6
LAM_TOL_FREE = 1e-4
ISNR_TOL = 0.01


@pytest.fixture(scope="module")
def ctx():
    c = gfd.Context(0)
    yield c
    c.close()


def record(name, **vals):
    import json
    import os
    # per-test error figures go to $GFD_ARTIFACT_DIR, default <repo>/artifacts
    d = os.environ.get("GFD_ARTIFACT_DIR") or os.path.join(
        os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "artifacts")
    try:
        os.makedirs(d, exist_ok=True)
        with open(os.path.join(d, "parity_metrics.jsonl"), "a") as f:
            f.write(json.dumps({"test": name, **{k: float(v) for k, v in vals.items()}}) + "\n")
    except OSError:
        pass


def cuda(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(DEV)


def host(t):
    return t.detach().cpu().numpy()


# ---------------------------------------------------------------------------
# 2-D real DFT (Sec. 3.1's diagonalisation)
# ---------------------------------------------------------------------------

def packed_ref(x):
    F = np.fft.fft2(x.astype(np.float64))
    M, N = x.shape
    P = F[:, : N // 2].copy()
    P[:, 0] = F[:, 0] + 1j * F[:, N // 2]
    return P


@pytest.mark.parametrize("M,N", [(8, 8), (16, 32), (64, 16), (32, 128), (256, 256),
                                 (512, 1024), (1024, 512), (4096, 64), (64, 4096), (2048, 2048)])
def test_fft2_r2c_matches_dft(ctx, M, N):
    rng = np.random.default_rng(M * 7 + N)
    x = rng.random((M, N)).astype(np.float32)
    X = host(ctx.fft2_r2c(cuda(x))).astype(np.complex128)
    ref = packed_ref(x)
    rel = np.linalg.norm(X - ref) / np.linalg.norm(ref)
    record(f"fft2_r2c_{M}x{N}", rel_rms=rel)
    assert rel < 1e-6, rel
    # c2r inverts it
    back = host(ctx.fft2_c2r(cuda(ref.astype(np.complex64))))
    assert np.abs(back - x).max() < 2e-6


# ---------------------------------------------------------------------------
# Guided filter (Sec. 2, Eq. 3-5)
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("M,N,w,eps", [(8, 8, 9, 1e-3), (16, 32, 3, 1e-3), (64, 64, 1, 1e-3),
                                       (64, 128, 5, 1e-3), (256, 256, 7, 1e-3),
                                       (256, 512, 9, 1e-4), (128, 128, 17, 1e-2),
                                       (32, 2048, 11, 1e-3)])
def test_guided_filter_matches_oracle(ctx, M, N, w, eps):
    rng = np.random.default_rng(M + N + w)
    u0 = S.image_polygons(3, M, N, n_poly=8, texture_std=0.02, rng=rng)
    I = (u0 + 0.01 * rng.standard_normal((M, N))).astype(np.float32)
    p = (u0 + 0.03 * rng.standard_normal((M, N))).astype(np.float32)
    got = host(ctx.guidfilter(cuda(I), cuda(p), w, eps))
    ref = O.guided_filter(I, p, w, eps)
    record(f"guided_filter_{M}x{N}_w{w}_eps{eps}", max_abs=np.abs(got - ref).max())
    assert np.abs(got - ref).max() < U_TOL


def test_guided_filter_constant_fixed_point(ctx):
    c = torch.full((64, 64), 0.37, device=DEV)
    out = host(ctx.guidfilter(c, c, 7, 1e-3))
    assert np.abs(out - 0.37).max() < 1e-6


# ---------------------------------------------------------------------------
# Teacher-forced single iterations: the GPU step from the oracle's u_E^k
# ---------------------------------------------------------------------------

@pytest.fixture(scope="module")
def c0_trace():
    p = S.config_c0()
    return p, O.solve(p.y, p.h, p.sigma, p.w, p.eps, p.iters, u_orig=p.u_orig, trace=True)


@pytest.fixture(scope="module")
def c1_trace():
    p = S.config_c1()
    return p, O.solve(p.y, p.h, p.sigma, p.w, p.eps, p.iters, u_orig=p.u_orig, trace=True)


def gpu_step(ctx, p, uE):
    items = [{"y": cuda(p.y), "h": cuda(p.h), "sigma": p.sigma, "w": p.w, "eps": p.eps,
              "u_init": cuda(uE.astype(np.float32))}]
    ctx.solve_batched(items, 1, want_res=True, want_uIp=True)
    torch.cuda.synchronize()
    it = items[0]
    return (float(host(it["lam"])[0]), float(host(it["res"])[0]), host(it["u"]),
            host(it["uI"]), host(it["up"]))


def oracle_step(p, uE):
    M, N = p.shape
    H = O.psf_spectrum(p.h, M, N)
    Y = np.fft.fft2(p.y.astype(np.float64))
    T = O.discrepancy_target(p.y, p.h, p.sigma)
    uE32 = uE.astype(np.float32).astype(np.float64)
    return O.iterate(H, Y, O.grad_weight(M, N), uE32, T, p.w, p.eps)


@pytest.mark.parametrize("k", [0, 1, 2, 5, 9])
def test_teacher_forced_step_c0(ctx, c0_trace, k):
    p, tr = c0_trace
    lam, res, u, uI, up = gpu_step(ctx, p, tr["uE"][k])
    ref = oracle_step(p, tr["uE"][k])
    record(f"teacher_forced_c0_k{k}", lam_rel=abs(lam / ref["lam"] - 1), res_rel=abs(res / ref["res"] - 1),
           u_max_abs=np.abs(u - ref["u"]).max(), uI_max_abs=np.abs(uI - ref["uI"]).max(),
           up_max_abs=np.abs(up - ref["up"]).max())
    assert res == pytest.approx(ref["res"], rel=RES_TOL)
    if math.isinf(ref["lam"]):
        assert math.isinf(lam)
    else:
        assert abs(lam / ref["lam"] - 1) < LAM_TOL_TF, (lam, ref["lam"])
    assert np.abs(up - ref["up"]).max() < U_TOL
    assert np.abs(uI - ref["uI"]).max() < U_TOL
    assert np.abs(u - ref["u"]).max() < U_TOL


@pytest.mark.parametrize("k", [0, 1, 2, 10, 19])
def test_teacher_forced_step_c1(ctx, c1_trace, k):
    p, tr = c1_trace
    lam, res, u, uI, up = gpu_step(ctx, p, tr["uE"][k])
    ref = oracle_step(p, tr["uE"][k])
    record(f"teacher_forced_c1_k{k}", lam_rel=abs(lam / ref["lam"] - 1), res_rel=abs(res / ref["res"] - 1),
           u_max_abs=np.abs(u - ref["u"]).max(), uI_max_abs=np.abs(uI - ref["uI"]).max(),
           up_max_abs=np.abs(up - ref["up"]).max())
    assert res == pytest.approx(ref["res"], rel=RES_TOL)
    assert abs(lam / ref["lam"] - 1) < LAM_TOL_TF, (lam, ref["lam"])
    assert np.abs(u - ref["u"]).max() < U_TOL


def lambda_condition(p, uE, lam):
    """kappa = 1 / |d ln f / d ln lambda| at the root of Eq. 11 (FP64)."""
    M, N = p.shape
    H = O.psf_spectrum(p.h, M, N)
    UE = np.fft.fft2(uE.astype(np.float32).astype(np.float64))
    Y = np.fft.fft2(p.y.astype(np.float64))
    a, r = np.abs(H) ** 2, np.abs(H * UE - Y) ** 2
    fp, fm = O.f_lambda(lam * 1.001, a, r, M * N), O.f_lambda(lam / 1.001, a, r, M * N)
    return 1.0 / abs((math.log(fp) - math.log(fm)) / (2 * math.log(1.001)))


# Bound on the relative error of the GPU's f(lambda_j) = (1/P) sum over bins
# of lambda_j^2 r / (a + lambda_j)^2.  H and Y come from a double-float
# transform (rounded once), the sums are double-float / FP64; what remains is
# the FP32 transform of u_E in every iteration, whose rounding leaves f off by
# ~2e-9 relative at most on the workloads tested (the errors of single bins
# average out; a small systematic part does not).  The root then moves by
# about kappa times that, kappa = 1 / |d ln f / d ln lambda|.
F_REL_ERR = 1e-8


@pytest.fixture(scope="module")
def c2_118_trace():
    """A heavily blurred canvas (25x25 Gaussian, sigma 2.7, BSNR 30) whose
    discrepancy function is nearly flat in lambda from the fifth iteration on
    (d ln f / d ln lambda ~ 3e-6): almost every bin has |H|^2 << lambda."""
    p = S.config_c2_image(118, iters=9)
    return p, O.solve(p.y, p.h, p.sigma, p.w, p.eps, 9, trace=True)


@pytest.mark.parametrize("k", [3, 8])
def test_teacher_forced_step_ill_conditioned_lambda(ctx, c2_118_trace, k):
    """lambda within kappa * F_REL_ERR (and never worse than 1e-6 where the
    root is well conditioned); u, u_I, u_p within 2e-5 regardless: the
    solves depend on lambda only through the bins with |H|^2 ~ lambda."""
    p, tr = c2_118_trace
    lam, res, u, uI, up = gpu_step(ctx, p, tr["uE"][k])
    ref = oracle_step(p, tr["uE"][k])
    kappa = lambda_condition(p, tr["uE"][k], ref["lam"])
    tol = max(LAM_TOL_TF, kappa * F_REL_ERR)
    record(f"teacher_forced_c2_118_k{k}", lam_rel=abs(lam / ref["lam"] - 1), kappa=kappa,
           res_rel=abs(res / ref["res"] - 1), u_max_abs=np.abs(u - ref["u"]).max(),
           uI_max_abs=np.abs(uI - ref["uI"]).max(), up_max_abs=np.abs(up - ref["up"]).max())
    assert res == pytest.approx(ref["res"], rel=RES_TOL)
    assert abs(lam / ref["lam"] - 1) < tol, (lam, ref["lam"], kappa)
    assert np.abs(uI - ref["uI"]).max() < U_TOL
    assert np.abs(up - ref["up"]).max() < U_TOL
    assert np.abs(u - ref["u"]).max() < U_TOL


@pytest.fixture(scope="module")
def c4_two_steps():
    """One 4096 x 4096 image of the bandwidth-stress workload (31 x 31 motion
    blur, BSNR 35, w = 9, eps = 1e-4) and the oracle's first two iterates."""
    p = S.config_c4_image(0, iters=2)
    return p, O.solve(p.y, p.h, p.sigma, p.w, p.eps, 2, trace=True)


@pytest.mark.parametrize("k", [0, 1])
def test_teacher_forced_step_4096(ctx, c4_two_steps, k):
    """Full-size canvas (every pass at its largest tile shapes): one GPU step
    from the oracle's u_E^k against the oracle's step, element by element."""
    p, tr = c4_two_steps
    lam, res, u, uI, up = gpu_step(ctx, p, tr["uE"][k])
    ref = oracle_step(p, tr["uE"][k])
    kappa = lambda_condition(p, tr["uE"][k], ref["lam"])
    record(f"teacher_forced_c4_k{k}", lam_rel=abs(lam / ref["lam"] - 1), kappa=kappa,
           res_rel=abs(res / ref["res"] - 1), u_max_abs=np.abs(u - ref["u"]).max(),
           uI_max_abs=np.abs(uI - ref["uI"]).max(), up_max_abs=np.abs(up - ref["up"]).max())
    assert res == pytest.approx(ref["res"], rel=RES_TOL)
    assert abs(lam / ref["lam"] - 1) < max(LAM_TOL_TF, kappa * F_REL_ERR), (lam, ref["lam"], kappa)
    assert np.abs(uI - ref["uI"]).max() < U_TOL
    assert np.abs(up - ref["up"]).max() < U_TOL
    assert np.abs(u - ref["u"]).max() < U_TOL


# ---------------------------------------------------------------------------
# Free trajectories of the whole method (Steps 0-3)
# ---------------------------------------------------------------------------

def check_trajectory(ctx, p, tr, iters):
    u, lam, isnr = ctx.solve(cuda(p.y), cuda(p.h), p.sigma, p.w, p.eps, iters,
                             u_orig=cuda(p.u_orig))
    torch.cuda.synchronize()
    lam, isnr, u = host(lam), host(isnr), host(u)
    fin = [k for k in range(iters) if math.isfinite(tr["lam"][k])]
    record(f"trajectory_{p.meta['name']}", u_max_abs=np.abs(u - tr["u"]).max(),
           lam_rel_max=max([abs(lam[k] / tr["lam"][k] - 1) for k in fin] or [0.0]),
           isnr_abs_max=max(abs(isnr[k] - tr["isnr"][k]) for k in range(iters)))
    for k in range(iters):
        if math.isinf(tr["lam"][k]):
            assert math.isinf(lam[k])
        else:
            assert abs(lam[k] / tr["lam"][k] - 1) < LAM_TOL_FREE, (k, lam[k], tr["lam"][k])
        assert abs(isnr[k] - tr["isnr"][k]) < ISNR_TOL, (k, isnr[k], tr["isnr"][k])
    assert np.abs(u - tr["u"]).max() < U_TOL
    assert ctx.status(1)[0] & ~gfd.STATUS_NONCONVERGED == 0


def test_trajectory_c0(ctx, c0_trace):
    p, tr = c0_trace
    check_trajectory(ctx, p, tr, p.iters)


def test_trajectory_c1(ctx, c1_trace):
    p, tr = c1_trace
    check_trajectory(ctx, p, tr, p.iters)


def test_every_iterate_c0(ctx, c0_trace):
    """u^k within tolerance at every iteration k (solves of 1..K iterations)."""
    p, tr = c0_trace
    for k in range(1, p.iters + 1):
        u, _, _ = ctx.solve(cuda(p.y), cuda(p.h), p.sigma, p.w, p.eps, k)
        torch.cuda.synchronize()
        assert np.abs(host(u) - tr["u_k"][k - 1]).max() < U_TOL, k


# ---------------------------------------------------------------------------
# Batched execution (uneven sizes) equals the plain path and the oracle
# ---------------------------------------------------------------------------

def c2_subset():
    # images of every canvas / PSF / window class, in index order
    return [S.config_c2_image(i, iters=15) for i in (0, 1, 2, 3, 4, 5, 6, 7)]


def test_batched_equals_plain_and_oracle(ctx):
    """A batched image runs the same arithmetic as the plain solve except for
    the order of the partial sums of Eq. 11 (which depends on how the image's
    tiles are split across blocks), so lambda agrees to ~1e-7 relative and u
    to a few 1e-6; both are checked against the oracle as well."""
    probs = c2_subset()
    iters = 4
    items = [{"y": cuda(p.y), "h": cuda(p.h), "sigma": p.sigma, "w": p.w, "eps": p.eps,
              "u_orig": cuda(p.u_orig)} for p in probs]
    ctx.solve_batched(items, iters)
    torch.cuda.synchronize()
    for p, it in zip(probs, items):
        u1, lam1, isnr1 = ctx.solve(cuda(p.y), cuda(p.h), p.sigma, p.w, p.eps, iters,
                                    u_orig=cuda(p.u_orig))
        torch.cuda.synchronize()
        assert np.abs(host(it["u"]) - host(u1)).max() < 1e-5
        np.testing.assert_allclose(host(it["lam"]), host(lam1), rtol=1e-5)
    for p, it in list(zip(probs, items))[:4]:
        ref = O.solve(p.y, p.h, p.sigma, p.w, p.eps, iters, u_orig=p.u_orig)
        assert np.abs(host(it["u"]) - ref["u"]).max() < U_TOL
        np.testing.assert_allclose(host(it["isnr"]), ref["isnr"], atol=ISNR_TOL)


def test_batched_host_entry_point(ctx):
    probs = c2_subset()[:3]
    iters = 3
    dev_items = [{"y": cuda(p.y), "h": cuda(p.h), "sigma": p.sigma, "w": p.w, "eps": p.eps,
                  "u_orig": cuda(p.u_orig)} for p in probs]
    ctx.solve_batched(dev_items, iters)
    torch.cuda.synchronize()
    host_items = [{"y": torch.from_numpy(p.y).pin_memory(), "h": torch.from_numpy(p.h).pin_memory(),
                   "sigma": p.sigma, "w": p.w, "eps": p.eps,
                   "u_orig": torch.from_numpy(p.u_orig).pin_memory()} for p in probs]
    arr = ctx.make_host_images(host_items, iters)
    ctx.solve_batched_host_images(arr, iters)
    for d, h in zip(dev_items, host_items):
        assert np.abs(host(d["u"]) - h["u"].numpy()).max() < 1e-6
        np.testing.assert_allclose(h["isnr"].numpy(), host(d["isnr"]), atol=1e-6)


def test_batched_host_entry_point_with_start_values(ctx):
    """Host buffers with u_init (the start values must reach u before any
    chain of the solve reads them) and pageable inputs (the path that copies
    outside the graph) both match the device-buffer solve."""
    probs = c2_subset()[3:6]
    iters = 2
    rng = np.random.default_rng(5)
    starts = [rng.random(p.shape, dtype=np.float64).astype(np.float32) for p in probs]
    dev_items = [{"y": cuda(p.y), "h": cuda(p.h), "sigma": p.sigma, "w": p.w, "eps": p.eps,
                  "u_init": cuda(u0)} for p, u0 in zip(probs, starts)]
    ctx.solve_batched(dev_items, iters)
    torch.cuda.synchronize()
    for pin in (True, False):
        mk = (lambda a: torch.from_numpy(a).pin_memory()) if pin else (lambda a: torch.from_numpy(a.copy()))
        host_items = [{"y": mk(p.y), "h": mk(p.h), "sigma": p.sigma, "w": p.w, "eps": p.eps,
                       "u_init": mk(u0)} for p, u0 in zip(probs, starts)]
        if not pin:
            for h in host_items:
                h["u"] = torch.empty(h["y"].shape, dtype=torch.float32)
        arr = ctx.make_host_images(host_items, iters)
        ctx.solve_batched_host_images(arr, iters)
        for d, h in zip(dev_items, host_items):
            assert np.abs(host(d["u"]) - h["u"].numpy()).max() < 1e-6, pin
            np.testing.assert_allclose(h["lam"].numpy(), host(d["lam"]), rtol=1e-12)


# ---------------------------------------------------------------------------
# Edge cases
# ---------------------------------------------------------------------------

def test_lambda_infinite_branch(ctx):
    """sigma so large that u_E = 0 already meets the discrepancy bound:
    lambda = inf (Sec. 3.2) and u stays 0 (guidfilter(0, 0) = 0)."""
    p = S.config_c0(M=32, N=32)
    sigma = 10.0
    ref = O.solve(p.y, p.h, sigma, p.w, p.eps, 2)
    assert all(math.isinf(l) for l in ref["lam"])
    u, lam, _ = ctx.solve(cuda(p.y), cuda(p.h), sigma, p.w, p.eps, 2)
    torch.cuda.synchronize()
    assert np.all(np.isinf(host(lam)))
    assert np.abs(host(u) - ref["u"]).max() < 1e-7


@pytest.mark.parametrize("M,N,w,k", [(8, 8, 9, 3), (8, 16, 3, 5), (16, 64, 5, 9), (128, 32, 7, 15),
                                     (4096, 64, 5, 9), (64, 4096, 9, 15), (2048, 128, 3, 5)])
def test_small_and_nonsquare(ctx, M, N, w, k):
    rng = np.random.default_rng(M * N + w)
    u0 = S.image_polygons(11, M, N, n_poly=3, texture_std=0.02, rng=rng)
    h = S.psf_gaussian(k, 1.2)
    yb = S.blur_circular(u0, h)
    sigma = 0.01
    y = (yb + sigma * rng.standard_normal((M, N))).astype(np.float32)
    h32 = h.astype(np.float32)
    ref = O.solve(y, h32, sigma, w, 1e-3, 3)
    u, lam, _ = ctx.solve(cuda(y), cuda(h32), sigma, w, 1e-3, 3)
    torch.cuda.synchronize()
    assert np.abs(host(u) - ref["u"]).max() < U_TOL
    for a, b in zip(host(lam), ref["lam"]):
        assert (math.isinf(a) and math.isinf(b)) or abs(a / b - 1) < LAM_TOL_FREE


def test_zero_iterations_returns_start(ctx):
    p = S.config_c0(M=64, N=64)
    u0 = np.full((64, 64), 0.25, dtype=np.float32)
    u, _, _ = ctx.solve(cuda(p.y), cuda(p.h), p.sigma, p.w, p.eps, 0, u_init=cuda(u0))
    torch.cuda.synchronize()
    assert np.all(host(u) == 0.25)


def test_invalid_arguments_rejected(ctx):
    y = torch.zeros((64, 64), device=DEV)
    h = torch.ones((3, 3), device=DEV) / 9
    with pytest.raises(gfd.GfdError) as e:
        ctx.solve(torch.zeros((48, 64), device=DEV), h, 0.01, 3, 1e-3, 1)
    assert e.value.code == -2
    with pytest.raises(gfd.GfdError) as e:
        ctx.solve(y, h, 0.01, 4, 1e-3, 1)          # even window
    assert e.value.code == -1
    with pytest.raises(gfd.GfdError) as e:
        ctx.solve(y, h, 0.01, 3, -1.0, 1)          # eps <= 0
    assert e.value.code == -1
    with pytest.raises(gfd.GfdError) as e:
        ctx.solve(y, h, float("nan"), 3, 1e-3, 1)  # non-finite sigma
    assert e.value.code == -3
    with pytest.raises(gfd.GfdError):
        ctx.solve(y, torch.ones((2, 3), device=DEV), 0.01, 3, 1e-3, 1)  # even PSF
    with pytest.raises(ValueError):
        ctx.solve(y.cpu(), h, 0.01, 3, 1e-3, 1)    # no CPU path


def test_bad_psf_reported_in_status(ctx):
    y = torch.rand((32, 32), device=DEV)
    h = -torch.ones((3, 3), device=DEV) / 9
    ctx.solve(y, h, 0.01, 3, 1e-3, 1)
    st = ctx.status(1)[0]
    assert st & gfd.STATUS_BAD_PSF


def test_launch_count_reported(ctx):
    p = S.config_c0(M=64, N=64)
    ctx.solve(cuda(p.y), cuda(p.h), p.sigma, p.w, p.eps, 2)
    torch.cuda.synchronize()
    assert ctx.last_launch_count() > 10
