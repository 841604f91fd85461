"""GPU parity: every step of the CUDA path, called through the C-ABI, against
the FP64 oracle on the same seeded inputs.

Tolerances:
  u          max-abs 2e-5 on [0, 1] images, per iteration
  lambda     1e-6 relative on a teacher-forced step (the GPU step fed the
             oracle's own u_E^k), max(1e-6, kappa * 1e-8) where the root of
             Eq. 11 is ill-conditioned (kappa = 1 / |d ln f / d ln lambda|);
             along a free trajectory, at every iteration: against the
             oracle's lambda at the GPU's own iterate with the same bound, and
             against the oracle's own trajectory with
             max(1e-6, 2 kappa (df + 1e-8)), df the measured change of f at
             the oracle's root between the two iterates (tests/oracle_runs.py)
  ISNR       0.01 dB
  FFT        relative rms error 1e-6 of the spectrum's norm
  residual   ||h*u_E - y||^2 to 1e-5 relative: it is a noise-level quantity
             (about sigma^2 per pixel) formed from FP32 spectra whose absolute
             error is about eps32 * sqrt(log2 P) * ||u_E||, so a few 1e-6 of
             it is the FP32 floor
Measured errors are appended to parity_metrics.jsonl in the run's output folder.
"""
import math
import multiprocessing as mp
import os

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import oracle as O  # noqa: E402
import synthetic as S  # noqa: E402
import paper_1609_01839_gb300 as gfd  # noqa: E402
import oracle_runs  # noqa: E402

DEV = torch.device("cuda:0")
RES_TOL = 1e-5
U_TOL = 2e-5
LAM_TOL_TF = 1e-6
ISNR_TOL = 0.01


@pytest.fixture(scope="module")
def ctx():
    c = gfd.Context(0)
    yield c
    c.close()


@pytest.fixture(scope="module")
def pool():
    """Worker processes for the oracle (spawned: no CUDA state is inherited)."""
    n = max(1, min(16, os.cpu_count() or 1))
    with mp.get_context("spawn").Pool(n) as pl:
        yield pl


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


def lambda_tolerance(kappa, res_rel):
    """max(1e-6, 2 kappa max(dres, 1e-8)): the GPU's f(lambda) carries the
    FP32 rounding of the spectra, which the residual f(inf) exposes as its
    relative error dres; the root moves by kappa times the relative error of f
    (tests/oracle_runs.py)."""
    return max(LAM_TOL_TF, 2.0 * kappa * max(res_rel, 1e-8))


@pytest.fixture(scope="module")
def c2_118_trace():
    """A heavily blurred canvas (25x25 Gaussian, sigma 2.7, BSNR 30) whose
    discrepancy function is nearly flat in lambda from the fifth iteration on
    (d ln f / d ln lambda ~ 3e-6): almost every bin has |H|^2 << lambda."""
    p = S.config_c2_image(118, iters=9)
    return p, O.solve(p.y, p.h, p.sigma, p.w, p.eps, 9, trace=True)


@pytest.mark.parametrize("k", [3, 8])
def test_teacher_forced_step_ill_conditioned_lambda(ctx, c2_118_trace, k):
    """lambda within lambda_tolerance (1e-6 where the root is well
    conditioned); u, u_I, u_p within 2e-5 regardless: the
    solves depend on lambda only through the bins with |H|^2 ~ lambda."""
    p, tr = c2_118_trace
    lam, res, u, uI, up = gpu_step(ctx, p, tr["uE"][k])
    ref = oracle_step(p, tr["uE"][k])
    kappa = lambda_condition(p, tr["uE"][k], ref["lam"])
    tol = lambda_tolerance(kappa, abs(res / ref["res"] - 1))
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
    assert abs(lam / ref["lam"] - 1) < lambda_tolerance(kappa, abs(res / ref["res"] - 1)), \
        (lam, ref["lam"], kappa)
    assert np.abs(uI - ref["uI"]).max() < U_TOL
    assert np.abs(up - ref["up"]).max() < U_TOL
    assert np.abs(u - ref["u"]).max() < U_TOL


# ---------------------------------------------------------------------------
# Free trajectories of the whole method (Steps 0-3), every iteration
# ---------------------------------------------------------------------------

def gpu_trajectory(ctx, probs, iters, tmp, tag):
    """The batched solve of ``probs`` for ``iters`` iterations (per-iteration
    lambda, ISNR, residual) and its iterates u^1..u^iters (solves of 1..iters
    iterations are the same computation cut short), saved as float32 .npy
    files.  Returns one oracle_runs job per image."""
    def make():
        return [{"y": cuda(p.y), "h": cuda(p.h), "sigma": p.sigma, "w": p.w, "eps": p.eps,
                 "u_orig": cuda(p.u_orig)} for p in probs]
    full = make()
    ctx.solve_batched(full, iters, want_res=True)
    torch.cuda.synchronize()
    paths = [[None] * iters for _ in probs]
    for k in range(1, iters):
        its = make()
        ctx.solve_batched(its, k)
        torch.cuda.synchronize()
        for i, it in enumerate(its):
            paths[i][k - 1] = str(tmp / f"{tag}_{i}_{k}.npy")
            np.save(paths[i][k - 1], host(it["u"]))
    for i, it in enumerate(full):
        paths[i][iters - 1] = str(tmp / f"{tag}_{i}_{iters}.npy")
        np.save(paths[i][iters - 1], host(it["u"]))
    return [{"p": p, "iters": iters, "lam": host(it["lam"]).tolist(),
             "isnr": host(it["isnr"]).tolist(), "res": host(it["res"]).tolist(),
             "paths": paths[i]} for i, (p, it) in enumerate(zip(probs, full))]


def assert_trajectory(name, m, status=None):
    """Every iteration: the GPU step within 2e-5 max-abs of the oracle step
    from the same iterate with the same lambda; the trajectory within
    max(2e-5, sum of the per-step errors so far) of the lambda-forced oracle
    trajectory, and within 2e-5 of both oracle trajectories where Eq. 11's
    root is well conditioned (kappa <= 1e4); ISNR within 0.01 dB; lambda
    within the kappa-derived bounds; the same branch of Sec. 3.2; residual
    within 1e-5 relative (tests/oracle_runs.py derives the bounds)."""
    K = len(m["u_err"])
    kmax = max(m["kappa"] or [0.0])
    record(name, u_max_abs=max(m["u_err"]), u_max_abs_lambda_forced=max(m["u_err_forced"]),
           u_max_abs_step=max(m["u_err_step"]), isnr_abs_max=max(m["isnr_err"] or [0.0]),
           lam_rel_free_max=max(m["lam_rel_free"]), lam_rel_tf_max=max(m["lam_rel_tf"]),
           kappa_max=kmax, res_rel_max=max(m["res_rel"]),
           free_over_tol=max(a / t for a, t in zip(m["lam_rel_free"], m["tol_free"])),
           tf_over_tol=max(a / t for a, t in zip(m["lam_rel_tf"], m["tol_tf"])))
    well = kmax <= oracle_runs.KAPPA_FREE_U
    for k in range(K):
        assert m["branch_gpu"][k] == m["branch_ref"][k], (name, k)
        assert m["res_rel"][k] < RES_TOL, (name, k, m["res_rel"][k])
        assert m["lam_rel_tf"][k] <= m["tol_tf"][k], (name, k, m["lam_rel_tf"][k], m["tol_tf"][k])
        assert m["lam_rel_free"][k] <= m["tol_free"][k], (name, k, m["lam_rel_free"][k],
                                                          m["tol_free"][k], m["kappa"][k], m["df"][k])
        assert m["u_err_step"][k] < U_TOL, (name, k, m["u_err_step"][k])
        forced_tol = U_TOL if well else m["drift_tol"][k]
        assert m["u_err_forced"][k] < forced_tol, (name, k, m["u_err_forced"][k], forced_tol)
        if well:
            assert m["u_err"][k] < U_TOL, (name, k, m["u_err"][k])
        if m["isnr_err"]:
            assert m["isnr_err_forced"][k] < ISNR_TOL, (name, k, m["isnr_err_forced"][k])
            assert m["isnr_err"][k] < ISNR_TOL, (name, k, m["isnr_err"][k])
    if status is not None:
        expect = gfd.STATUS_NONCONVERGED if any(m["flag_ref"]) else 0
        assert status == expect, (name, status, m["flag_ref"])


def test_trajectory_c0(ctx, pool, tmp_path):
    p = S.config_c0()
    jobs = gpu_trajectory(ctx, [p], p.iters, tmp_path, "c0")
    st = ctx.status(1)[0]
    assert_trajectory("trajectory_c0", pool.map(oracle_runs.compare_trajectory, jobs)[0], st)


def test_trajectory_c1(ctx, pool, tmp_path):
    p = S.config_c1()
    jobs = gpu_trajectory(ctx, [p], p.iters, tmp_path, "c1")
    st = ctx.status(1)[0]
    assert_trajectory("trajectory_c1", pool.map(oracle_runs.compare_trajectory, jobs)[0], st)


# One image of every (canvas, PSF, window) class of the 256-image batch (4 x 3
# x 3 = 36 classes; the first image of each class in batch order) and image
# 118, the ill-conditioned one (25 x 25 Gaussian, sigma 2.7, BSNR 30).
C2_COVER = (7, 35, 70, 0, 95, 47, 79, 51, 13, 8, 5, 3, 87, 23, 50, 40, 32, 167, 10, 9, 4, 14,
            2, 83, 33, 25, 29, 22, 49, 64, 57, 42, 1, 17, 41, 31, 118)


def test_c2_cover_is_every_class():
    seen = set()
    for i in C2_COVER:
        p = S.config_c2_image(i, iters=1)
        seen.add((p.shape, p.true_shape, p.meta["psf"], p.w))
    assert len(seen) == 36


def test_batched_trajectories_every_class(ctx, pool, tmp_path):
    """The batched solve (one graph over uneven sizes) of C2_COVER for all 15
    iterations against the oracle, image by image, at every iteration."""
    probs = pool.map(oracle_runs.make_c2_image, C2_COVER)
    jobs = gpu_trajectory(ctx, probs, 15, tmp_path, "c2")
    st = ctx.status(len(probs))
    res = pool.map(oracle_runs.compare_trajectory, jobs, chunksize=1)
    for i, m, s_ in zip(C2_COVER, res, st):
        assert_trajectory(f"batched_trajectory_c2_{i}", m, s_)


def test_table1_settings_trajectories(ctx, pool, tmp_path):
    """The paper's five experiment settings (Sec. 4, Table 1 PSFs and noise
    levels; eps = 7.5e-4, w = 3, 30 iterations) on synthetic 256^2 images,
    solved as one batch: every iteration against the oracle."""
    probs = [S.config_table1(t) for t in range(1, 6)]
    jobs = gpu_trajectory(ctx, probs, 30, tmp_path, "t1")
    st = ctx.status(len(probs))
    for t, m, s_ in zip(range(1, 6), pool.map(oracle_runs.compare_trajectory, jobs), st):
        assert_trajectory(f"table1_test{t}", m, s_)


@pytest.fixture(scope="module")
def c4_trajectory(ctx, pool, tmp_path_factory):
    """Five free iterations of one 4096 x 4096 image of the bandwidth-stress
    workload (31 x 31 motion blur, BSNR 35, w = 9, eps = 1e-4)."""
    p = S.config_c4_image(0, iters=5)
    jobs = gpu_trajectory(ctx, [p], 5, tmp_path_factory.mktemp("c4"), "c4")
    st = ctx.status(1)[0]
    return pool.map(oracle_runs.compare_trajectory, jobs)[0], st


def test_trajectory_4096(c4_trajectory):
    m, st = c4_trajectory
    assert_trajectory("trajectory_c4_4096", m, st)


def c2_subset():
    # images of every canvas / PSF / window class, in index order
    return [S.config_c2_image(i, iters=15) for i in (0, 1, 2, 3, 4, 5, 6, 7)]


def test_batched_equals_plain(ctx):
    """A batched image runs the same arithmetic as the plain solve except for
    the order of the partial sums of Eq. 11 (which depends on how the image's
    tiles are split across blocks), so lambda agrees to ~1e-7 relative and u
    to a few 1e-6 (both are held to the oracle by the trajectory tests)."""
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
        np.testing.assert_allclose(host(it["isnr"]), host(isnr1), atol=1e-4)


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
def test_small_and_nonsquare(ctx, tmp_path, M, N, w, k):
    """Three free iterations on tiny, window-wider-than-canvas and very
    elongated canvases, every iteration against the oracle."""
    rng = np.random.default_rng(M * N + w)
    u0 = S.image_polygons(11, M, N, n_poly=3, texture_std=0.02, rng=rng)
    h = S.psf_gaussian(k, 1.2)
    yb = S.blur_circular(u0, h)
    sigma = 0.01
    y = (yb + sigma * rng.standard_normal((M, N))).astype(np.float32)
    p = S.Problem(y, h.astype(np.float32), sigma, w, 1e-3, 3, u0.astype(np.float32), (M, N),
                  {"name": f"small_{M}x{N}"})
    jobs = gpu_trajectory(ctx, [p], 3, tmp_path, "small")
    st = ctx.status(1)[0]
    assert_trajectory(f"small_{M}x{N}_w{w}_k{k}", oracle_runs.compare_trajectory(jobs[0]), st)


@pytest.mark.parametrize("M,N", [(8, 8), (16, 8), (8, 32)])
def test_tiny_canvases_many_iterations(ctx, tmp_path, M, N):
    """Twelve free iterations on canvases whose column passes run blocks of
    fewer than 32 threads, so that the per-image lambda update (interpolated
    roots of the first passes from iteration 2 on, narrow 8-node brackets from
    iteration 5 on) runs on a partial warp; every iteration against the
    oracle.  Lambda is held to max(the kappa-derived bound, 1e-5): with 32 to
    128 bins nothing averages the FP32 rounding of the spectra of u_E, which
    errs by up to ~1e-6 relative per bin and moves the root by a few 1e-6
    (measured 1.6e-6 on 8 x 8); a wrong bracket or root logic errs by percents."""
    rng = np.random.default_rng(7 * M + N)
    u0 = S.image_polygons(13, M, N, n_poly=3, texture_std=0.02, rng=rng)
    h = S.psf_gaussian(3, 1.0)
    y = (S.blur_circular(u0, h) + 0.01 * rng.standard_normal((M, N))).astype(np.float32)
    p = S.Problem(y, h.astype(np.float32), 0.01, 3, 1e-3, 12, u0.astype(np.float32), (M, N),
                  {"name": f"tiny_{M}x{N}"})
    jobs = gpu_trajectory(ctx, [p], 12, tmp_path, "tiny")
    st = ctx.status(1)[0]
    m = oracle_runs.compare_trajectory(jobs[0])
    m["tol_tf"] = [max(t, 1e-5) for t in m["tol_tf"]]
    m["tol_free"] = [max(t, 1e-5) for t in m["tol_free"]]
    assert_trajectory(f"tiny_{M}x{N}_12it", m, st)


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


# ---------------------------------------------------------------------------
# Options: window-statistics arithmetic, truncated windows, fixed rho, the
# lambda pass schedule and tolerance; the build's target architecture
# ---------------------------------------------------------------------------

VAR_MODES = (gfd.VAR_COMPENSATED, gfd.VAR_DOUBLE_FLOAT, gfd.VAR_FP64, gfd.VAR_FP32,
             gfd.VAR_FP32_RAW)


@pytest.fixture(scope="module")
def var_ctx():
    cs = {m: gfd.Context(0, var_precision=m) for m in VAR_MODES}
    yield cs
    for c in cs.values():
        c.close()


@pytest.fixture(scope="module")
def trunc_ctx():
    c = gfd.Context(0, boundary=gfd.BOUNDARY_TRUNCATED)
    yield c
    c.close()


def gf_inputs(M, N, seed, offset=0.0, step=0.0, tex=0.02):
    rng = np.random.default_rng(seed)
    u0 = S.image_polygons(3, M, N, n_poly=8, texture_std=tex, rng=rng) + offset
    if step:
        yy, xx = np.mgrid[0:M, 0:N]
        u0 = u0 + step * (((yy // 24) + (xx // 40)) % 2)
    I = (u0 + 0.01 * rng.standard_normal((M, N))).astype(np.float32)
    p = (u0 + 0.03 * rng.standard_normal((M, N))).astype(np.float32)
    return I, p


@pytest.mark.parametrize("mode", VAR_MODES)
@pytest.mark.parametrize("M,N,w,eps", [(8, 8, 9, 1e-3), (64, 128, 5, 1e-3), (256, 512, 9, 1e-4),
                                       (128, 128, 17, 1e-2), (32, 2048, 11, 1e-3)])
def test_guided_filter_every_arithmetic(var_ctx, mode, M, N, w, eps):
    I, p = gf_inputs(M, N, M + N + w)
    got = host(var_ctx[mode].guidfilter(cuda(I), cuda(p), w, eps))
    err = np.abs(got - O.guided_filter(I, p, w, eps)).max()
    record(f"gf_{gfd.VAR_NAMES[mode]}_{M}x{N}_w{w}_eps{eps}", max_abs=err)
    assert err < U_TOL


def test_guided_filter_precision_study(var_ctx):
    """Window statistics of a guidance image with a large offset and steps of
    height 3 inside every strip (eps = 1e-4, w = 9), where E[I^2] - mu^2
    cancels heavily: the compensated and FP64 sums hold 2e-5; the FP32
    variants' errors are recorded (the plain sums of the raw values lose it)."""
    M, N, w, eps = 512, 512, 9, 1e-4
    I, p = gf_inputs(M, N, 77, offset=4.0, step=3.0, tex=0.003)
    ref = O.guided_filter(I, p, w, eps)
    errs = {}
    for mode in VAR_MODES:
        got = host(var_ctx[mode].guidfilter(cuda(I), cuda(p), w, eps))
        errs[mode] = float(np.abs(got - ref).max())
    record("gf_precision_study_offset4_step3_eps1e-4",
           **{gfd.VAR_NAMES[m]: e for m, e in errs.items()})
    assert errs[gfd.VAR_COMPENSATED] < U_TOL
    assert errs[gfd.VAR_DOUBLE_FLOAT] < U_TOL
    assert errs[gfd.VAR_FP64] < U_TOL
    assert errs[gfd.VAR_FP32_RAW] > errs[gfd.VAR_COMPENSATED]


@pytest.mark.parametrize("mode", (gfd.VAR_DOUBLE_FLOAT, gfd.VAR_FP64, gfd.VAR_FP32,
                                  gfd.VAR_FP32_RAW))
def test_trajectory_every_arithmetic(var_ctx, tmp_path, mode):
    """The whole method on the 256^2 workload with each window-statistics
    arithmetic (the default, compensated, is covered above).  The plain FP32
    sums of raw values are a precision-study variant: their errors are
    recorded, not held to the tolerances."""
    p = S.config_c0()
    jobs = gpu_trajectory(var_ctx[mode], [p], p.iters, tmp_path, "var")
    st = var_ctx[mode].status(1)[0]
    m = oracle_runs.compare_trajectory(jobs[0])
    name = f"trajectory_c0_{gfd.VAR_NAMES[mode]}"
    if mode == gfd.VAR_FP32_RAW:
        record(name, u_max_abs=max(m["u_err"]), u_max_abs_lambda_forced=max(m["u_err_forced"]),
               isnr_abs_max=max(m["isnr_err"]))
    else:
        assert_trajectory(name, m, st)


@pytest.mark.parametrize("M,N,w,eps", [(8, 8, 9, 1e-3), (16, 32, 3, 1e-3), (64, 128, 5, 1e-3),
                                       (256, 256, 7, 1e-4), (128, 128, 17, 1e-2),
                                       (32, 2048, 11, 1e-3), (1024, 64, 1, 1e-3)])
def test_guided_filter_truncated_windows(trunc_ctx, M, N, w, eps):
    I, p = gf_inputs(M, N, 3 * M + N + w)
    got = host(trunc_ctx.guidfilter(cuda(I), cuda(p), w, eps))
    err = np.abs(got - O.guided_filter(I, p, w, eps, boundary="truncated")).max()
    record(f"gf_truncated_{M}x{N}_w{w}_eps{eps}", max_abs=err)
    assert err < U_TOL


def test_trajectory_truncated_windows(trunc_ctx, tmp_path):
    p = S.config_c0()
    jobs = gpu_trajectory(trunc_ctx, [p], p.iters, tmp_path, "trunc")
    jobs[0]["boundary"] = "truncated"
    st = trunc_ctx.status(1)[0]
    assert_trajectory("trajectory_c0_truncated", oracle_runs.compare_trajectory(jobs[0]), st)


def test_fixed_rho(tmp_path):
    """rho given instead of Eq. 12 (Sec. 3.2): T = rho P sigma^2."""
    p = S.config_c0()
    with gfd.Context(0, rho=0.8) as c:
        jobs = gpu_trajectory(c, [p], 5, tmp_path, "rho")
        st = c.status(1)[0]
    jobs[0]["rho"] = 0.8
    m = oracle_runs.compare_trajectory(jobs[0])
    assert_trajectory("trajectory_c0_rho0.8", m, st)
    ref = O.solve(p.y, p.h, p.sigma, p.w, p.eps, 1, rho=0.8)
    assert m["lam_ref"][0] == pytest.approx(ref["lam"][0], rel=1e-12)


def test_pass_schedule_exhausted_is_reported():
    """With one pass after the fused one, iteration 0's root (bracket
    [1e-8, 1e4], geometric nodes) is still open when the schedule ends: the
    status says so, and lambda is the bracket's midpoint.  With the default
    schedule it resolves and the bit stays clear."""
    p = S.config_c0(M=64, N=64)
    with gfd.Context(0, lambda_max_passes=1) as c:
        c.solve(cuda(p.y), cuda(p.h), p.sigma, p.w, p.eps, 1)
        torch.cuda.synchronize()
        assert c.status(1)[0] & gfd.STATUS_PASSES_EXHAUSTED
    with gfd.Context(0) as c:
        _, lam, _ = c.solve(cuda(p.y), cuda(p.h), p.sigma, p.w, p.eps, 1)
        torch.cuda.synchronize()
        assert c.status(1)[0] & gfd.STATUS_PASSES_EXHAUSTED == 0
    ref = O.solve(p.y, p.h, p.sigma, p.w, p.eps, 1)
    assert abs(float(host(lam)[0]) / ref["lam"][0] - 1) < LAM_TOL_TF


def test_lambda_rtol_option():
    """A coarse lambda_rtol stops the root search early: lambda stays within
    that tolerance of the oracle's root (and is not the fine answer)."""
    p = S.config_c0()
    ref = O.solve(p.y, p.h, p.sigma, p.w, p.eps, 1)
    with gfd.Context(0, lambda_rtol=1e-3) as c:
        _, lam, _ = c.solve(cuda(p.y), cuda(p.h), p.sigma, p.w, p.eps, 1)
        torch.cuda.synchronize()
        assert c.status(1)[0] == 0
    err = abs(float(host(lam)[0]) / ref["lam"][0] - 1)
    record("lambda_rtol_1e-3", lam_rel=err)
    assert err < 1e-3


def test_invalid_options_rejected():
    for kw in ({"var_precision": 5}, {"boundary": 2}, {"lambda_max_passes": 17},
               {"lambda_rtol": 1e-16}, {"lambda_rtol": 0.5}, {"rho": 1.5}):
        with pytest.raises(gfd.GfdError) as e:
            gfd.Context(0, **kw)
        assert e.value.code == -1, kw


def test_library_kernels_built_for_sm_103a():
    built, dev = gfd.device_arch(0)
    assert built == 103, built
    assert dev == 103, dev


# ---------------------------------------------------------------------------
# Autotuner: tile shapes chosen by measurement, stored, read back, and every
# shape it can choose computing the same method
# ---------------------------------------------------------------------------

def test_autotune_writes_reads_and_solves(ctx, pool, tmp_path):
    probs = [S.config_c2_image(i, iters=4) for i in (13, 3, 1)]  # 256^2, 512^2, 1024^2
    items = [{"y": cuda(p.y), "h": cuda(p.h), "sigma": p.sigma, "w": p.w, "eps": p.eps}
             for p in probs]
    path = str(tmp_path / "tune.txt")
    with gfd.Context(0) as c:
        arr = c.make_images(items, 4)
        c.autotune(arr, 4, path)
        chains, table = gfd.tune_read(path)
        assert set(table) == {p.shape for p in probs}
        for (M, N), shp in table.items():
            assert c.tune_get(M, N) == (*shp, chains)
    with gfd.Context(0, tune_cache=path) as c:
        for (M, N), shp in table.items():
            assert c.tune_get(M, N) == (*shp, chains)
        jobs = gpu_trajectory(c, probs, 4, tmp_path, "tuned")
        st = c.status(len(probs))
    for i, m, s_ in zip((13, 3, 1), pool.map(oracle_runs.compare_trajectory, jobs), st):
        assert_trajectory(f"autotuned_c2_{i}", m, s_)


@pytest.mark.parametrize("shape", [(64, 64, 16, 1), (128, 256, 32, 2), (64, 128, 64, 4)])
def test_every_searched_shape_matches_the_oracle(pool, tmp_path, shape):
    """Column-pass threads (tile width), row-pass threads, guided-filter rows
    and chain count from the autotuner's search space, on a batch of every
    canvas size of the uneven workload."""
    col, row, gfr, chains = shape
    probs = [S.config_c2_image(i, iters=3) for i in (13, 3, 1, 64)]
    path = tmp_path / "shapes.txt"
    path.write_text(f"chains {chains}\n" + "".join(
        f"class {M} {N} col_threads {col} row_threads {row} gf_rows {gfr}\n"
        for (M, N) in {p.shape for p in probs}))
    with gfd.Context(0, tune_cache=str(path)) as c:
        jobs = gpu_trajectory(c, probs, 3, tmp_path, f"shape{col}_{row}_{gfr}")
        st = c.status(len(probs))
    for i, m, s_ in zip((13, 3, 1, 64), pool.map(oracle_runs.compare_trajectory, jobs), st):
        assert_trajectory(f"shape_{col}_{row}_{gfr}_{chains}_c2_{i}", m, s_)


# ---------------------------------------------------------------------------
# Colour guidance (3 x 3 window covariance solve)
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("M,N,w,eps", [(8, 8, 9, 1e-3), (16, 64, 3, 1e-3), (64, 128, 5, 1e-4),
                                       (256, 256, 7, 1e-3), (128, 32, 17, 1e-2)])
@pytest.mark.parametrize("boundary", ("periodic", "truncated"))
def test_guided_filter_color(ctx, trunc_ctx, M, N, w, eps, boundary):
    rng = np.random.default_rng(M * 5 + N + w)
    base = S.image_polygons(5, M, N, n_poly=6, texture_std=0.02, rng=rng)
    I = np.stack([base + 0.05 * rng.standard_normal((M, N)),
                  0.7 * base + 0.2 + 0.05 * rng.standard_normal((M, N)),
                  S.image_polygons(6, M, N, n_poly=6, texture_std=0.02, rng=rng)]).astype(np.float32)
    p = (base + 0.03 * rng.standard_normal((M, N))).astype(np.float32)
    c = trunc_ctx if boundary == "truncated" else ctx
    got = host(c.guidfilter_color(cuda(I), cuda(p), w, eps))
    ref = O.guided_filter_color(np.moveaxis(I, 0, -1), p, w, eps, boundary)
    err = np.abs(got - ref).max()
    record(f"gf_color_{boundary}_{M}x{N}_w{w}_eps{eps}", max_abs=err)
    assert err < U_TOL


def test_guided_filter_color_equal_channels_is_grey(ctx):
    """Three equal guidance channels: the grey-scale filter with eps / 3."""
    rng = np.random.default_rng(9)
    G = rng.random((64, 64)).astype(np.float32)
    p = rng.random((64, 64)).astype(np.float32)
    col = host(ctx.guidfilter_color(cuda(np.stack([G, G, G])), cuda(p), 5, 3e-3))
    grey = host(ctx.guidfilter(cuda(G), cuda(p), 5, 1e-3))
    assert np.abs(col - grey).max() < U_TOL


# ---------------------------------------------------------------------------
# Padding only the observation: pad, solve on the canvas, crop
# ---------------------------------------------------------------------------

def test_pad_and_crop_kernels(ctx):
    rng = np.random.default_rng(3)
    for (m, n), (M, N) in (((384, 384), (512, 512)), ((768, 1024), (1024, 1024)),
                           ((5, 7), (16, 8)), ((8, 8), (32, 64))):
        y = rng.random((m, n)).astype(np.float32)
        yc = host(ctx.pad_symmetric(cuda(y), M, N))
        assert np.array_equal(yc, O.pad_symmetric(y, M, N).astype(np.float32))
        assert np.array_equal(host(ctx.crop(cuda(yc), m, n)), y)
    with pytest.raises(gfd.GfdError):
        ctx.pad_symmetric(cuda(np.zeros((9, 8), np.float32)), 8, 8)


def test_solve_padded_matches_oracle(ctx):
    """A 384 x 384 observation (blurred scene cropped from a larger one)
    padded to 512^2, solved, cropped: against the oracle's pad -> solve ->
    crop at every iteration count."""
    p = S.config_c2_image(5, iters=4)  # true size 384^2 on a 512^2 canvas
    m, n = p.true_shape
    y_true = np.ascontiguousarray(p.y[:m, :n])
    yc = O.pad_symmetric(y_true, *p.shape).astype(np.float32)
    ref = O.solve(yc, p.h, p.sigma, p.w, p.eps, 4, trace=True)
    for k in (1, 4):
        u, lam = ctx.solve_padded(cuda(y_true), cuda(p.h), p.sigma, p.w, p.eps, k)
        torch.cuda.synchronize()
        assert np.abs(host(u) - O.crop(ref["u_k"][k - 1], m, n)).max() < U_TOL
        assert abs(float(host(lam)[0]) / ref["lam"][0] - 1) < LAM_TOL_TF
