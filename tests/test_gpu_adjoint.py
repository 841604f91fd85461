"""GPU gradients of the unrolled method (gfdeconv_backward_batched, the
hand-written adjoint) against the oracle's FP64 gradient (oracle/adjoint.py,
itself pinned by central finite differences) on the same FP32 inputs.

Tolerance: the GPU's forward and backward run in FP32 spectra and planes
with compensated window sums and FP64 reductions; its gradients are held to
1e-4 relative in norm (g_y, g_h) and in value (g_eps) against the FP64 oracle
(the bar the differentiation workload states for its finite-difference
check; the measured errors are recorded with each run)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import oracle as O  # noqa: E402
import synthetic as S  # noqa: E402
import paper_1609_01839_gb300 as gfd  # noqa: E402
from oracle import adjoint as A  # noqa: E402
from test_gpu_parity import record  # noqa: E402

DEV = torch.device("cuda:0")
GRAD_RTOL = 1e-4


def cuda(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(DEV)


def diff_problem(M=64, k=25, psf_sigma=1.6, noise=1.0 / 255.0, w=7, eps=1e-3, seed=11):
    """The differentiation workload's settings (25 x 25 Gaussian PSF, sigma 1.6,
    noise 1/255, w = 7, eps = 1e-3) on an M x M canvas; FP32 inputs."""
    rng = np.random.default_rng(seed)
    u0 = S.image_polygons(seed, M, M, n_poly=8, texture_std=0.02, rng=rng)
    h = S.psf_gaussian(k, psf_sigma)
    y = S.blur_circular(u0, h) + noise * rng.standard_normal((M, M))
    return (y.astype(np.float32), h.astype(np.float32), noise, w, eps, u0.astype(np.float32))


@pytest.fixture(scope="module")
def ctx():
    c = gfd.Context(0)
    yield c
    c.close()


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a, np.float64) - b) / np.linalg.norm(b))


def gpu_grads(ctx, probs, iters):
    items = [{"y": cuda(y), "h": cuda(h), "sigma": s, "w": w, "eps": e}
             for (y, h, s, w, e, _) in probs]
    ctx.solve_batched(items, iters, want_checkpoints=True)
    g_us = [2.0 * (it["u"] - cuda(uc)) / uc.size for it, (*_, uc) in zip(items, probs)]
    res = ctx.backward_batched(items, iters, g_us)
    torch.cuda.synchronize()
    return items, [(r[0].cpu().numpy(), r[1].cpu().numpy(), float(r[2].cpu())) for r in res]


@pytest.mark.parametrize("iters", [1, 3, 10])
def test_gradients_match_oracle(ctx, iters):
    p = diff_problem()
    y, h, s, w, eps, uc = p
    ref = A.solve_with_grad(y, h, s, w, eps, iters, uc)
    assert all(np.isfinite(ref["lam"]))
    _, [(gy, gh, ge)] = gpu_grads(ctx, [p], iters)
    e_y, e_h, e_e = rel(gy, ref["g_y"]), rel(gh, ref["g_h"]), abs(ge / ref["g_eps"] - 1)
    record(f"adjoint_64_{iters}it", g_y_rel=e_y, g_h_rel=e_h, g_eps_rel=e_e)
    assert e_y < GRAD_RTOL and e_h < GRAD_RTOL and e_e < GRAD_RTOL, (e_y, e_h, e_e)


def test_gradients_512_image(ctx):
    """One 512 x 512 image of the differentiation workload, 10 iterations."""
    p = diff_problem(M=512, seed=3)
    y, h, s, w, eps, uc = p
    ref = A.solve_with_grad(y, h, s, w, eps, 10, uc)
    _, [(gy, gh, ge)] = gpu_grads(ctx, [p], 10)
    e_y, e_h, e_e = rel(gy, ref["g_y"]), rel(gh, ref["g_h"]), abs(ge / ref["g_eps"] - 1)
    record("adjoint_512_10it", g_y_rel=e_y, g_h_rel=e_h, g_eps_rel=e_e)
    assert e_y < GRAD_RTOL and e_h < GRAD_RTOL and e_e < GRAD_RTOL, (e_y, e_h, e_e)


def test_gradients_through_the_infinite_lambda_branch(ctx):
    """Start at the clean image with sigma twice the noise: the first two
    steps take the lambda = inf branch (u_E in the feasible set), the later
    ones solve Eq. 11; the gradient matches the oracle's through both."""
    y, h, s, w, eps, uc = diff_problem()
    s2 = 2.0 * s
    ref = A.solve_with_grad(y, h, s2, w, eps, 4, uc, u_init=uc)
    assert np.isinf(ref["lam"][0]) and np.isfinite(ref["lam"][3])
    items = [{"y": cuda(y), "h": cuda(h), "sigma": s2, "w": w, "eps": eps, "u_init": cuda(uc)}]
    ctx.solve_batched(items, 4, want_checkpoints=True)
    lam = items[0]["lam"].cpu().numpy()
    assert np.isinf(lam[0]) and np.isinf(lam[1]) and np.all(np.isfinite(lam[2:]))
    [(gy, gh, ge)] = ctx.backward_batched(items, 4, [2.0 * (items[0]["u"] - cuda(uc)) / uc.size])
    torch.cuda.synchronize()
    e_y, e_h = rel(gy.cpu().numpy(), ref["g_y"]), rel(gh.cpu().numpy(), ref["g_h"])
    e_e = abs(float(ge) / ref["g_eps"] - 1)
    record("adjoint_64_branch", g_y_rel=e_y, g_h_rel=e_h, g_eps_rel=e_e)
    assert e_y < GRAD_RTOL and e_h < GRAD_RTOL and e_e < GRAD_RTOL, (e_y, e_h, e_e)


def test_batch_equals_single_images(ctx):
    probs = [diff_problem(M=128, seed=s) for s in (21, 22, 23)]
    _, batch = gpu_grads(ctx, probs, 4)
    for p, (gy, gh, ge) in zip(probs, batch):
        _, [(sy, sh, se)] = gpu_grads(ctx, [p], 4)
        assert rel(gy, sy.astype(np.float64)) < 1e-5
        assert rel(gh, sh.astype(np.float64)) < 1e-5
        assert abs(ge / se - 1) < 1e-5


def test_autograd_function(ctx):
    """torch.autograd through Context.deconv: the same gradients as the
    library's backward entry point, for a batch with one shared PSF."""
    probs = [diff_problem(M=64, seed=s) for s in (31, 32)]
    Y = cuda(np.stack([p[0] for p in probs])).requires_grad_(True)
    Hh = cuda(probs[0][1]).requires_grad_(True)
    E = torch.tensor([1e-3, 2e-3], dtype=torch.float64, device=DEV, requires_grad=True)
    UC = cuda(np.stack([p[5] for p in probs]))
    u = ctx.deconv(Y, Hh, E, 1.0 / 255.0, 7, 3)
    loss = ((u - UC) ** 2).mean(dim=(1, 2)).sum()
    loss.backward()
    for b, p in enumerate(probs):
        y, h, s, w, _, uc = p
        ref = A.solve_with_grad(y, h, s, w, float(E[b].detach()), 3, uc)
        assert rel(Y.grad[b].cpu().numpy(), ref["g_y"]) < GRAD_RTOL
        assert abs(float(E.grad[b]) / ref["g_eps"] - 1) < GRAD_RTOL
    ref_h = sum(A.solve_with_grad(p[0], p[1], p[2], p[3], float(E[b].detach()), 3, p[5])["g_h"]
                for b, p in enumerate(probs))
    assert rel(Hh.grad.cpu().numpy(), ref_h) < GRAD_RTOL


def test_backward_needs_the_forward_lambdas(ctx):
    """The backward step recomputes each iteration with the forward solve's
    lambda_k: descriptors without lambda_out are refused before any launch."""
    y, h, s_, w, e, uc = diff_problem(M=64, seed=41)
    items = [{"y": cuda(y), "h": cuda(h), "sigma": s_, "w": w, "eps": e}]
    ctx.solve_batched(items, 2, want_checkpoints=True)
    arr = ctx.make_images(items, 2, want_checkpoints=True)
    arr[0].lambda_out = None
    grads = (gfd.Grad * 1)()
    gy, gh = torch.empty_like(items[0]["y"]), torch.empty_like(items[0]["h"])
    ge = torch.empty((), dtype=torch.float64, device=DEV)
    gu = torch.zeros_like(items[0]["y"])
    grads[0].g_u, grads[0].g_y, grads[0].g_h, grads[0].g_eps = (
        gu.data_ptr(), gy.data_ptr(), gh.data_ptr(), ge.data_ptr())
    rc = gfd._lib.gfdeconv_backward_batched(ctx._h, 1, arr, grads, 2, gfd._stream(None))
    assert rc == gfd.ERR_INVALID_ARG
