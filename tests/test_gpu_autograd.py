"""Differentiable prediction on the GPU (needs a GB300).

The loss is L(I) = ||P I - V||^2 with P the prediction operator (pad + correct, FFT,
degrid; Section 2.1 read as a linear map from image to visibilities) and I a real float32
image. `lmg.predict` is a torch.autograd.Function whose backward is the gridding path
(dirty image of the residuals, the adjoint of P). L is quadratic in I, so a central
difference (L(I + e d) - L(I - e d)) / 2e equals the directional derivative exactly up to
rounding, for any step e.

* Multi-channel tracks on a 1024^2 grid, W = 8: the gradient against the FP64 oracle's
  gradient 2 Re P^H (P I - V) element by element, and against central differences.
* The differentiable-imaging workload at full size (64 antennas, 384 time samples x 64
  channels over 0.95-1.05 GHz = 49.5e6 visibilities, 4096^2 grid, x0 = 0.5, W = 8):
  central differences at 32 random pixels, the adjoint identity <P I, r> = <I, P^H r>
  summed over every visibility, and the forward pass against the oracle on 2000
  sampled visibilities.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import imaging as I  # noqa: E402
from paper_1906_07102_gb300 import lmg  # noqa: E402
from paper_1906_07102_gb300 import synthetic as S  # noqa: E402
from tests.cases import oracle_hvec, oracle_table, rel_rms, track_case  # noqa: E402

pytestmark = pytest.mark.gpu

W, MS = 8, 1000


def loss_and_grad(plan, image, V):
    """L = sum |P I - V|^2 accumulated in float64, and dL/dI by autograd."""
    img = image.clone().requires_grad_(True)
    r = lmg.predict(img, plan) - V
    L = (r.real.double() ** 2 + r.imag.double() ** 2).sum()
    L.backward()
    return float(L.detach()), img.grad.detach(), r.detach()


def loss(plan, image, V):
    with torch.no_grad():
        r = lmg.predict(image, plan) - V
        return float((r.real.double() ** 2 + r.imag.double() ** 2).sum())


def central_differences(plan, image, V, pixels, step):
    """(L(I + step e_p) - L(I - step e_p)) / (2 step) for each pixel p = (row, col)."""
    out = []
    for (py, px) in pixels:
        Ip = image.clone()
        Ip[py, px] += step
        Im = image.clone()
        Im[py, px] -= step
        out.append((loss(plan, Ip, V) - loss(plan, Im, V)) / (2 * step))
    return np.array(out)


def fd_step(image):
    """Step of the size of the image's 2-norm: the float32 rounding of P(I +- e d) then
    weighs about equally on the image and on the step, which keeps the difference
    quotient within ~1e-4 of the gradient."""
    return float(torch.linalg.vector_norm(image.double()))


def random_pixels(n, count, seed):
    g = np.random.default_rng(seed)
    return list(zip(g.integers(0, n, count), g.integers(0, n, count)))


def check_fd(fd, g, tol):
    """Per-pixel agreement relative to the RMS gradient over the sampled pixels."""
    scale = np.sqrt(np.mean(g ** 2))
    assert scale > 0
    err = np.abs(fd - g)
    assert err.max() <= tol * scale, (err.max() / scale, fd[:4], g[:4])


# ----------------------------------------------------------------------------------------
# 1024^2 grid: 16 antennas, 64 time samples x 16 channels (122,880 visibilities)
# ----------------------------------------------------------------------------------------
N_S, n_S = 1024, 512


@pytest.fixture(scope="module")
def small():
    freqs = np.linspace(0.95e9, 1.05e9, 16)
    uv, dl, vis = track_case(n_ant=16, n_times=64, N=N_S, n_src=50, seed=11, freqs=freqs)
    image = S.gaussian_blob_image(n_S, 64, seed=11).astype(np.float32)
    tab = lmg.Table(W, 0.5, MS, "linear")
    plan = lmg.Plan(tab, n_S, dl, uv.shape[0], "c64")
    plan.bin(torch.from_numpy(uv).cuda())
    return uv, dl, vis, image, plan


def test_gradient_matches_fp64_oracle(small):
    uv, dl, vis, image, plan = small
    V = torch.from_numpy(vis.astype(np.complex64)).cuda()
    L, g, _ = loss_and_grad(plan, torch.from_numpy(image).cuda(), V)
    T = oracle_table(W, 0.5, MS)
    hv = oracle_hvec(T, MS, "linear", W, n_S, N_S)
    uc = I.cells_from_wavelengths(uv, N_S, dl)
    op = I.Plan(uc[:, 0], uc[:, 1], W, N_S, single_precision_s=False)
    r = I.predict_vis(op, T, MS, 1, hv, image.astype(np.complex128)) - vis.astype(np.complex64)
    g_ref = 2.0 * I.dirty_image(op, T, MS, 1, hv, n_S, r).real
    L_ref = float(np.sum(np.abs(r) ** 2))
    assert abs(L - L_ref) <= 1e-5 * L_ref
    assert rel_rms(g.cpu().numpy(), g_ref) < 1e-5


def test_gradient_matches_central_differences_small(small):
    uv, dl, vis, image, plan = small
    V = torch.from_numpy(vis.astype(np.complex64)).cuda()
    img = torch.from_numpy(image).cuda()
    _, g, _ = loss_and_grad(plan, img, V)
    pix = random_pixels(n_S, 32, 5)
    fd = central_differences(plan, img, V, pix, fd_step(img))
    gp = g.cpu().numpy()[tuple(np.array(pix).T)]
    check_fd(fd, gp, 1e-3)


def test_complex_image_gradient_is_adjoint(small):
    """For a complex image the gradient is 2 P^H (P I - V) (PyTorch's convention)."""
    uv, dl, vis, image, plan = small
    V = torch.from_numpy(vis.astype(np.complex64)).cuda()
    img = torch.from_numpy((image + 0.5j * image[::-1]).astype(np.complex64)).cuda()
    _, g, r = loss_and_grad(plan, img, V)
    ref = 2.0 * plan.dirty_image(r)
    assert g.dtype == torch.complex64
    assert rel_rms(g.cpu().numpy(), ref.cpu().numpy()) < 1e-6


# ----------------------------------------------------------------------------------------
# full size: 49.5e6 visibilities, 4096^2 grid, W = 8
# ----------------------------------------------------------------------------------------
N_F, n_F = 4096, 2048


@pytest.fixture(scope="module")
def full():
    freqs = np.linspace(0.95e9, 1.05e9, 64)
    uv = S.array_tracks(n_ant=64, n_times=384, freqs_hz=freqs, seed=12)
    dl = S.pixel_scale_for(uv)
    l, m, f = S.point_source_sky(4, 0.45 * n_F * dl, seed=12)
    vis = S.visibilities(uv, l, m, f, noise_sigma=0.1, seed=12).astype(np.complex64)
    image = S.gaussian_blob_image(n_F, 64, seed=12).astype(np.float32)
    tab = lmg.Table(W, 0.5, MS, "linear")
    plan = lmg.Plan(tab, n_F, dl, uv.shape[0], "c64")
    uv_d = torch.from_numpy(uv).cuda()
    plan.bin(uv_d)
    V = torch.from_numpy(vis).cuda()
    img = torch.from_numpy(image).cuda()
    return uv, dl, V, img, plan


def test_full_size_central_differences(full):
    uv, dl, V, img, plan = full
    assert uv.shape[0] == 64 * 384 * 2016
    _, g, _ = loss_and_grad(plan, img, V)
    pix = random_pixels(n_F, 32, 6)
    fd = central_differences(plan, img, V, pix, fd_step(img))
    gp = g.cpu().numpy()[tuple(np.array(pix).T)]
    check_fd(fd, gp, 1e-3)


def test_full_size_adjoint_identity(full):
    """<P I, r> = <I, P^H r> over all 49.5e6 visibilities, summed in float64."""
    uv, dl, V, img, plan = full
    _, g, r = loss_and_grad(plan, img, V)
    with torch.no_grad():
        PI = lmg.predict(img, plan)
    lhs = torch.sum(PI.real.double() * r.real.double() + PI.imag.double() * r.imag.double()).item()
    rhs = 0.5 * torch.sum(img.double() * g.double()).item()
    scale = (torch.linalg.vector_norm(PI.to(torch.complex128)).item()
             * torch.linalg.vector_norm(r.to(torch.complex128)).item())
    assert abs(lhs - rhs) <= 1e-6 * scale


def test_full_size_forward_on_sampled_visibilities(full):
    uv, dl, V, img, plan = full
    with torch.no_grad():
        PI = lmg.predict(img, plan).cpu().numpy()
    k = np.sort(np.random.default_rng(7).choice(uv.shape[0], 2000, replace=False))
    T = oracle_table(W, 0.5, MS)
    hv = oracle_hvec(T, MS, "linear", W, n_F, N_F)
    uc = I.cells_from_wavelengths(uv[k], N_F, dl)
    op = I.Plan(uc[:, 0], uc[:, 1], W, N_F, single_precision_s=False)
    ref = I.predict_vis(op, T, MS, 1, hv, img.cpu().numpy().astype(np.complex128))
    assert rel_rms(PI[k], ref) < 1e-5
