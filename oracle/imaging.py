"""Gridding, FFT imaging, correction, degridding and their DFT references in float64
(oracle; test infrastructure only).

Conventions (Section 2.1):

* grid index i = 0..N-1 holds G_n with n = i - N/2 (Eq. 4 sums n = -N/2 .. N/2-1);
* image pixel p = 0..n_img-1 sits at x_p = (p - n_img/2) / N, so the kept field is the
  central n_img of the N-pixel FFT image (|x| <= x0 with the paper's x0 = n_img / 2N);
* imaging uses exp(+i 2 pi n x) without normalisation (Eqs. 3-4), prediction uses
  exp(-i 2 pi (u l + v m)) (Eq. 2);
* u, v are in grid cells (the paper's u' = u L); the API's wavelengths are converted by
  the FP64 product u_cells = u_lambda * (N * pixel_scale);
* grid points outside [-N/2, N/2) wrap modulo N (exact at pixel centres).

Arrays are indexed [row, column] = [v, u].
"""
import numpy as np

from . import design as D

TWO_PI = 2.0 * np.pi

# Positions are quantised to FRAC_BITS fractional bits before the support rule is
# applied, so that the integer decision ceil(u - W/2) is exact and identical on every
# implementation; 2^-32 cell is far below the float32 offset precision.
FRAC_BITS = 32
MAX_ABS_CELLS = 2.0 ** 30


def cells_from_wavelengths(uv_lambda, N, pixel_scale):
    """u_cells = fl64(u_lambda * (N * pixel_scale)) (Section 2.1's u' = u L, L = N dl)."""
    scale = np.float64(N) * np.float64(pixel_scale)
    return np.asarray(uv_lambda, dtype=np.float64) * scale


def support_rule(u_cells, W):
    """Support start and table coordinate of each position (Eq. 6).

    Returns ``(n_start, S, valid)`` with n_start = ceil(u - W/2) (the lowest n with
    u - W/2 <= n) and S = (n_start - (u - W/2)) * 2^32 in [0, 2^32), computed exactly on
    u quantised to 2^-32 cell (round half to even). Positions that are not finite or
    whose magnitude reaches 2^30 cells are flagged invalid (they contribute nothing).
    """
    u = np.asarray(u_cells, dtype=np.float64)
    valid = np.isfinite(u) & (np.abs(u) < MAX_ABS_CELLS)
    uq = np.where(valid, u, 0.0)
    U = np.rint(np.ldexp(uq, FRAC_BITS)).astype(np.int64)
    Y = U - (W % 2) * (1 << (FRAC_BITS - 1))          # (u - W/2 + floor(W/2)) * 2^32
    c = -((-Y) >> FRAC_BITS)                           # ceil(Y / 2^32)
    n_start = c - W // 2
    S = (c << FRAC_BITS) - Y
    return n_start, S, valid


def s_float32(S):
    """Table coordinate rounded once to float32. Diagnostic only (``Plan(...,
    single_precision_s=True)``): it shows how much one float32 rounding of s moves a
    result; every parity reference uses the exact float64 coordinate."""
    return (np.asarray(S, dtype=np.float64) * 2.0 ** -FRAC_BITS).astype(np.float32)


def s_float64(S):
    """Table coordinate of the quantised position in float64 (exact: S < 2^32)."""
    return np.asarray(S, dtype=np.float64) * 2.0 ** -FRAC_BITS


def s_exact(u_cells, S):
    """Table coordinate of the unquantised position, s = n_start - (u - W/2), as
    fl(S 2^-32 + delta) with delta = u_q - u = (U - u 2^32) 2^-32 (exact: U is the
    integer nearest to u 2^32), so that the fraction keeps the full float64 precision of
    u while n_start comes from the exact integer rule. Invalid positions give 0."""
    u = np.asarray(u_cells, dtype=np.float64)
    valid = np.isfinite(u) & (np.abs(u) < MAX_ABS_CELLS)
    p = np.ldexp(np.where(valid, u, 0.0), FRAC_BITS)
    U = np.rint(p)
    delta = np.ldexp(U - p, -FRAC_BITS)
    return np.where(valid, s_float64(S) + delta, 0.0)


def table_lookup(T, Ms, S, s, interp):
    """Table weights (Section 5.1, Appendix F) with the row decision taken on the fixed-point
    coordinate S (exact integers: nearest row (S Ms + 2^31) >> 32, linear row (S Ms) >> 32,
    Lagrange first row ((S Ms) - (d - 1) 2^31) >> 32 clamped to [0, Ms - d]), identical on
    every implementation, and the interpolation fraction from the float64 coordinate s:
    t = s Ms, f = t - k."""
    P = np.asarray(S, dtype=np.int64) * np.int64(Ms)        # < 2^52
    t = np.asarray(s, dtype=np.float64) * Ms
    if interp == D.INTERP_NEAREST:
        return T[(P + (1 << (FRAC_BITS - 1))) >> FRAC_BITS]
    if interp == D.INTERP_LINEAR:
        k = P >> FRAC_BITS
        f = (t - k)[:, None]
        return (1.0 - f) * T[k] + f * T[k + 1]
    d = interp
    k0 = np.clip((P - (d - 1) * (1 << (FRAC_BITS - 1))) >> FRAC_BITS, 0, Ms - d)
    L = D.lagrange_basis(t - k0, d)
    return sum(L[:, m, None] * T[k0 + m] for m in range(d + 1))


class Plan:
    """Support starts and table coordinates for a set of (u, v) cell positions.

    The support starts and table rows come from the exact integer rule on the positions
    quantised to 2^-32 cell; the table coordinate s itself keeps the full float64 precision
    of the position (``s_exact``; the default, used by every parity reference). Two named
    diagnostics replace it: ``quantized_s=True`` uses the quantised coordinate S 2^-32 (its
    position error of up to 2^-33 cell bounds float64 results near 1e-10), and
    ``single_precision_s=True`` rounds that to float32 and takes the nearest-row decision in
    float32."""

    def __init__(self, u_cells, v_cells, W, N, single_precision_s=False, quantized_s=False):
        self.W, self.N = W, N
        self.n0, self.Su, vu = support_rule(u_cells, W)
        self.m0, self.Sv, vv = support_rule(v_cells, W)
        self.valid = vu & vv
        if single_precision_s:
            self.su, self.sv = s_float32(self.Su).astype(np.float64), s_float32(self.Sv).astype(np.float64)
        elif quantized_s:
            self.su, self.sv = s_float64(self.Su), s_float64(self.Sv)
        else:
            self.su, self.sv = s_exact(u_cells, self.Su), s_exact(v_cells, self.Sv)
        self.single = single_precision_s

    def weights(self, T, Ms, interp):
        """Per-axis weights Cu (K, W) and Cv (K, W) from the table (Section 5.1, App. F), or,
        when T is a function of s (direct calculation, Section 5.2), T(s) itself."""
        if callable(T):
            Cu, Cv = T(self.su), T(self.sv)
        elif self.single:
            Cu = D.table_weights(T, Ms, self.su, interp, np.float32)
            Cv = D.table_weights(T, Ms, self.sv, interp, np.float32)
        else:
            Cu = table_lookup(T, Ms, self.Su, self.su, interp)
            Cv = table_lookup(T, Ms, self.Sv, self.sv, interp)
        Cu[~self.valid] = 0.0
        Cv[~self.valid] = 0.0
        return Cu, Cv


def grid(plan, T, Ms, interp, vis, weights=None):
    """Gridding sum G_n = sum_k w_k V_k C(n - u_k) C(m - v_k) over the support (Eqs. 5-6),
    separable in u and v (Section 1, condition (i)); G[i_v, i_u] with i = n + N/2 mod N."""
    N, W = plan.N, plan.W
    Cu, Cv = plan.weights(T, Ms, interp)
    wv = np.asarray(vis, dtype=np.complex128)
    if weights is not None:
        wv = wv * np.asarray(weights, dtype=np.float64)
    G = np.zeros(N * N, dtype=np.complex128)
    chunk = max(1, (1 << 22) // (W * W))
    for k0 in range(0, wv.size, chunk):
        sl = slice(k0, k0 + chunk)
        flat, contrib = [], []
        for j in range(W):
            rows = (plan.m0[sl] + j + N // 2) % N
            for i in range(W):
                cols = (plan.n0[sl] + i + N // 2) % N
                flat.append(rows * N + cols)
                contrib.append(wv[sl] * Cv[sl, j] * Cu[sl, i])
        flat = np.concatenate(flat)
        contrib = np.concatenate(contrib)
        G += np.bincount(flat, weights=contrib.real, minlength=N * N)
        G += 1j * np.bincount(flat, weights=contrib.imag, minlength=N * N)
    return G.reshape(N, N)


def degrid(plan, T, Ms, interp, G):
    """Degridding, the transpose of gridding (Section 4):
    V_k = sum_{i,j} C(n_i - u_k) C(m_j - v_k) G[m_j, n_i]."""
    N, W = plan.N, plan.W
    Cu, Cv = plan.weights(T, Ms, interp)
    out = np.zeros(Cu.shape[0], dtype=np.complex128)
    for j in range(W):
        rows = (plan.m0 + j + N // 2) % N
        for i in range(W):
            cols = (plan.n0 + i + N // 2) % N
            out += Cv[:, j] * Cu[:, i] * G[rows, cols]
    return out


def pixel_coords(n_img, N):
    """x_p = (p - n_img/2) / N for p = 0..n_img-1."""
    return (np.arange(n_img, dtype=np.float64) - n_img // 2) / N


def fft_image(G):
    """F(x_q) = sum_{n=-N/2}^{N/2-1} G_n exp(i 2 pi n q / N) for q = 0..N-1 (Eq. 4 before
    correction), via numpy's unnormalised inverse FFT."""
    N = G.shape[0]
    return np.fft.ifft2(np.fft.ifftshift(G)) * (N * N)


def correct_crop(F, hvec, n_img):
    """Keep the central n_img pixels and multiply by h(x) h(y) (Eqs. 4, 15)."""
    N = F.shape[0]
    q = (np.arange(n_img) - n_img // 2) % N
    return F[np.ix_(q, q)] * hvec[:, None] * hvec[None, :]


def dirty_image(plan, T, Ms, interp, hvec, n_img, vis, weights=None):
    """FFT dirty image on the kept field: grid, FFT (+i), correct, crop."""
    return correct_crop(fft_image(grid(plan, T, Ms, interp, vis, weights)), hvec, n_img)


def pad_correct(image, hvec, N):
    """Adjoint of correct_crop: corrected image on the kept pixels of an N x N array
    indexed by q = p - n_img/2 mod N, zero elsewhere."""
    n_img = image.shape[0]
    P = np.zeros((N, N), dtype=np.complex128)
    q = (np.arange(n_img) - n_img // 2) % N
    P[np.ix_(q, q)] = image * hvec[:, None] * hvec[None, :]
    return P


def model_grid(P):
    """G_n = sum_q P_q exp(-i 2 pi n q / N) for n = -N/2..N/2-1 (forward FFT, adjoint of
    fft_image), returned in grid index order i = n + N/2."""
    return np.fft.fftshift(np.fft.fft2(P))


def predict_vis(plan, T, Ms, interp, hvec, image):
    """Predicted visibilities of a model image: pad and correct, FFT (-i), degrid."""
    return degrid(plan, T, Ms, interp, model_grid(pad_correct(image, hvec, plan.N)))


# ---------------------------------------------------------------------------------------
# Direct (DFT) references and the Cauchy-Schwarz bound
# ---------------------------------------------------------------------------------------
def dft_dirty_image(u, v, vis, weights, x, y):
    """I_D(x, y) = sum_k w_k V_k exp(i 2 pi (u_k x + v_k y)) (Eq. 3 in two dimensions)
    on the pixel grid x (columns) by y (rows)."""
    wv = np.asarray(vis, dtype=np.complex128) * (1.0 if weights is None else weights)
    out = np.zeros((y.size, x.size), dtype=np.complex128)
    for k0 in range(0, wv.size, 2048):
        sl = slice(k0, k0 + 2048)
        ex = np.exp(1j * TWO_PI * np.outer(u[sl], x))     # (K, X)
        ey = np.exp(1j * TWO_PI * np.outer(v[sl], y))     # (K, Y)
        out += (ey * wv[sl, None]).T @ ex
    return out


def dft_predict(u, v, image, x, y):
    """V_k = sum_p I_p exp(-i 2 pi (u_k x_p + v_k y_p)) (Eq. 2 on the pixel grid)."""
    out = np.empty(u.size, dtype=np.complex128)
    for k0 in range(0, u.size, 1024):
        sl = slice(k0, k0 + 1024)
        ex = np.exp(-1j * TWO_PI * np.outer(u[sl], x))    # (K, X)
        ey = np.exp(-1j * TWO_PI * np.outer(v[sl], y))    # (K, Y)
        out[sl] = np.einsum("ky,yx,kx->k", ey, image, ex)
    return out


def footprint_factor(plan, Cu, Cv, u, v, x, y, hx, hy):
    """h(x)h(y) a_k(x) a'_k(y) with a_k(x) = sum_i Cu_i exp(i 2 pi (n0 + i - u_k) x)
    (the factor multiplying V_k exp(i 2 pi (u x + v y)) in the FFT image, Eq. 7)."""
    W = plan.W
    du = (plan.n0[:, None] + np.arange(W)[None, :]) - u[:, None]
    dv = (plan.m0[:, None] + np.arange(W)[None, :]) - v[:, None]
    ax = np.einsum("ki,kix->kx", Cu, np.exp(1j * TWO_PI * du[:, :, None] * x[None, None, :]))
    ay = np.einsum("kj,kjy->ky", Cv, np.exp(1j * TWO_PI * dv[:, :, None] * y[None, None, :]))
    return ax * hx[None, :], ay * hy[None, :]


def image_bound(plan, T, Ms, interp, u, v, vis, weights, x, y, hx, hy=None):
    """Per-pixel Cauchy-Schwarz bound of Eq. 8 in two dimensions:
    |I_fft - I_D|^2 <= (sum_k w_k |V_k|^2) (sum_k w_k |1 - h h a_k a'_k|^2)
    on the pixel grid x (columns, factors hx) by y (rows, factors hy)."""
    Cu, Cv = plan.weights(T, Ms, interp)
    w = np.ones(u.size) if weights is None else np.asarray(weights, dtype=np.float64)
    ax, ay = footprint_factor(plan, Cu, Cv, u, v, x, y, hx, hx if hy is None else hy)
    ell = np.zeros((y.size, x.size))
    for k0 in range(0, u.size, 512):
        sl = slice(k0, k0 + 512)
        b = 1.0 - ay[sl, :, None] * ax[sl, None, :]
        ell += np.einsum("k,kyx->yx", w[sl], np.abs(b) ** 2)
    return float(np.sum(w * np.abs(vis) ** 2)) * ell


def predict_bound(plan, T, Ms, interp, u, v, image, x, y, hx, hy=None):
    """Per-visibility bound for prediction: |V_fft - V_D|^2 <= (sum_p |I_p|^2)
    (sum_p |1 - h h conj(a_k a'_k)|^2) -- the same Cauchy-Schwarz step as Eq. 8."""
    Cu, Cv = plan.weights(T, Ms, interp)
    ax, ay = footprint_factor(plan, Cu, Cv, u, v, x, y, hx, hx if hy is None else hy)
    b2 = np.abs(1.0 - ay[:, :, None] * ax[:, None, :]) ** 2
    return float(np.sum(np.abs(image) ** 2)) * b2.sum(axis=(1, 2))


def dirty_pixels_direct(plan, T, Ms, interp, hvec_x, hvec_y, vis, weights, x, y):
    """FFT dirty image at a few pixels without forming the grid: by linearity the image is
    sum_k w_k V_k h(x)h(y) sum_i Cu_i e^{i 2 pi (n0+i) x} sum_j Cv_j e^{i 2 pi (m0+j) y}
    (Eqs. 4-5); used to spot-check large grids. x, y are paired pixel coordinates."""
    Cu, Cv = plan.weights(T, Ms, interp)
    W = plan.W
    wv = np.asarray(vis, dtype=np.complex128)
    if weights is not None:
        wv = wv * weights
    out = np.empty(x.size, dtype=np.complex128)
    for p in range(x.size):
        ax = (Cu * np.exp(1j * TWO_PI * (plan.n0[:, None] + np.arange(W)) * x[p])).sum(1)
        ay = (Cv * np.exp(1j * TWO_PI * (plan.m0[:, None] + np.arange(W)) * y[p])).sum(1)
        out[p] = hvec_x[p] * hvec_y[p] * np.sum(wv * ax * ay)
    return out
