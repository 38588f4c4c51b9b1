"""Shared builders for the GPU parity tests: seeded inputs and oracle references.

The oracle and the CUDA path each build their own least-misfit table; `caller_table`
gives a closed-form table (Kaiser-Bessel-like window evaluated here, in the test) that is
handed to both sides when a test needs identical tables to isolate kernel arithmetic.
"""
import functools

import numpy as np

from oracle import design as D
from oracle import imaging as I
from paper_1906_07102_gb300 import synthetic as S

INTERP = {"nearest": 0, "linear": 1, "quadratic": 2, "cubic": 3}


@functools.lru_cache(maxsize=None)
def oracle_table(W, x0_api, Ms):
    h = D.least_misfit_h(W, x0_api / 2)
    return D.lm_table(h, W, x0_api / 2, Ms)


def caller_table(W, Ms, beta=None):
    """C(d) = I0(beta sqrt(1 - (2d/W)^2)) / I0(beta) on the table layout (row i at
    s = i/Ms, entry j at d = j - W/2 + s)."""
    beta = 2.3 * W if beta is None else beta
    s = np.arange(Ms + 1) / Ms
    d = np.arange(W)[None, :] - W / 2 + s[:, None]
    z = np.clip(1 - (2 * d / W) ** 2, 0, None)
    return np.i0(beta * np.sqrt(z)) / np.i0(beta)


def oracle_hvec(T, Ms, interp, W, n_img, N):
    return D.correction_factors(T, Ms, INTERP[interp], W, I.pixel_coords(n_img, N))


def rel_rms(a, b):
    a = np.asarray(a)
    b = np.asarray(b)
    return float(np.sqrt(np.mean(np.abs(a - b) ** 2)) / np.sqrt(np.mean(np.abs(b) ** 2)))


def disk_case(nvis, N, seed=0):
    """Config-1 style positions: uniform in the disk of radius 0.45 N cells; the pixel
    scale is 1/N so that wavelengths equal cells."""
    return S.disk_uniform(nvis, 0.45 * N, seed), 1.0 / N


def track_case(n_ant, n_times, N, n_src=200, noise=0.1, seed=0, freqs=(1.4e9,), n_img=None):
    """Earth-rotation tracks with a point-source sky: (uv_lambda, pixel_scale, vis c128)."""
    uv = S.array_tracks(n_ant=n_ant, n_times=n_times, freqs_hz=freqs, seed=seed)
    dl = S.pixel_scale_for(uv)
    n_img = n_img or N // 2
    l, m, f = S.point_source_sky(n_src, 0.45 * n_img * dl, seed=seed)
    vis = S.visibilities(uv, l, m, f, noise_sigma=noise, seed=seed)
    return uv, dl, vis
