"""Seeded synthetic inputs shared by the tests, the benchmark and the oracle checks.

This module holds none of the gridding method's arithmetic: it only draws positions,
values and images. Every generator is deterministic for a given seed (numpy PCG64 with
``SeedSequence`` substreams) and computes in float64 on the host.

Workloads (stand-ins for the paper's VLA simulations, whose antenna layout and imaging
parameters are not given):

* ``disk_uniform``        (u, v) uniform in a disk, in grid cells (small parity cases).
* ``array_tracks``        Earth-rotation (u, v) tracks of a random array: antenna east and
                          north offsets ~ N(0, sigma), all i<j baselines, hour angle
                          uniformly sampled over the track, time-major order
                          (all baselines of time 0, then time 1, ...), one block per channel.
* ``point_source_sky``    point sources uniform in the kept field with log-uniform flux.
* ``visibilities``        V = sum_s S_s exp(-i 2 pi (u l_s + v m_s)) + complex noise.
* ``gaussian_blob_image`` a sum of Gaussian blobs (differentiable-imaging model).
"""
import numpy as np

C_LIGHT = 299792458.0


def _rng(seed, *stream):
    return np.random.Generator(np.random.PCG64(np.random.SeedSequence([seed, *stream])))


def disk_uniform(nvis, radius, seed=0):
    """(u, v) uniform in the disk of the given radius; returns float64 [nvis, 2]."""
    g = _rng(seed, 1)
    r = radius * np.sqrt(g.random(nvis))
    th = 2.0 * np.pi * g.random(nvis)
    return np.stack([r * np.cos(th), r * np.sin(th)], axis=1)


def complex_normal(n, seed=0, stream=2, sigma=1.0):
    """iid N(0, sigma^2) + i N(0, sigma^2), complex128."""
    g = _rng(seed, stream)
    return sigma * g.standard_normal(n) + 1j * sigma * g.standard_normal(n)


def array_tracks(n_ant=64, sigma_m=1000.0, hours=6.0, n_times=2048, dec_deg=-30.0,
                 lat_deg=-30.0, freqs_hz=(1.4e9,), seed=0):
    """Earth-rotation (u, v) tracks in wavelengths, float64 [n_chan * n_times * n_bl, 2].

    ENU -> equatorial: X = -N sin(lat), Y = E, Z = N cos(lat) (antennas at zero height);
    (u, v) = (sinH X + cosH Y, -sin(dec) cosH X + sin(dec) sinH Y + cos(dec) Z) / lambda
    with hour angles H at the midpoints of n_times equal steps over the track.
    """
    g = _rng(seed, 3)
    east = g.normal(0.0, sigma_m, n_ant)
    north = g.normal(0.0, sigma_m, n_ant)
    i, j = np.triu_indices(n_ant, k=1)
    lat, dec = np.deg2rad(lat_deg), np.deg2rad(dec_deg)
    dE, dN = east[j] - east[i], north[j] - north[i]
    X, Y, Z = -dN * np.sin(lat), dE, dN * np.cos(lat)
    half = np.deg2rad(15.0 * hours) / 2.0
    H = -half + (np.arange(n_times) + 0.5) * (2.0 * half / n_times)
    sH, cH = np.sin(H)[:, None], np.cos(H)[:, None]
    u_m = sH * X[None, :] + cH * Y[None, :]
    v_m = -np.sin(dec) * cH * X[None, :] + np.sin(dec) * sH * Y[None, :] + np.cos(dec) * Z[None, :]
    out = []
    for f in freqs_hz:
        lam = C_LIGHT / f
        out.append(np.stack([(u_m / lam).ravel(), (v_m / lam).ravel()], axis=1))
    return np.concatenate(out, axis=0)


def pixel_scale_for(uv, fill=0.45):
    """Pixel scale (rad) that maps the largest |u|, |v| onto fill * N cells."""
    return fill / float(np.max(np.abs(uv)))


def point_source_sky(n_src, half_width_rad, flux_lo=1e-3, flux_hi=1.0, seed=0):
    """(l, m, flux): positions uniform in the square |l|, |m| < half_width_rad,
    fluxes log-uniform in [flux_lo, flux_hi]."""
    g = _rng(seed, 4)
    l = g.uniform(-half_width_rad, half_width_rad, n_src)
    m = g.uniform(-half_width_rad, half_width_rad, n_src)
    flux = np.exp(g.uniform(np.log(flux_lo), np.log(flux_hi), n_src))
    return l, m, flux


def visibilities(uv_lambda, l, m, flux, noise_sigma=0.0, seed=0, chunk=1 << 20):
    """V = sum_s S_s exp(-i 2 pi (u l_s + v m_s)) + (N(0, s^2) + i N(0, s^2)) noise, complex128.

    Computed in float64 with torch CPU threads (input synthesis only)."""
    import torch
    u = torch.from_numpy(np.ascontiguousarray(uv_lambda[:, 0]))
    v = torch.from_numpy(np.ascontiguousarray(uv_lambda[:, 1]))
    lt = torch.from_numpy(np.asarray(l, dtype=np.float64))
    mt = torch.from_numpy(np.asarray(m, dtype=np.float64))
    ft = torch.from_numpy(np.asarray(flux, dtype=np.float64))
    out = np.empty(u.numel(), dtype=np.complex128)
    for k0 in range(0, u.numel(), chunk):
        ph = -2.0 * np.pi * (u[k0:k0 + chunk, None] * lt[None, :] + v[k0:k0 + chunk, None] * mt[None, :])
        re = (torch.cos(ph) * ft).sum(1)
        im = (torch.sin(ph) * ft).sum(1)
        out[k0:k0 + chunk] = re.numpy() + 1j * im.numpy()
    if noise_sigma > 0:
        out += complex_normal(out.size, seed, stream=5, sigma=noise_sigma)
    return out


def gaussian_blob_image(n, n_blobs=64, seed=0, centre_frac=0.8, sigma_px=(1.0, 8.0),
                        amp=(1e-3, 1.0)):
    """Real image [n, n]: sum of Gaussian blobs with centres uniform in the central
    centre_frac of the field, widths and amplitudes log-uniform."""
    g = _rng(seed, 6)
    half = 0.5 * centre_frac * n
    cx = n / 2 + g.uniform(-half, half, n_blobs)
    cy = n / 2 + g.uniform(-half, half, n_blobs)
    sg = np.exp(g.uniform(np.log(sigma_px[0]), np.log(sigma_px[1]), n_blobs))
    a = np.exp(g.uniform(np.log(amp[0]), np.log(amp[1]), n_blobs))
    yy, xx = np.mgrid[0:n, 0:n].astype(np.float64)
    img = np.zeros((n, n))
    for k in range(n_blobs):
        r = int(np.ceil(6 * sg[k]))
        x0, x1 = max(0, int(cx[k]) - r), min(n, int(cx[k]) + r + 1)
        y0, y1 = max(0, int(cy[k]) - r), min(n, int(cy[k]) + r + 1)
        img[y0:y1, x0:x1] += a[k] * np.exp(-((xx[y0:y1, x0:x1] - cx[k]) ** 2 + (yy[y0:y1, x0:x1] - cy[k]) ** 2)
                                           / (2 * sg[k] ** 2))
    return img


def random_image(n, seed=0, stream=7):
    """Complex image with iid N(0,1) + i N(0,1) pixels."""
    return complex_normal(n * n, seed, stream).reshape(n, n)
