"""Seeded random fields with an energy spectrum falling as k^slope (default -3),
the spectral shape the paper's synthetic and model data share (Sect. 4-5)."""

import numpy as np
import torch


def log_wavenumbers(lam_max, lam_min, count):
    """`count` wavenumbers k = 2*pi/lambda, log-spaced between 2*pi/lam_max and
    2*pi/lam_min, ascending (radians per length unit)."""
    return np.geomspace(2 * np.pi / lam_max, 2 * np.pi / lam_min, count)


def grf_periodic(nx, ny, h=1.0, seed=1, slope=-3.0):
    """Gaussian random field on the nx*ny periodic grid of spacing h.

    Fourier coefficient of mode kappa has a random Gaussian value times
    |kappa|^((slope-1)/2) (so the isotropic 2-D spectrum E(k) ~ k^slope); the
    mean mode is zero.  Values at the grid points (i*h, j*h), array [ny*nx]
    in vertex order j*nx + i."""
    rng = np.random.default_rng(seed)
    kx = 2 * np.pi * np.fft.fftfreq(nx, d=h)
    ky = 2 * np.pi * np.fft.fftfreq(ny, d=h)
    KX, KY = np.meshgrid(kx, ky, indexing="xy")
    kk = np.sqrt(KX ** 2 + KY ** 2)
    amp = np.zeros_like(kk)
    nz = kk > 0
    amp[nz] = kk[nz] ** ((slope - 1.0) / 2.0)
    c = (rng.normal(size=kk.shape) + 1j * rng.normal(size=kk.shape)) * amp
    f = np.real(np.fft.ifft2(c))
    f /= np.sqrt(np.mean(f ** 2))
    return f.ravel().astype(np.float64)


def grf_sphere(points, seed=13, n_features=512, k_min=None, k_max=None, slope=-3.0,
               chunk=1 << 18):
    """Random-Fourier-feature field evaluated at 3-D points (on a sphere).

    f(x) = sum_i a_i cos(kappa_i . x + theta_i) with directions uniform on the
    sphere, |kappa_i| log-uniform in [k_min, k_max] and a_i ~ |kappa_i|^((slope+1)/2),
    so that the energy per logarithmic band scales as k^(slope+1) (E(k) ~ k^slope).
    Returned with unit RMS, float64 [P]."""
    pts = np.asarray(points, dtype=np.float64)
    r = np.linalg.norm(pts[0])
    if k_min is None:
        k_min = 2 * np.pi / (np.pi * r)
    if k_max is None:
        k_max = 2 * np.pi / (r * 0.01)
    rng = np.random.default_rng(seed)
    d = rng.normal(size=(n_features, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    kmag = np.exp(rng.uniform(np.log(k_min), np.log(k_max), size=n_features))
    kap = d * kmag[:, None]
    theta = rng.uniform(0, 2 * np.pi, size=n_features)
    amp = kmag ** ((slope + 1.0) / 2.0) * rng.normal(size=n_features)
    dev = "cuda" if (pts.shape[0] > 2_000_000 and torch.cuda.is_available()) else "cpu"
    kap_t = torch.tensor(kap, device=dev)
    th_t = torch.tensor(theta, device=dev)
    amp_t = torch.tensor(amp, device=dev)
    out = np.empty(pts.shape[0], dtype=np.float64)
    for s in range(0, pts.shape[0], chunk):
        x = torch.tensor(pts[s:s + chunk], device=dev)
        ph = (x[:, 0:1] * kap_t[:, 0] + x[:, 1:2] * kap_t[:, 1] + x[:, 2:3] * kap_t[:, 2]) + th_t
        out[s:s + chunk] = (torch.cos(ph) * amp_t).sum(dim=1).cpu().numpy()
    out /= np.sqrt(np.mean(out ** 2))
    return out
