"""Seeded synthetic inputs for registration workloads.

This module only draws random numbers and builds test volumes (phantoms,
random band-limited velocity fields, noise).  It holds none of the
registration method's arithmetic: no shooting, no transport, no adjoint.
Both the CPU oracle tests and the GPU path consume what it returns.

Every generator takes a ``numpy.random.Generator`` and draws in a fixed order,
so one seed gives one volume on every machine.  All arrays are float64,
laid out ``[n0][n1][n2]`` (scalar) or ``[3][n0][n1][n2]`` (vector field),
axis 2 fastest, on the periodic box ``[0, l_a)`` with ``h_a = l_a / n_a``.
"""
from __future__ import annotations

import numpy as np

TWO_PI = 2.0 * np.pi


def rng_for(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def _voxel_coords(n):
    return np.meshgrid(*[np.arange(m, dtype=np.float64) for m in n], indexing="ij")


def _min_image(d, m):
    """Periodic minimum-image difference in voxel units."""
    return d - m * np.round(d / m)


def _random_rotation(rng):
    q, r = np.linalg.qr(rng.standard_normal((3, 3)))
    q = q @ np.diag(np.sign(np.diag(r)))
    if np.linalg.det(q) < 0:
        q[:, 0] = -q[:, 0]
    return q


def spectral_gaussian_smooth(f, sigma_vox):
    """Periodic Gaussian blur of a scalar volume, sigma in voxels."""
    n = f.shape
    k = [np.fft.fftfreq(n[0]), np.fft.fftfreq(n[1]), np.fft.rfftfreq(n[2])]
    g = np.exp(-0.5 * (TWO_PI * sigma_vox) ** 2 * (
        k[0][:, None, None] ** 2 + k[1][None, :, None] ** 2 + k[2][None, None, :] ** 2))
    return np.fft.irfftn(np.fft.rfftn(f) * g, s=n, axes=(0, 1, 2))


def blob_phantom(n, rng, nblobs=8, amp=(0.2, 1.0), sigma_vox=(2.0, 5.0)):
    """Sum of ``nblobs`` anisotropic, randomly rotated Gaussian blobs.

    Centre ~ U[0, n) voxels, amplitude ~ U(amp), per-axis sigma ~ U(sigma_vox)
    voxels, distances taken as periodic minimum images.
    """
    n = tuple(int(x) for x in n)
    x = _voxel_coords(n)
    img = np.zeros(n)
    for _ in range(nblobs):
        c = rng.uniform(0.0, 1.0, 3) * np.array(n)
        a = rng.uniform(*amp)
        s = rng.uniform(*sigma_vox, 3)
        rot = _random_rotation(rng)
        d = np.stack([_min_image(x[i] - c[i], n[i]) for i in range(3)])
        y = np.einsum("ij,j...->i...", rot.T, d)
        img += a * np.exp(-0.5 * ((y[0] / s[0]) ** 2 + (y[1] / s[1]) ** 2 + (y[2] / s[2]) ** 2))
    return img


def ellipsoid_phantom(n, rng, perturb_vox=0.0, smooth_vox=1.0):
    """Three nested random ellipsoids with intensities 0.2 / 0.5 / 0.9.

    Outer semi-axes ~ U(0.30, 0.42) of each axis length, middle = outer x
    U(0.6, 0.75), inner = outer x U(0.35, 0.5); one common random rotation;
    centre jittered by +-2 voxels.  With ``perturb_vox > 0`` every boundary is
    displaced by a sum of three random sinusoids of that amplitude (the
    "brain-shaped" variant).  The result is smoothed by a periodic Gaussian.
    """
    n = tuple(int(x) for x in n)
    x = _voxel_coords(n)
    nn = np.array(n, dtype=np.float64)
    outer = rng.uniform(0.30, 0.42, 3) * nn
    mid = outer * rng.uniform(0.6, 0.75)
    inner = outer * rng.uniform(0.35, 0.5)
    rot = _random_rotation(rng)
    c = nn / 2.0 + rng.uniform(-2.0, 2.0, 3)
    d = np.stack([_min_image(x[i] - c[i], n[i]) for i in range(3)])
    y = np.einsum("ij,j...->i...", rot.T, d)
    pert = np.zeros(n)
    if perturb_vox > 0.0:
        amps = rng.uniform(0.3, 1.0, 3)
        amps /= amps.max()
        for j in range(3):
            kv = rng.integers(-3, 4, 3)
            while np.linalg.norm(kv) == 0 or np.linalg.norm(kv) > 3:
                kv = rng.integers(-3, 4, 3)
            ph = rng.uniform(0.0, TWO_PI)
            arg = sum(TWO_PI * kv[i] * x[i] / n[i] for i in range(3)) + ph
            pert += amps[j] * np.sin(arg)
    img = np.zeros(n)
    for semi, level in ((outer, 0.2), (mid, 0.5), (inner, 0.9)):
        r = np.sqrt((y[0] / semi[0]) ** 2 + (y[1] / semi[1]) ** 2 + (y[2] / semi[2]) ** 2)
        r_mean = float(np.mean(semi))
        f = r - 1.0 - (perturb_vox / r_mean) * pert
        img = np.where(f < 0.0, level, img)
    if smooth_vox > 0.0:
        img = spectral_gaussian_smooth(img, smooth_vox)
    return img


def random_velocity(n, rng, kmax, max_disp_vox, lengths=None):
    """Random smooth periodic vector field band-limited to integer |k|_2 <= kmax.

    Each component gets complex normal Fourier coefficients on the integer
    wave vectors with 0 < |k|_2 <= kmax; the field is the real part of their
    Fourier synthesis, scaled so that ``max_x |v(x)|_2 = max_disp_vox * min(h)``.
    """
    n = tuple(int(x) for x in n)
    lengths = tuple(lengths) if lengths is not None else (TWO_PI,) * 3
    kr = int(np.floor(kmax))
    ks = np.arange(-kr, kr + 1)
    kk = np.stack(np.meshgrid(ks, ks, ks, indexing="ij"), -1).reshape(-1, 3)
    nrm = np.linalg.norm(kk, axis=1)
    kk = kk[(nrm > 0) & (nrm <= kmax)]
    v = np.zeros((3,) + n)
    for c in range(3):
        coef = rng.standard_normal(len(kk)) + 1j * rng.standard_normal(len(kk))
        spec = np.zeros(n, dtype=np.complex128)
        np.add.at(spec, (kk[:, 0] % n[0], kk[:, 1] % n[1], kk[:, 2] % n[2]), coef)
        v[c] = (np.fft.ifftn(spec) * spec.size).real
    h = min(L / m for L, m in zip(lengths, n))
    peak = np.sqrt((v ** 2).sum(0)).max()
    return v * (max_disp_vox * h / peak)


def band_limited_field(n, rng, kmax, ncomp=3, lengths=None):
    """Unit-L2 (grid mean-square one) random field band-limited to |k|_2 <= kmax."""
    n = tuple(int(x) for x in n)
    shape = (ncomp,) + n
    k = [np.fft.fftfreq(n[0]) * n[0], np.fft.fftfreq(n[1]) * n[1], np.fft.rfftfreq(n[2]) * n[2]]
    kn = np.sqrt(k[0][:, None, None] ** 2 + k[1][None, :, None] ** 2 + k[2][None, None, :] ** 2)
    spec = rng.standard_normal((ncomp,) + kn.shape) + 1j * rng.standard_normal((ncomp,) + kn.shape)
    spec = spec * (kn <= kmax)
    f = np.fft.irfftn(spec, s=n, axes=(-3, -2, -1))
    f /= np.sqrt(np.mean(f ** 2))
    return f.reshape(shape) if ncomp > 1 else f.reshape(n)


def noise(n, rng, sigma):
    return rng.normal(0.0, sigma, tuple(int(x) for x in n))


# ---------------------------------------------------------------------------
# Workload recipes (the phantom / velocity part; targets are produced by
# whoever runs the workload, from the velocity returned here).
# ---------------------------------------------------------------------------

def blob_pair_inputs(n, seed, kmax=4, max_disp_vox=2.0, lengths=None):
    """Blob phantom + random v0 (|k| <= kmax, peak displacement in voxels)."""
    rng = rng_for(seed)
    img = blob_phantom(n, rng)
    v0 = random_velocity(n, rng, kmax, max_disp_vox, lengths)
    return img, v0


def ellipsoid_pair_inputs(n, seed, kmax=6, max_disp_vox=6.0, noise_sigma=0.02,
                          perturb_vox=0.0, lengths=None):
    """Nested-ellipsoid phantom, random v0, and two independent noise draws.

    Returns ``(phantom, v0_true, noise_source, noise_target)``; the source is
    ``phantom + noise_source`` and the target is the warped phantom plus
    ``noise_target``.
    """
    rng = rng_for(seed)
    img = ellipsoid_phantom(n, rng, perturb_vox=perturb_vox)
    v0 = random_velocity(n, rng, kmax, max_disp_vox, lengths)
    n0 = noise(n, rng, noise_sigma)
    n1 = noise(n, rng, noise_sigma)
    return img, v0, n0, n1
