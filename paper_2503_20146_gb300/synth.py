"""Seeded synthetic inputs shaped like the paper's own simulations.

The paper validates PWF on a numerical phantom with Poisson noise (Fig. S7) and
on a numerically rotated phantom for tomography (Fig. S8). Its beamline data are
not available, so every workload here is synthetic and seeded.

This module holds NO arithmetic of the PWF method (no propagation, no forward
model, no gradient): only object phases, diffuser phase screens, ellipsoid
phantom line integrals and Poisson counting noise. Both the FP64 oracle and the
CUDA path take their inputs from here, so the generators are the one thing the
two sides share.

Seeds: ``numpy.random.default_rng(20146000 + 100 * config + proj)``.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

SEED_BASE = 20146000

# 20 keV photons: lambda = h c / E = 1.23984198e-6 eV m / 2e4 eV.
WAVELENGTH_20KEV_M = 1.23984198e-6 / 2.0e4
PIXEL_M = 1.0e-6
# Sample -> diffuser 0.1 m; sample -> detector 0.5 m, so diffuser -> detector 0.4 m.
L1_M = 0.1
L2_M = 0.4


def rng_for(config: int, proj: int = 0) -> np.random.Generator:
    """The seeded generator for projection ``proj`` of workload ``config``."""
    return np.random.default_rng(SEED_BASE + 100 * config + proj)


def xcoh_from_blur_sigma(sigma_px: float, pixel_m: float = PIXEL_M) -> float:
    """Coherence length whose intensity PSF is a Gaussian of std ``sigma_px``.

    The IPSF of Eq. (4) is proportional to exp(-2 pi x^2 / x_coh^2), a Gaussian
    of standard deviation x_coh / sqrt(4 pi). A blur of sigma pixels therefore
    corresponds to x_coh = sigma * sqrt(4 pi) pixels.
    """
    return sigma_px * math.sqrt(4.0 * math.pi) * pixel_m


# ----------------------------------------------------------------------------
# Object: sum of Gaussian blobs (Fig. S7-style phantom)
# ----------------------------------------------------------------------------
def blob_phase(ny: int, nx: int, rng: np.random.Generator, n_blobs: int = 8,
               peak_rad: float = 2.0, xp=np, device=None):
    """Phase map made of ``n_blobs`` Gaussian blobs, rescaled to max |phi| = peak.

    Centres are uniform in the central 80 % of the field, standard deviations
    uniform in [n/32, n/8] pixels (n = min(ny, nx)), amplitudes uniform in
    [-1, 1] before the rescale. The draws come from ``rng`` (numpy); the grid
    arithmetic runs on ``xp`` (numpy, or torch with ``device``).
    """
    n = min(ny, nx)
    kw = {} if xp is np else {"device": device}
    yy = xp.arange(ny, dtype=xp.float64, **kw)[:, None]
    xx = xp.arange(nx, dtype=xp.float64, **kw)[None, :]
    phi = xp.zeros((ny, nx), dtype=xp.float64, **kw)
    for _ in range(n_blobs):
        cy = rng.uniform(0.1 * ny, 0.9 * ny)
        cx = rng.uniform(0.1 * nx, 0.9 * nx)
        sd = rng.uniform(n / 32.0, n / 8.0)
        amp = rng.uniform(-1.0, 1.0)
        phi = phi + amp * xp.exp(-((yy - cy) ** 2 + (xx - cx) ** 2) / (2.0 * sd * sd))
    m = float(abs(phi).max())
    if m > 0:
        phi = phi * (peak_rad / m)
    return phi


def complex_phase_from(phi: np.ndarray, absorption_ratio: float = 0.05) -> np.ndarray:
    """psi = -ratio * phi + i phi, i.e. amplitude exp(-ratio * phi), phase phi."""
    return (-absorption_ratio * phi + 1j * phi).astype(np.complex128)


# ----------------------------------------------------------------------------
# Diffuser: random phase screen, Gaussian-correlated
# ----------------------------------------------------------------------------
def _periodic_gaussian_smooth(a: np.ndarray, sigma_px: float) -> np.ndarray:
    """Periodic Gaussian smoothing by separable circular convolution (direct sums)."""
    out = a
    for axis in (0, 1):
        n = a.shape[axis]
        half = min(n // 2, int(math.ceil(5 * sigma_px)))
        offs = np.arange(-half, half + 1)
        w = np.exp(-0.5 * (offs / sigma_px) ** 2)
        w /= w.sum()
        acc = np.zeros_like(out)
        for o, wk in zip(offs, w):
            acc += wk * np.roll(out, int(o), axis=axis)
        out = acc
    return out


def diffuser(ny: int, nx: int, rng: np.random.Generator, corr_px: float = 3.0,
             std_rad: float = 1.0) -> np.ndarray:
    """Pure-phase diffuser t = exp(i theta), |t| = 1.

    theta is white N(0, 1) noise smoothed (periodically) by a Gaussian of std
    ``corr_px`` pixels and rescaled to standard deviation ``std_rad``.
    """
    theta = rng.standard_normal((ny, nx))
    theta = _periodic_gaussian_smooth(theta, corr_px)
    theta -= theta.mean()
    theta *= std_rad / theta.std()
    return np.exp(1j * theta)


# ----------------------------------------------------------------------------
# Measurement noise
# ----------------------------------------------------------------------------
def poisson_measurement(intensity: np.ndarray, photons_per_px: float,
                        rng: np.random.Generator) -> np.ndarray:
    """y = Poisson(photons * I) / photons, in flat-field units (mean ~ 1)."""
    lam = np.clip(photons_per_px * np.asarray(intensity, dtype=np.float64), 0.0, None)
    return rng.poisson(lam).astype(np.float64) / photons_per_px


# ----------------------------------------------------------------------------
# Ellipsoid phantom for a tomographic series (Fig. S8-style)
# ----------------------------------------------------------------------------
@dataclass
class EllipsoidPhantom:
    """Random ellipsoids in a cubic volume of ``size`` voxels (1 voxel = 1 pixel).

    Coordinates are in voxels with the origin at the volume centre; the rotation
    axis is the y axis (detector rows).
    """
    size: int
    centres: np.ndarray = field(repr=False)    # [n, 3] (x, y, z)
    rotations: np.ndarray = field(repr=False)  # [n, 3, 3]
    semi_axes: np.ndarray = field(repr=False)  # [n, 3]
    delta: np.ndarray = field(repr=False)      # [n]
    beta: np.ndarray = field(repr=False)       # [n]


def _random_rotation(rng: np.random.Generator) -> np.ndarray:
    q, r = np.linalg.qr(rng.standard_normal((3, 3)))
    q = q @ np.diag(np.sign(np.diag(r)))
    if np.linalg.det(q) < 0:
        q[:, 0] = -q[:, 0]
    return q


def ellipsoid_phantom(rng: np.random.Generator, size: int = 1024, n_ellipsoids: int = 40,
                      axis_range=(20.0, 150.0), delta_range=(1e-7, 1e-6),
                      beta_over_delta: float = 0.01) -> EllipsoidPhantom:
    """Seeded phantom: centres within radius 0.4*size of the rotation axis,
    |y| <= 0.4*size, semi-axes U[axis_range] voxels (scaled by size/1024),
    random orientation, delta U[delta_range], beta = delta/100."""
    scale = size / 1024.0
    cen = np.zeros((n_ellipsoids, 3))
    rot = np.zeros((n_ellipsoids, 3, 3))
    ax = np.zeros((n_ellipsoids, 3))
    dl = np.zeros(n_ellipsoids)
    for i in range(n_ellipsoids):
        rad = 0.4 * size * math.sqrt(rng.uniform(0.0, 1.0))
        ang = rng.uniform(0.0, 2.0 * math.pi)
        cen[i] = (rad * math.cos(ang), rng.uniform(-0.4 * size, 0.4 * size),
                  rad * math.sin(ang))
        rot[i] = _random_rotation(rng)
        ax[i] = rng.uniform(axis_range[0], axis_range[1], size=3) * scale
        dl[i] = rng.uniform(delta_range[0], delta_range[1])
    return EllipsoidPhantom(size, cen, rot, ax, dl, beta_over_delta * dl)


def ellipsoid_chord_coefficients(ph: EllipsoidPhantom, angle_rad: float):
    """Per-ellipsoid quadratic coefficients of the ray/ellipsoid intersection.

    For the detector pixel at (xd, yd) (voxels from the axis) the ray in the
    rotated sample frame is o + s d. With A = R diag(1/a^2) R^T and m = o - c,
    the chord length is 2 sqrt(max(b^2 - a c, 0)) / a with
    a = d^T A d, b = d^T A m, c = m^T A m - 1. Both b and c are polynomials
    in (xd, yd); this returns their coefficients so the evaluation over the
    pixel grid can run on any array library.
    """
    ca, sa = math.cos(angle_rad), math.sin(angle_rad)
    # Rotating the sample by +angle about y equals rotating the ray by -angle.
    ex = np.array([ca, 0.0, sa])    # R_y(-angle) (1, 0, 0)
    ey = np.array([0.0, 1.0, 0.0])
    d = np.array([-sa, 0.0, ca])    # R_y(-angle) (0, 0, 1)
    out = []
    for i in range(len(ph.delta)):
        R = ph.rotations[i]
        A = R @ np.diag(1.0 / ph.semi_axes[i] ** 2) @ R.T
        c = ph.centres[i]
        qa = d @ A @ d
        # b = d^T A (xd ex + yd ey - c)
        bx, by, b0 = d @ A @ ex, d @ A @ ey, -(d @ A @ c)
        # c = (xd ex + yd ey - c)^T A (...) - 1
        cxx, cyy, cxy = ex @ A @ ex, ey @ A @ ey, 2.0 * (ex @ A @ ey)
        cx, cy = -2.0 * (ex @ A @ c), -2.0 * (ey @ A @ c)
        c0 = c @ A @ c - 1.0
        out.append((qa, bx, by, b0, cxx, cyy, cxy, cx, cy, c0,
                    float(ph.delta[i]), float(ph.beta[i])))
    return out


def ellipsoid_projection(ph: EllipsoidPhantom, angle_rad: float, xd, yd, wavelength_m: float,
                         voxel_m: float = PIXEL_M):
    """Complex phase psi = -k int beta - i k int delta for one projection angle.

    ``xd`` and ``yd`` are broadcastable coordinate grids in voxels, numpy arrays
    or torch tensors; the arithmetic uses only operators both libraries share.
    Returns (re, im) so the caller chooses the complex dtype.
    """
    k = 2.0 * math.pi / wavelength_m
    int_delta = 0.0 * xd * yd
    int_beta = 0.0 * xd * yd
    for (qa, bx, by, b0, cxx, cyy, cxy, cx, cy, c0, dl, bt) in \
            ellipsoid_chord_coefficients(ph, angle_rad):
        b = bx * xd + by * yd + b0
        c = cxx * xd * xd + cyy * yd * yd + cxy * xd * yd + cx * xd + cy * yd + c0
        disc = (b * b - qa * c).clip(min=0.0)
        chord = (2.0 * voxel_m / qa) * disc ** 0.5
        int_delta = int_delta + dl * chord
        int_beta = int_beta + bt * chord
    return -k * int_beta, -k * int_delta


def detector_grid(ny: int, nx: int, xp=np):
    """Pixel-centre coordinates (voxels) relative to the rotation axis."""
    if xp is np:
        yd = (np.arange(ny, dtype=np.float64) - ny / 2 + 0.5)[:, None]
        xd = (np.arange(nx, dtype=np.float64) - nx / 2 + 0.5)[None, :]
        return xd, yd
    import torch  # noqa: F401  (only when a torch grid is requested)
    yd = (xp.arange(ny, dtype=xp.float64) - ny / 2 + 0.5)[:, None]
    xd = (xp.arange(nx, dtype=xp.float64) - nx / 2 + 0.5)[None, :]
    return xd, yd


# ----------------------------------------------------------------------------
# Named workloads
# ----------------------------------------------------------------------------
@dataclass(frozen=True)
class Workload:
    """Sizes, geometry and solver settings of one synthetic workload."""
    name: str
    config: int
    batch: int
    ny: int
    nx: int
    n_iter: int
    xcoh_m: float
    ycoh_m: float
    photons: float
    wavelength_m: float = WAVELENGTH_20KEV_M
    pixel_m: float = PIXEL_M
    L1_m: float = L1_M
    L2_m: float = L2_M
    gamma: float = 1.0
    alpha: complex = 0.1 + 0.01j
    # Step size: the largest power of two for which the FP64 oracle's loss on
    # the blob workloads stays bounded (the paper's eta = 1 belongs to its own
    # geometry, lambda L2 / p^2 ~ 6, against ~25 here).
    eta: float = 2.0 ** -9
    # source-mode variant of partial coherence (0: the paper's IOTF form)
    n_modes: int = 0
    mode_sigma_px: float = 0.0

    @property
    def mpx_per_iter(self) -> float:
        return self.batch * self.ny * self.nx / 1e6


WORKLOADS = {
    # Single projection, fully coherent (IOTF = 1), blob object.
    "blob128_coherent": Workload("blob128_coherent", 1, 1, 128, 128, 50, 0.0, 0.0, 1e4,
                                 eta=2.0 ** -10),
    # Single projection, Gaussian partial coherence of sigma = 2 px.
    "blob512_iotf": Workload("blob512_iotf", 2, 1, 512, 512, 100,
                             xcoh_from_blur_sigma(2.0), xcoh_from_blur_sigma(2.0), 1e4),
    # Tomographic series: 180 angles over [0, 180) degrees of an ellipsoid phantom.
    "tomo180x1024_iotf": Workload("tomo180x1024_iotf", 3, 180, 1024, 1024, 100,
                                  xcoh_from_blur_sigma(2.0), xcoh_from_blur_sigma(2.0), 1e4),
    # The same series with partial coherence as 9 tilted source modes (sigma = 2 px).
    "tomo180x1024_k9": Workload("tomo180x1024_k9", 3, 180, 1024, 1024, 100,
                                xcoh_from_blur_sigma(2.0), xcoh_from_blur_sigma(2.0), 1e4,
                                n_modes=9, mode_sigma_px=2.0),
    # Differentiation workload: 16 projections at 2048^2.
    "grad16x2048_iotf": Workload("grad16x2048_iotf", 4, 16, 2048, 2048, 1,
                                 xcoh_from_blur_sigma(2.0), xcoh_from_blur_sigma(2.0), 1e4),
    # Uneven batch: 16 projections each of 256^2, 768^2, 1536^2, 2048^2 (one
    # plan per size class in a group), 25 source modes, photons log-uniform in
    # [1e3, 1e5] per projection.
    "mixed64_k25": Workload("mixed64_k25", 5, 64, 0, 0, 100,
                            xcoh_from_blur_sigma(2.0), xcoh_from_blur_sigma(2.0), 0.0,
                            n_modes=25, mode_sigma_px=2.0),
    "grad16x2048_k25": Workload("grad16x2048_k25", 4, 16, 2048, 2048, 1,
                                xcoh_from_blur_sigma(2.0), xcoh_from_blur_sigma(2.0), 1e4,
                                n_modes=25, mode_sigma_px=2.0),
}


def blob_case(w: Workload, proj: int = 0):
    """(psi_true, t) for a blob workload projection; t is shared (drawn from proj 0)."""
    rng_t = rng_for(w.config, 99)
    t = diffuser(w.ny, w.nx, rng_t)
    rng = rng_for(w.config, proj)
    psi = complex_phase_from(blob_phase(w.ny, w.nx, rng))
    return psi, t


MIXED_SIZES = (256, 768, 1536, 2048)
MIXED_PER_SIZE = 16


def mixed_photons(config: int, index: int) -> float:
    """Photons per pixel of projection ``index`` of the uneven batch: log-uniform in [1e3, 1e5]."""
    return float(np.exp(rng_for(config, 300 + index).uniform(np.log(1e3), np.log(1e5))))


def tomo_angles(n: int) -> np.ndarray:
    """n projection angles evenly covering [0, 180) degrees, in radians."""
    return np.arange(n, dtype=np.float64) * (math.pi / n)
