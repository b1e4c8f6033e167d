"""Pins of the FBP oracle (CPU only): the Ram-Lak kernel against the ramp it
samples, and reconstructions of objects whose projections are known in closed
form (a uniform disc; ellipsoids from the phantom generator's exact chords)."""
import math

import numpy as np
import pytest

from oracle import fbp_oracle as F
from paper_2503_20146_gb300 import synth as S


def test_ramlak_kernel_spectrum_is_the_ramp():
    # sum_k h(k) e^{-i w k} = |w| / (2 pi) on [-pi, pi]; truncating the kernel at
    # |k| < n drops at most sum_{k >= n, odd} 2 / (pi^2 k^2) <= 1 / (pi^2 (n - 1))
    n = 2049
    h = F.ramlak_kernel(n)
    k = np.arange(-(n - 1), n)
    w = np.linspace(-math.pi, math.pi, 101)
    H = (h[None, :] * np.cos(w[:, None] * k[None, :])).sum(axis=1)
    assert np.max(np.abs(H - np.abs(w) / (2 * math.pi))) < 1.0 / (math.pi ** 2 * (n - 1))


def _disc_sinogram(n, R, x0, z0, angles):
    s = F.detector_coords(n)
    out = np.zeros((len(angles), n))
    for a, th in enumerate(angles):
        d = s - (x0 * math.cos(th) + z0 * math.sin(th))
        out[a] = 2.0 * np.sqrt(np.clip(R * R - d * d, 0.0, None))
    return out


def test_fbp_recovers_an_off_axis_uniform_disc():
    n, R, x0, z0 = 128, 22.0, 25.0, -12.0
    angles = np.deg2rad(np.arange(180.0))
    f = F.fbp_slice(_disc_sinogram(n, R, x0, z0, angles), angles)
    c = F.detector_coords(n)
    dist = np.hypot(c[None, :] - x0, c[:, None] - z0)
    inside, outside = dist < R - 3, (dist > R + 3) & (np.hypot(c[None, :], c[:, None]) < n / 2 - 4)
    assert abs(f[inside].mean() - 1.0) < 0.01
    assert np.max(np.abs(f[inside] - 1.0)) < 0.05
    # point samples of a disc's chords alias: streaks of a few per cent outside
    assert np.max(np.abs(f[outside])) < 0.08 and np.mean(np.abs(f[outside])) < 0.015
    # the mirrored position stays empty: the angle convention matches the projector
    assert np.abs(f[np.hypot(c[None, :] + x0, c[:, None] + z0) < R - 3]).max() < 0.08


def test_fbp_recovers_an_off_axis_gaussian_to_high_accuracy():
    # f = exp(-r^2 / (2 s^2)) has the projection sqrt(2 pi) s exp(-d^2 / (2 s^2));
    # what remains is the linear interpolation of the back projection, about
    # 7e-3 at s = 5 px (it halves at s = 7 px and does not depend on n or the
    # number of angles)
    n, sg, x0, z0 = 96, 5.0, -11.0, 7.0
    angles = np.deg2rad(np.arange(0.0, 180.0, 0.5))
    s = F.detector_coords(n)
    sino = np.stack([math.sqrt(2 * math.pi) * sg * np.exp(-(s - x0 * math.cos(t) - z0 * math.sin(t)) ** 2 / (2 * sg * sg))
                     for t in angles])
    f = F.fbp_slice(sino, angles)
    c = F.detector_coords(n)
    truth = np.exp(-((c[None, :] - x0) ** 2 + (c[:, None] - z0) ** 2) / (2 * sg * sg))
    disc = np.hypot(c[None, :], c[:, None]) < n / 2 - 2
    assert np.max(np.abs(f - truth)[disc]) < 1e-2, np.max(np.abs(f - truth)[disc])


def _phantom():
    """Three large ellipsoids in a 96-voxel volume (orientations random, seeded)."""
    rng = np.random.default_rng(7)
    cen = np.array([[12.0, 0.0, -8.0], [-15.0, 2.0, 10.0], [5.0, -1.0, 18.0]])
    rot = np.stack([S._random_rotation(rng) for _ in range(3)])
    ax = np.array([[20.0, 14.0, 11.0], [12.0, 16.0, 9.0], [10.0, 8.0, 13.0]])
    dl = np.array([6e-7, 3e-7, 9e-7])
    return S.EllipsoidPhantom(96, cen, rot, ax, dl, 0.01 * dl)


def _phantom_slice(ph, y, n):
    c = F.detector_coords(n)
    X, Z = np.meshgrid(c, c)                       # [z][x]
    dl = np.zeros((n, n))
    depth = np.full((n, n), np.inf)                # distance inside the nearest boundary
    for i in range(len(ph.delta)):
        R = ph.rotations[i]
        A = R @ np.diag(1.0 / ph.semi_axes[i] ** 2) @ R.T
        m = np.stack([X - ph.centres[i][0], np.full_like(X, y - ph.centres[i][1]), Z - ph.centres[i][2]], -1)
        qf = np.einsum("...i,ij,...j->...", m, A, m)
        dl = dl + ph.delta[i] * (qf <= 1.0)
        depth = np.minimum(depth, np.abs(np.sqrt(qf) - 1.0) * ph.semi_axes[i].min())
    return dl, depth


def test_fbp_of_phantom_projections_recovers_delta_and_beta():
    ph = _phantom()
    n, rows = 96, (40, 47, 55)
    angles = np.deg2rad(np.arange(180.0))
    xd, _ = S.detector_grid(1, n)
    psi = np.zeros((len(angles), len(rows), n), dtype=np.complex128)
    for a, th in enumerate(angles):
        for r, row in enumerate(rows):
            yd = np.array([[row - n / 2 + 0.5]])
            re, im = S.ellipsoid_projection(ph, th, xd, yd, S.WAVELENGTH_20KEV_M, S.PIXEL_M)
            psi[a, r] = re[0] + 1j * im[0]
    vol = F.fbp_volume(psi, angles, S.WAVELENGTH_20KEV_M, S.PIXEL_M)
    for r, row in enumerate(rows):
        truth, depth = _phantom_slice(ph, row - n / 2 + 0.5, n)
        deep = depth > 3.0                          # 3 px or more from every surface
        inside = deep & (truth > 0)
        assert inside.sum() > 100
        err_d = np.abs(vol[r].imag[deep] - truth[deep])
        err_b = np.abs(vol[r].real[deep] - 0.01 * truth[deep])
        # edge streaks of point-sampled chords reach ~6 % of the largest delta
        assert np.max(err_d) < 0.08 * ph.delta.max(), np.max(err_d)
        assert np.mean(err_d) < 0.015 * ph.delta.max()
        assert np.max(err_b) < 0.08 * 0.01 * ph.delta.max()
        # the scale lambda / (2 pi p) and the sign: interior values within 1.5 %
        assert abs(np.mean(vol[r].imag[inside] / truth[inside]) - 1.0) < 0.015
        assert abs(np.mean(vol[r].real[inside] / (0.01 * truth[inside])) - 1.0) < 0.015


def test_fbp_is_linear_and_takes_complex_fields():
    rng = np.random.default_rng(3)
    angles = np.deg2rad(np.arange(0.0, 180.0, 6.0))
    a = rng.standard_normal((30, 24))
    b = rng.standard_normal((30, 24))
    fc = F.fbp_slice(a + 1j * b, angles)
    assert np.allclose(fc.real, F.fbp_slice(a, angles), atol=1e-12)
    assert np.allclose(fc.imag, F.fbp_slice(b, angles), atol=1e-12)


@pytest.mark.parametrize("bad", ["swap_trig", "no_weight", "kernel_sign"])
def test_planted_fbp_mistakes_are_caught(monkeypatch, bad):
    if bad == "swap_trig":
        orig = F.backproject

        def swapped(q, angles):
            return orig(q, math.pi / 2 - np.asarray(angles))
        monkeypatch.setattr(F, "backproject", swapped)
    elif bad == "no_weight":
        orig = F.backproject
        monkeypatch.setattr(F, "backproject", lambda q, ang: orig(q, ang) * len(ang) / math.pi)
    else:
        orig = F.ramlak_kernel

        def flipped(n):
            h = orig(n)
            h[n - 1] = -h[n - 1]
            return h
        monkeypatch.setattr(F, "ramlak_kernel", flipped)
    with pytest.raises(AssertionError):
        test_fbp_recovers_an_off_axis_gaussian_to_high_accuracy()
