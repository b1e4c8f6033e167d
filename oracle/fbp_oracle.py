"""FP64 CPU oracle of the tomographic step after PWF: filtered back projection.

TEST INFRASTRUCTURE ONLY (imported by ``tests/``, ``__graft_entry__.smoke()``
and the CPU-baseline leg of ``bench.py``; never by the CUDA library, with which
it shares no code).

Methods, "Reconstruction procedure": the retrieved fields are turned into a
tomogram by standard filtered back projection (FBP) with the Ram-Lak filter,
applied independently to every vertical position (detector row), and the
result is multiplied by lambda / p / (2 pi) to give delta and beta. The paper
names the method and calls a library routine; the definition written out here
is the textbook one for parallel-beam data (Kak and Slaney, "Principles of
Computerized Tomographic Imaging", ch. 3):

  * projection p_theta(s) sampled at s_j = j - n/2 + 1/2 (pixel units), the
    rotation axis between the two central pixels (the detector grid of the
    phantom generator);
  * band-limited ramp (Ram-Lak) kernel with unit sampling: h(0) = 1/4,
    h(k) = -1/(pi^2 k^2) for odd k, 0 for even k != 0;
  * filtered projection q = h * p, a LINEAR convolution over the n samples;
  * back projection f(x, z) = (pi / N_theta) sum_a q_a(x cos theta_a +
    z sin theta_a), q interpolated linearly between samples and zero outside
    the detector; the reconstruction grid has the detector's pixel pitch and
    centring, x along the detector row and z along the beam at theta = 0.

Readings (R15 in the design notes' numbering):
  * angles cover [0, pi) uniformly (the tomographic workload's 0..179 degrees);
  * psi = -k int beta - i k int delta, so FBP of psi scaled by
    -lambda / (2 pi p) gives beta + i delta (both parts at once, because the
    filter and the back projection are real and linear);
  * no interpolation beyond linear, no extra apodisation of the ramp, no
    low-frequency background correction (the paper's curvature removal is
    post-processing and out of scope).
"""
from __future__ import annotations

import math

import numpy as np


def ramlak_kernel(n: int) -> np.ndarray:
    """h(k) for k = -(n-1)..(n-1) (index k + n - 1), unit sampling interval."""
    k = np.arange(-(n - 1), n)
    h = np.zeros(2 * n - 1, dtype=np.float64)
    h[k == 0] = 0.25
    odd = (k % 2) != 0
    h[odd] = -1.0 / (math.pi ** 2 * k[odd].astype(np.float64) ** 2)
    return h


def ramp_filter(p: np.ndarray) -> np.ndarray:
    """q_j = sum_k h(j - k) p_k over the last axis (linear convolution)."""
    p = np.asarray(p)
    n = p.shape[-1]
    h = ramlak_kernel(n)
    flat = p.reshape(-1, n)
    out = np.empty(flat.shape, dtype=np.result_type(p.dtype, np.float64))
    for r in range(flat.shape[0]):
        out[r] = np.convolve(flat[r], h)[n - 1:2 * n - 1]
    return out.reshape(p.shape)


def detector_coords(n: int) -> np.ndarray:
    """Pixel-centre coordinates relative to the rotation axis."""
    return np.arange(n, dtype=np.float64) - n / 2 + 0.5


def backproject(q: np.ndarray, angles_rad: np.ndarray) -> np.ndarray:
    """f[z][x] = (pi / N) sum_a q_a(x cos theta_a + z sin theta_a) on the n x n
    grid; q is [N][n] (real or complex), linear interpolation, zero outside."""
    q = np.asarray(q)
    n_ang, n = q.shape
    c = detector_coords(n)
    x = c[None, :]
    z = c[:, None]
    f = np.zeros((n, n), dtype=np.result_type(q.dtype, np.float64))
    for a in range(n_ang):
        s = x * math.cos(angles_rad[a]) + z * math.sin(angles_rad[a])
        u = s + n / 2 - 0.5                      # fractional detector index
        j0 = np.floor(u).astype(np.int64)
        w = u - j0
        v0 = np.where((j0 >= 0) & (j0 < n), q[a][np.clip(j0, 0, n - 1)], 0.0)
        v1 = np.where((j0 + 1 >= 0) & (j0 + 1 < n), q[a][np.clip(j0 + 1, 0, n - 1)], 0.0)
        f = f + (1.0 - w) * v0 + w * v1
    return f * (math.pi / n_ang)


def fbp_slice(sino: np.ndarray, angles_rad: np.ndarray) -> np.ndarray:
    """One slice from its sinogram [N_theta][n]: ramp filter, then back projection."""
    return backproject(ramp_filter(sino), angles_rad)


def fbp_volume(psi: np.ndarray, angles_rad: np.ndarray, wavelength_m: float, voxel_m: float) -> np.ndarray:
    """beta + i delta, [ny][n][n] (slice y, then z, then x), from the retrieved
    fields psi [N_theta][ny][n]; every detector row is one slice."""
    psi = np.asarray(psi, dtype=np.complex128)
    n_ang, ny, n = psi.shape
    scale = -wavelength_m / (2.0 * math.pi * voxel_m)
    out = np.empty((ny, n, n), dtype=np.complex128)
    for y in range(ny):
        out[y] = fbp_slice(psi[:, y, :], angles_rad) * scale
    return out
