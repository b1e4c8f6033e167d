"""Seeded parity cases shared by the GPU tests: inputs from the generators,
expected values from the FP64 oracle only (never from the CUDA path)."""
from __future__ import annotations

import numpy as np

from oracle import pwf_oracle as O
from paper_2503_20146_gb300 import synth as S


def to_c64(a):
    return np.ascontiguousarray(a, dtype=np.complex64)


def to_f32(a):
    return np.ascontiguousarray(a, dtype=np.float32)


def geometry(w: S.Workload, ny=None, nx=None, xcoh=None, eta=None):
    xc = w.xcoh_m if xcoh is None else xcoh
    return O.Geometry(ny or w.ny, nx or w.nx, w.pixel_m, w.wavelength_m, w.L1_m, w.L2_m, xc,
                      xc if xcoh is not None else w.ycoh_m, w.gamma, w.alpha, w.eta if eta is None else eta)


def blob_batch(w: S.Workload, batch: int, ny=None, nx=None, seed_proj0=0):
    """psi_true [B], shared t, at (ny, nx) (defaults: the workload's)."""
    ny, nx = ny or w.ny, nx or w.nx
    rng_t = S.rng_for(w.config, 99)
    t = S.diffuser(ny, nx, rng_t)
    psis = [S.complex_phase_from(S.blob_phase(ny, nx, S.rng_for(w.config, seed_proj0 + b))) for b in range(batch)]
    return np.stack(psis), t


def measurement(psi_true_b, t, geom, photons, config):
    """y = Poisson(photons * f(psi_true)) / photons, f from the oracle."""
    f = O.intensity_batch(psi_true_b, t, geom)
    return np.stack([S.poisson_measurement(f[b], photons, S.rng_for(config, 50 + b)) for b in range(len(f))])


def rel_l2(a, b):
    a = np.asarray(a)
    b = np.asarray(b)
    return float(np.linalg.norm((a - b).ravel()) / np.linalg.norm(b.ravel()))


def phase_rms(psi_a, psi_b):
    d = np.asarray(psi_a).imag - np.asarray(psi_b).imag
    return float(np.sqrt(np.mean(d ** 2)))
