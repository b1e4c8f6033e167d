"""Oracle work for the workload-size parity tests, run in worker processes.

Every function here takes seeds and sizes (or arrays the oracle itself
produced) and returns FP64 oracle results; none of them receives anything
computed by the CUDA path. They are module-level so that a ``spawn`` process
pool can import them; numpy's FFT runs single-threaded, so one worker per core
keeps the host busy while the GPU side of a test runs.
"""
from __future__ import annotations

import numpy as np

from oracle import pwf_oracle as O
from paper_2503_20146_gb300 import synth as S

from _cases import blob_batch, geometry, to_c64

SIGMA = 2.0


def pool(max_workers=None):
    import multiprocessing as mp
    import os
    from concurrent.futures import ProcessPoolExecutor
    n = max_workers or max(2, min(16, os.cpu_count() or 2))
    return ProcessPoolExecutor(max_workers=n, mp_context=mp.get_context("spawn"))


# ----------------------------------------------------------------------------
# tomographic series (180 x 1024^2 ellipsoid phantom)
# ----------------------------------------------------------------------------
def tomo_t32(n=1024):
    w = S.WORKLOADS["tomo180x1024_iotf"]
    return to_c64(S.diffuser(n, n, S.rng_for(w.config, 99)))


def tomo_measurement(b, n=1024, n_angles=180):
    """y of projection b: Poisson(photons f(psi_true)) / photons with f the
    oracle's forward model (IOTF form) of the phantom's projection."""
    w = S.WORKLOADS["tomo180x1024_iotf"]
    ph = S.ellipsoid_phantom(S.rng_for(w.config, 0), size=n)
    xd, yd = S.detector_grid(n, n)
    re, im = S.ellipsoid_projection(ph, float(S.tomo_angles(n_angles)[b]), xd, yd, w.wavelength_m)
    f = O.intensity(re + 1j * im, tomo_t32(n).astype(np.complex128), geometry(w))
    return S.poisson_measurement(f, w.photons, S.rng_for(w.config, 50 + b)).astype(np.float32)


def tomo_solve(b, iters, n_modes=0):
    """Oracle iterate after ``iters`` iterations on projection b of the series
    (IOTF form, or n_modes source modes), from its own measurement."""
    w = S.WORKLOADS["tomo180x1024_iotf"]
    y = tomo_measurement(b).astype(np.float64)
    t = tomo_t32().astype(np.complex128)
    geom = geometry(w)
    if n_modes > 1:
        return O.modal_solve(y, t, geom, O.source_modes(geom, n_modes, SIGMA), iters).psi
    return O.solve(y, t, geom, iters).psi


# ----------------------------------------------------------------------------
# single 512^2 projection with source modes
# ----------------------------------------------------------------------------
def blob_modal_measurement(n, K):
    w = S.WORKLOADS["blob512_iotf"]
    geom = geometry(w, n, n)
    psi_true, t = blob_batch(w, 1, n, n)
    t = to_c64(t)
    f = O.modal_intensity(psi_true[0], t.astype(np.complex128), geom, O.source_modes(geom, K, SIGMA))
    return S.poisson_measurement(f, w.photons, S.rng_for(w.config, 77)).astype(np.float32), t


def blob_modal_solve(n, K, iters):
    w = S.WORKLOADS["blob512_iotf"]
    geom = geometry(w, n, n)
    y, t = blob_modal_measurement(n, K)
    r = O.modal_solve(y.astype(np.float64), t.astype(np.complex128), geom, O.source_modes(geom, K, SIGMA), iters)
    return r.psi, r.losses


# ----------------------------------------------------------------------------
# differentiation workload (16 x 2048^2, K = 25)
# ----------------------------------------------------------------------------
def grad_inputs(seed=21):
    """(psi, t, weights) of the differentiation workload, float32-rounded."""
    w = S.WORKLOADS["grad16x2048_k25"]
    psi, t = blob_batch(w, w.batch, w.ny, w.nx)
    rng = np.random.default_rng(seed)
    t = t * (1.0 + 0.1 * rng.standard_normal(t.shape))
    wts = rng.standard_normal((w.batch, w.ny, w.nx)).astype(np.float32)
    return to_c64(psi), to_c64(t), wts


def _grad_geom():
    w = S.WORKLOADS["grad16x2048_k25"]
    geom = geometry(w)
    return geom, O.source_modes(geom, w.n_modes, w.mode_sigma_px)


def grad_vjp(b):
    """Oracle VJP (grad_psi, grad_t) of projection b for the cotangent weights."""
    psi, t, wts = grad_inputs()
    geom, modes = _grad_geom()
    return O.modal_forward_vjp(psi[b].astype(np.complex128), t.astype(np.complex128), wts[b].astype(np.float64),
                               geom, modes)


def grad_weighted_intensity(projs, eps, d_psi=None, d_t=None):
    """sum over projections in ``projs`` of sum(w_b f_b) at psi + eps d_psi
    (d_psi applied to projs[0] only) and t + eps d_t, in FP64."""
    psi, t, wts = grad_inputs()
    geom, modes = _grad_geom()
    t64 = t.astype(np.complex128) + (0 if d_t is None else eps * d_t)
    total = 0.0
    for k, b in enumerate(projs):
        p = psi[b].astype(np.complex128)
        if d_psi is not None and k == 0:
            p = p + eps * d_psi
        total += float(np.sum(wts[b].astype(np.float64) * O.modal_intensity(p, t64, geom, modes)))
    return total


# ----------------------------------------------------------------------------
# uneven batch (16 each of 256^2, 768^2, 1536^2, 2048^2; K = 25)
# ----------------------------------------------------------------------------
def mixed_class_t32(n):
    return to_c64(blob_batch(S.WORKLOADS["blob512_iotf"], 1, n, n)[1])


def mixed_projection(k, n, b, count=16):
    """(psi_true, photons) of projection b of size class k (n x n), a blob object."""
    w = S.WORKLOADS["mixed64_k25"]
    psi_true, _ = blob_batch(S.WORKLOADS["blob512_iotf"], 1, n, n, seed_proj0=100 * (k + 1) + b)
    return psi_true[0], S.mixed_photons(w.config, k * count + b)


def mixed_measurement(k, n, b, count=16):
    """y of projection b of class k from the oracle's IOTF forward model."""
    w = S.WORKLOADS["mixed64_k25"]
    psi_true, photons = mixed_projection(k, n, b, count)
    f = O.intensity(psi_true, mixed_class_t32(n).astype(np.complex128), geometry(w, n, n))
    return S.poisson_measurement(f, photons, S.rng_for(w.config, 400 + k * count + b)).astype(np.float32)


def mixed_solve(k, n, b, iters):
    """Oracle iterate of projection b of class k after ``iters`` iterations with
    the workload's 25 source modes."""
    w = S.WORKLOADS["mixed64_k25"]
    geom = geometry(w, n, n)
    y = mixed_measurement(k, n, b)
    return O.modal_solve(y.astype(np.float64), mixed_class_t32(n).astype(np.complex128), geom,
                         O.source_modes(geom, w.n_modes, w.mode_sigma_px), iters).psi
