"""FP64 CPU oracle of preconditioned Wirtinger flow (PWF), arXiv 2503.20146.

TEST INFRASTRUCTURE ONLY. This module is imported by ``tests/``, by
``__graft_entry__.smoke()`` and by the CPU-baseline / reference leg of
``bench.py``. The CUDA library never calls it, links it or imports it, and it
shares no code with the CUDA path: only the seeded input generators of
``paper_2503_20146_gb300.synth`` serve both.

What it computes, in the paper's order and notation:
  * Algorithm S1 (PWF): psi = 0, phi = 0, mu = 1; per iteration the physical
    model, residual e = y - f, Wirtinger derivative, preconditioner plus
    regularizer, and Nesterov's update.
  * Algorithm S2: PhysicalModel, WirtingerDerivative, Preconditioner,
    Regularizer, FreePropagation and Filter.
  * Eq. (1) forward model, Eq. (2) loss, Eq. (5) IOTF, Eq. (11)
    preconditioning filter, Eqs. (14)-(15) STF and regularization window.
Every array is complex128 / float64; numpy's FFT is the one library primitive
(Filter of Algorithm S2 is F^-1{F{x} W}, circular, no padding).

Readings where the paper is silent or ambiguous (R1 onwards, the numbering the design notes use):
  R1  FreePropagation: Q = exp(i 2 pi w L) carries the constant piston
      exp(i 2 pi L / lambda). It is a global phase that cancels in |v|^2 and in
      the back-propagation, so it is dropped, and w - 1/lambda is evaluated in
      the cancellation-free form -rho^2 / (1/lambda + w).
  R2  Bins with rho^2 > lambda^-2 (evanescent) get Q = 0. None occur at the
      geometries used here, so P(-L) = conj(Q) = the exact adjoint.
  R3  Frequencies u, v are numpy fftfreq in cycles per metre for Q, IOTF and
      STF (they multiply lengths in metres). For the preconditioner P^-1 =
      1/(u^2 + v^2) the units are not stated; it is evaluated in cycles per
      PIXEL, so P^-1 ranges over [2, N^2]. The overall scale is the step size's.
  R4  x_coh = y_coh = 0 means a fully coherent beam: IOTF = 1, STF = 1 and the
      regularization window Gamma^2 = 0 (the regularizer vanishes).
  R5  Filter of a real field (the intensity, the residual, Im g) keeps the real
      part of the inverse transform.
  R6  The stopping test compares the object fields x = exp(psi) of successive
      iterations by |<x_k, x_{k-1}>| / (||x_k|| ||x_{k-1}||); the threshold is
      10^(-0.00001) (Reconstruction procedure, Methods).
  R7  The gradient w.r.t. the diffuser (simultaneous retrieval, Methods and
      Fig. S12) is not printed; it is derived here from Eq. (1) in the same
      Wirtinger convention as the sample gradient.
  R13 K-mode variant (not the paper's form; a workload option): mutually
      incoherent tilted plane-wave modes of a Gaussian source replace the IPSF
      convolution. Nodes and weights are the tensor Gauss-Hermite rule of the
      standard normal (k1 = 1, 3, 5 per axis, K = k1^2); a node n walks the
      pattern by sigma n pixels at the detector, i.e. a tilt of
      sigma n p / (lambda (L1 + L2)) cycles/m, rounded to whole bins.
  R14 Calibration (Methods): g2 is the circular, line-averaged intensity
      autocorrelation over the squared mean; the Gaussian model is fitted in
      log space over lags 1..max_lag; the Wiener filter is IOTF/(IOTF^2 + eps);
      negative deconvolved intensities are clipped before the square root.
  R16 Joint diffuser refinement (Methods, "Diffuser transmission function",
      and Fig. S12: t shared by, and updated across, all projections). The
      update rule is not printed. Reading: after each iteration of Algorithm S1
      over the whole series, t <- t - eta_t sum_b g_t,b, a plain gradient step
      (no preconditioner, no momentum) with g_t the Wirtinger derivative of
      the loss w.r.t. conj(t) in Algorithm S2's normalisation (factor 2
      dropped, divided by max|t|^2 of the current t), evaluated at the same
      point as the sample gradient. Fixed iteration count (no stopping rule).
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

STOP_CORRELATION = 10.0 ** (-0.00001)


@dataclass(frozen=True)
class Geometry:
    """Inputs of Algorithm S1 other than y and t.

    Lengths in metres. ``xcoh``/``ycoh`` are the coherence lengths of Eqs. (4),
    (5) and (14); zero means fully coherent (reading R4).
    """
    ny: int
    nx: int
    pixel: float
    wavelength: float
    L1: float
    L2: float
    xcoh: float = 0.0
    ycoh: float = 0.0
    gamma: float = 1.0
    alpha: complex = 0.1 + 0.01j
    eta: float = 1.0


# ----------------------------------------------------------------------------
# Spatial frequencies and the filters of Algorithm S1's input list
# ----------------------------------------------------------------------------
def frequencies(geom: Geometry):
    """(u, v) grids in cycles/m, u along x (columns), v along y (rows)."""
    u = np.fft.fftfreq(geom.nx, d=geom.pixel)[None, :]
    v = np.fft.fftfreq(geom.ny, d=geom.pixel)[:, None]
    return u, v


def transfer_function(geom: Geometry, L: float) -> np.ndarray:
    """Q_k of FreePropagation (Algorithm S2), piston removed (reading R1).

    w = sqrt(lambda^-2 - u^2 - v^2); Q = exp(i 2 pi (w - 1/lambda) L) with
    w - 1/lambda = -rho^2 / (1/lambda + w), an exact identity.
    """
    u, v = frequencies(geom)
    inv_lam = 1.0 / geom.wavelength
    rho2 = u * u + v * v
    arg = inv_lam * inv_lam - rho2
    prop = arg > 0
    w = np.sqrt(np.where(prop, arg, 0.0))
    w_minus = -rho2 / (inv_lam + w)
    Q = np.exp(1j * 2.0 * np.pi * w_minus * L)
    return np.where(prop, Q, 0.0)          # reading R2


def transfer_function_literal(geom: Geometry, L: float) -> np.ndarray:
    """Q = exp(i 2 pi w L) exactly as printed, piston included (for the R1 pin)."""
    u, v = frequencies(geom)
    w = np.sqrt(1.0 / geom.wavelength ** 2 - u * u - v * v)
    return np.exp(1j * 2.0 * np.pi * w * L)


def iotf(geom: Geometry) -> np.ndarray:
    """IOTF_k = exp[-pi/2 (u^2 x_coh^2 + v^2 y_coh^2)], Eq. (5)."""
    u, v = frequencies(geom)
    return np.exp(-0.5 * np.pi * (u * u * geom.xcoh ** 2 + v * v * geom.ycoh ** 2))


def precond_filter(geom: Geometry) -> np.ndarray:
    """P^-1_k = 1/(u^2 + v^2), zero at u = v = 0, Eq. (11); cycles/pixel (R3)."""
    u = np.fft.fftfreq(geom.nx)[None, :]
    v = np.fft.fftfreq(geom.ny)[:, None]
    rho2 = u * u + v * v
    out = np.zeros((geom.ny, geom.nx))
    nz = rho2 > 0
    out[nz] = 1.0 / rho2[nz]
    return out


def stf(geom: Geometry) -> np.ndarray:
    """STF_k = exp[-pi gamma (u^2 x_coh^2 + v^2 y_coh^2)], Eq. (14)."""
    u, v = frequencies(geom)
    return np.exp(-np.pi * geom.gamma * (u * u * geom.xcoh ** 2 + v * v * geom.ycoh ** 2))


def reg_window(geom: Geometry) -> np.ndarray:
    """Gamma^2_k = 1 - STF_k, Eq. (15)."""
    return 1.0 - stf(geom)


# ----------------------------------------------------------------------------
# Algorithm S2
# ----------------------------------------------------------------------------
def Filter(x: np.ndarray, W: np.ndarray) -> np.ndarray:
    """x <- F^-1{ F{x} W } (Algorithm S2, Filter)."""
    return np.fft.ifft2(np.fft.fft2(x) * W)


def FreePropagation(x: np.ndarray, geom: Geometry, L: float) -> np.ndarray:
    """Angular-spectrum propagation over distance L (Algorithm S2)."""
    return Filter(x, transfer_function(geom, L))


def PhysicalModel(psi: np.ndarray, t: np.ndarray, geom: Geometry):
    """f(x), x, v of Algorithm S2 / Eq. (1)."""
    x = np.exp(psi)
    v = FreePropagation(x, geom, geom.L1)          # sample to diffuser
    v = FreePropagation(t * v, geom, geom.L2)      # diffuser to detector
    f = Filter(np.abs(v) ** 2, iotf(geom)).real    # IPSF convolution (R5)
    return f, x, v


def WirtingerDerivative(e, x, v, t, geom: Geometry) -> np.ndarray:
    """g of Algorithm S2: Filter(-e, IOTF), times v, back over L2, times t*,
    back over L1, times x*, divided by max |t|^2."""
    g = Filter(-e, iotf(geom)).real                # R5
    g = FreePropagation(v * g, geom, -geom.L2)
    g = FreePropagation(np.conj(t) * g, geom, -geom.L1)
    g = np.conj(x) * g
    g = g / np.max(np.abs(t) ** 2)
    return g


def Preconditioner(g: np.ndarray, Pinv: np.ndarray) -> np.ndarray:
    """Filter Im g with P^-1; keep Re g (Algorithm S2, Eq. (11))."""
    g2 = g.imag
    g2 = Filter(g2, Pinv).real                     # R5
    return g.real + 1j * g2


def Regularizer(psi: np.ndarray, Gamma2: np.ndarray, alpha: complex) -> np.ndarray:
    """rho = Filter(psi, Gamma^2); Re(alpha) Re(rho) + i Im(alpha) Im(rho)."""
    rho = Filter(psi, Gamma2)
    return alpha.real * rho.real + 1j * alpha.imag * rho.imag


def loss(y: np.ndarray, f: np.ndarray) -> float:
    """Sum_r (y_r - f_r)^2, Eq. (2)."""
    return float(np.sum((y - f) ** 2))


def correlation(x_new: np.ndarray, x_old: np.ndarray) -> float:
    """Normalised correlation of successive fields (reading R6)."""
    num = np.abs(np.vdot(x_old, x_new))
    den = np.sqrt(np.vdot(x_new, x_new).real * np.vdot(x_old, x_old).real)
    return float(num / den)


def nesterov_mu(mu: float) -> float:
    """mu <- (1 + sqrt(1 + 4 mu^2)) / 2 (Algorithm S1)."""
    return (1.0 + np.sqrt(1.0 + 4.0 * mu * mu)) / 2.0


# ----------------------------------------------------------------------------
# Algorithm S1
# ----------------------------------------------------------------------------
@dataclass
class PWFResult:
    psi: np.ndarray
    iterations: int
    losses: list          # loss of the model at the start of each iteration
    correlations: list    # correlation after each iteration


def pwf_iteration(psi, phi, mu, y, t, geom: Geometry, Pinv=None, Gamma2=None):
    """One pass of the while-loop body of Algorithm S1.

    Returns (psi_new, phi_new, mu_new, loss_before).
    """
    if Pinv is None:
        Pinv = precond_filter(geom)
    if Gamma2 is None:
        Gamma2 = reg_window(geom)
    phi_prev = phi
    mu_prev = mu
    f, x, v = PhysicalModel(psi, t, geom)
    e = y - f
    g = WirtingerDerivative(e, x, v, t, geom)
    g = Preconditioner(g, Pinv) + Regularizer(psi, Gamma2, geom.alpha)
    phi = psi - geom.eta * g
    mu = nesterov_mu(mu)
    psi_new = phi + ((mu_prev - 1.0) / mu) * (phi - phi_prev)
    return psi_new, phi, mu, loss(y, f)


def pwf(y: np.ndarray, t: np.ndarray, geom: Geometry, max_iter: int,
        corr_tol: float | None = None, psi0: np.ndarray | None = None) -> PWFResult:
    """Algorithm S1. ``corr_tol`` None runs exactly ``max_iter`` iterations;
    otherwise the loop also stops once the correlation exceeds ``corr_tol``."""
    psi = np.zeros((geom.ny, geom.nx), np.complex128) if psi0 is None else psi0.astype(np.complex128)
    phi = np.zeros_like(psi)
    mu = 1.0
    Pinv, Gamma2 = precond_filter(geom), reg_window(geom)
    losses, corrs = [], []
    it = 0
    while it < max_iter:
        x_old = np.exp(psi)
        psi, phi, mu, L = pwf_iteration(psi, phi, mu, y, t, geom, Pinv, Gamma2)
        it += 1
        losses.append(L)
        c = correlation(np.exp(psi), x_old)
        corrs.append(c)
        if corr_tol is not None and c > corr_tol:
            break
    return PWFResult(psi, it, losses, corrs)


# ----------------------------------------------------------------------------
# Gradient and vector-Jacobian products in PyTorch's convention
# ----------------------------------------------------------------------------
def gradient(psi, t, y, geom: Geometry):
    """(g, loss) with g the raw WirtingerDerivative output of Algorithm S2."""
    f, x, v = PhysicalModel(psi, t, geom)
    e = y - f
    return WirtingerDerivative(e, x, v, t, geom), loss(y, f)


def loss_gradient_real(psi, t, y, geom: Geometry):
    """dL/dRe(psi) + i dL/dIm(psi) of Eq. (2).

    Algorithm S2 drops the factor 2 of the Wirtinger calculus (Preconditioning
    filter section) and divides by max|t|^2, so the true gradient of the loss
    is 4 max|t|^2 g.
    """
    g, L = gradient(psi, t, y, geom)
    return 4.0 * np.max(np.abs(t) ** 2) * g, L


def forward_vjp(psi, t, grad_f, geom: Geometry):
    """Vector-Jacobian product of f = PhysicalModel(psi, t) for a real cotangent.

    Returns (grad_psi, grad_t) in the convention dL/dRe + i dL/dIm, for a
    scalar L with dL/df = grad_f. grad_psi reuses WirtingerDerivative with
    e = -grad_f / 2 (then scaled by 4 max|t|^2). grad_t (reading R7):
    f depends on t through v = P2{t u1}, u1 = P1{x}; dL = 2 Re<v G, P2{dt u1}>
    with G = Filter(grad_f, IOTF), so grad_t = 2 conj(u1) P2^H{v G}.
    """
    f, x, v = PhysicalModel(psi, t, geom)
    m = np.max(np.abs(t) ** 2)
    grad_psi = 4.0 * m * WirtingerDerivative(-0.5 * grad_f, x, v, t, geom)
    u1 = FreePropagation(x, geom, geom.L1)
    G = Filter(grad_f, iotf(geom)).real
    g2 = FreePropagation(v * G, geom, -geom.L2)
    grad_t = 2.0 * np.conj(u1) * g2
    return grad_psi, grad_t


def diffuser_gradient(psi, t, y, geom: Geometry):
    """g_t = conj(P1{x}) P2^H{ v Filter(-e, IOTF) } / max|t|^2 (reading R16):
    the diffuser counterpart of WirtingerDerivative, so that the gradient of
    the loss in the dL/dRe t + i dL/dIm t convention is 4 max|t|^2 g_t."""
    f, x, v = PhysicalModel(psi, t, geom)
    e = y - f
    G = Filter(-e, iotf(geom)).real                # R5
    g2 = FreePropagation(v * G, geom, -geom.L2)
    u1 = FreePropagation(x, geom, geom.L1)
    return np.conj(u1) * g2 / np.max(np.abs(t) ** 2)


@dataclass
class JointResult:
    psi: np.ndarray       # [B][ny][nx]
    t: np.ndarray         # refined diffuser
    losses: list          # total loss of the series at the start of each iteration


def joint_pwf(y_b, t0, geom: Geometry, max_iter: int, eta_t: float) -> JointResult:
    """Algorithm S1 over a series of projections that share the diffuser, with
    t refined after every iteration (reading R16)."""
    B = len(y_b)
    psi = np.zeros((B, geom.ny, geom.nx), np.complex128)
    phi = np.zeros_like(psi)
    mu = 1.0
    t = np.asarray(t0, np.complex128).copy()
    Pinv, Gamma2 = precond_filter(geom), reg_window(geom)
    losses = []
    for _ in range(max_iter):
        gt = np.zeros_like(t)
        total = 0.0
        mu_next = mu
        for b in range(B):
            gt = gt + diffuser_gradient(psi[b], t, y_b[b], geom)
            psi[b], phi[b], mu_next, L = pwf_iteration(psi[b], phi[b], mu, y_b[b], t, geom, Pinv, Gamma2)
            total += L
        mu = mu_next
        t = t - eta_t * gt
        losses.append(total)
    return JointResult(psi, t, losses)


# ----------------------------------------------------------------------------
# Batched helpers (independent projections, shared diffuser)
# ----------------------------------------------------------------------------
def physical_model_batch(psi_b, t, geom: Geometry) -> np.ndarray:
    return np.stack([PhysicalModel(p, t, geom)[0] for p in psi_b])


def gradient_batch(psi_b, t, y_b, geom: Geometry):
    gs, Ls = zip(*[gradient(p, t, y, geom) for p, y in zip(psi_b, y_b)])
    return np.stack(gs), np.array(Ls)


def forward_vjp_batch(psi_b, t, grad_f_b, geom: Geometry):
    """grad_t is summed over the batch: the diffuser is shared."""
    gp, gt = zip(*[forward_vjp(p, t, gf, geom) for p, gf in zip(psi_b, grad_f_b)])
    return np.stack(gp), np.sum(np.stack(gt), axis=0)


def pwf_batch(y_b, t, geom: Geometry, max_iter: int, corr_tol=None):
    return [pwf(y, t, geom, max_iter, corr_tol) for y in y_b]


# ----------------------------------------------------------------------------
# K-mode partial-coherence variant (a workload option, not the paper's form)
# ----------------------------------------------------------------------------
# The paper models partial coherence by the IPSF convolution of Eq. (1). The
# variant below instead sums the intensities of K mutually incoherent source
# modes: tilted plane waves s_j(r) = exp(i 2 pi q_j . r) with weights w_j,
#   f = sum_j w_j |P2{ t P1{ x s_j } }|^2,
# the tilts on a tensor Gauss-Hermite grid of a Gaussian source whose walk-off
# over L1 + L2 has standard deviation sigma pixels at the detector (reading
# R13). Tilts are rounded to whole frequency bins so that s_j is periodic on
# the grid. The gradient follows by the same Wirtinger calculus as Algorithm
# S2's WirtingerDerivative, with the IOTF filter replaced by the mode sum:
#   g = sum_j w_j conj(x s_j) P1^H{ conj(t) P2^H{ v_j (-e) } } / max|t|^2.
def gauss_hermite(k1: int):
    """Nodes and weights (summing to 1) of the k1-point Gauss-Hermite rule for
    the standard normal density (probabilists' Hermite polynomials)."""
    if k1 == 1:
        return np.array([0.0]), np.array([1.0])
    if k1 == 3:
        r3 = np.sqrt(3.0)
        return np.array([-r3, 0.0, r3]), np.array([1.0 / 6, 2.0 / 3, 1.0 / 6])
    if k1 == 5:
        a, b = np.sqrt(5.0 - np.sqrt(10.0)), np.sqrt(5.0 + np.sqrt(10.0))
        wa, wb = (7.0 + 2.0 * np.sqrt(10.0)) / 60.0, (7.0 - 2.0 * np.sqrt(10.0)) / 60.0
        return np.array([-b, -a, 0.0, a, b]), np.array([wb, wa, 8.0 / 15, wa, wb])
    raise ValueError("k1 must be 1, 3 or 5")


def source_modes(geom: Geometry, n_modes: int, sigma_px: float):
    """[(mx, my, w)] for K = n_modes = k1^2 modes: integer tilt bins along x and
    y and the weight. A detector walk-off of s metres needs the tilt
    q = s / (lambda (L1 + L2)) cycles/m, i.e. q N p bins."""
    k1 = int(round(np.sqrt(n_modes)))
    if k1 * k1 != n_modes:
        raise ValueError("n_modes must be a square (1, 9, 25)")
    nodes, weights = gauss_hermite(k1)
    z = geom.wavelength * (geom.L1 + geom.L2)
    modes = []
    for ny_i, wy in zip(nodes, weights):
        for nx_i, wx in zip(nodes, weights):
            sx, sy = sigma_px * nx_i * geom.pixel, sigma_px * ny_i * geom.pixel
            mx = int(np.rint(sx / z * geom.nx * geom.pixel)) if z > 0 else 0
            my = int(np.rint(sy / z * geom.ny * geom.pixel)) if z > 0 else 0
            modes.append((mx, my, wx * wy))
    return modes


def mode_wave(geom: Geometry, mx: int, my: int) -> np.ndarray:
    """s(r) = exp(i 2 pi (mx x / nx + my y / ny)) on the pixel grid."""
    y = np.arange(geom.ny)[:, None]
    x = np.arange(geom.nx)[None, :]
    return np.exp(2j * np.pi * (mx * x / geom.nx + my * y / geom.ny))


def ModalPhysicalModel(psi, t, geom: Geometry, modes):
    """f = sum_j w_j |P2{t P1{x s_j}}|^2; returns f, x and the fields v_j."""
    x = np.exp(psi)
    f = np.zeros(psi.shape)
    vs = []
    for mx, my, w in modes:
        v = FreePropagation(x * mode_wave(geom, mx, my), geom, geom.L1)
        v = FreePropagation(t * v, geom, geom.L2)
        f += w * np.abs(v) ** 2
        vs.append(v)
    return f, x, vs


def ModalWirtingerDerivative(e, x, vs, t, geom: Geometry, modes):
    """g = sum_j w_j conj(x s_j) P1^H{conj(t) P2^H{v_j (-e)}} / max|t|^2."""
    g = np.zeros(x.shape, complex)
    for (mx, my, w), v in zip(modes, vs):
        gj = FreePropagation(v * (-e), geom, -geom.L2)
        gj = FreePropagation(np.conj(t) * gj, geom, -geom.L1)
        g += w * np.conj(x * mode_wave(geom, mx, my)) * gj
    return g / np.max(np.abs(t) ** 2)


def modal_gradient(psi, t, y, geom: Geometry, modes):
    f, x, vs = ModalPhysicalModel(psi, t, geom, modes)
    e = y - f
    return ModalWirtingerDerivative(e, x, vs, t, geom, modes), loss(y, f)


def modal_pwf_iteration(psi, phi, mu, y, t, geom: Geometry, modes, Pinv=None, Gamma2=None):
    """Algorithm S1's loop body with the modal model in place of PhysicalModel /
    WirtingerDerivative (the preconditioner, regularizer and Nesterov steps are
    unchanged; Gamma^2 uses x_coh, y_coh of geom)."""
    if Pinv is None:
        Pinv = precond_filter(geom)
    if Gamma2 is None:
        Gamma2 = reg_window(geom)
    phi_prev, mu_prev = phi, mu
    f, x, vs = ModalPhysicalModel(psi, t, geom, modes)
    e = y - f
    g = ModalWirtingerDerivative(e, x, vs, t, geom, modes)
    g = Preconditioner(g, Pinv) + Regularizer(psi, Gamma2, geom.alpha)
    phi = psi - geom.eta * g
    mu = nesterov_mu(mu)
    psi_new = phi + ((mu_prev - 1.0) / mu) * (phi - phi_prev)
    return psi_new, phi, mu, loss(y, f)


def modal_pwf(y, t, geom: Geometry, modes, max_iter: int, corr_tol=None) -> PWFResult:
    psi = np.zeros((geom.ny, geom.nx), np.complex128)
    phi = np.zeros_like(psi)
    mu = 1.0
    Pinv, Gamma2 = precond_filter(geom), reg_window(geom)
    losses, corrs = [], []
    it = 0
    while it < max_iter:
        x_old = np.exp(psi)
        psi, phi, mu, L = modal_pwf_iteration(psi, phi, mu, y, t, geom, modes, Pinv, Gamma2)
        it += 1
        losses.append(L)
        c = correlation(np.exp(psi), x_old)
        corrs.append(c)
        if corr_tol is not None and c > corr_tol:
            break
    return PWFResult(psi, it, losses, corrs)


def modal_forward_vjp(psi, t, grad_f, geom: Geometry, modes):
    """VJP of the modal f for a real cotangent grad_f, convention dL/dRe + i dL/dIm:
    grad_psi = 2 sum_j w_j conj(x s_j) P1^H{conj(t) P2^H{v_j grad_f}} and
    grad_t   = 2 sum_j w_j conj(P1{x s_j}) P2^H{v_j grad_f} (same derivation as R7)."""
    x = np.exp(psi)
    gp = np.zeros(psi.shape, complex)
    gt = np.zeros(psi.shape, complex)
    for mx, my, w in modes:
        s = mode_wave(geom, mx, my)
        u1 = FreePropagation(x * s, geom, geom.L1)
        v = FreePropagation(t * u1, geom, geom.L2)
        g2 = FreePropagation(v * grad_f, geom, -geom.L2)
        gt += 2.0 * w * np.conj(u1) * g2
        gp += 2.0 * w * np.conj(x * s) * FreePropagation(np.conj(t) * g2, geom, -geom.L1)
    return gp, gt


# ----------------------------------------------------------------------------
# Calibration from the reference speckle (Methods: "Intensity optical transfer
# function (IOTF)" and "Diffuser transmission function")
# ----------------------------------------------------------------------------
# Readings (R14): g2 is the circular, line-averaged autocorrelation normalised
# by the squared mean intensity; the Gaussian model g2 = 1 + A exp(-pi D^2 /
# x_coh^2) is fitted by least squares on ln(g2 - 1) against D^2 over lags
# 1..max_lag (lag 0 carries the shot-noise spike); the Wiener filter is
# IOTF / (IOTF^2 + eps) with eps a noise-to-signal constant the caller picks;
# negative deconvolved intensities are clipped to zero before the square root.
def intensity_autocorrelation(I: np.ndarray, axis: int) -> np.ndarray:
    """g2(D) = <I(r) I(r + D e_axis)> / <I>^2, averaged over all r (circular)."""
    n = I.shape[axis]
    ac = np.fft.ifft(np.abs(np.fft.fft(I, axis=axis)) ** 2, axis=axis).real / n
    return ac.mean(axis=1 - axis) / np.mean(I) ** 2


def fit_coherence_length(g2: np.ndarray, max_lag: int):
    """(x_coh in pixels, A) of g2(D) - 1 = A exp(-pi D^2 / x_coh^2), D = 1..max_lag."""
    lags = np.arange(1, max_lag + 1, dtype=np.float64)
    z = np.log(np.clip(g2[1:max_lag + 1] - 1.0, 1e-300, None))
    slope, intercept = np.polyfit(lags * lags, z, 1)
    return float(np.sqrt(-np.pi / slope)), float(np.exp(intercept))


def calibrate_coherence(I_ref: np.ndarray, pixel: float, max_lag: int):
    """(x_coh, y_coh) in metres from the reference speckle."""
    xc, _ = fit_coherence_length(intensity_autocorrelation(I_ref, 1), max_lag)
    yc, _ = fit_coherence_length(intensity_autocorrelation(I_ref, 0), max_lag)
    return xc * pixel, yc * pixel


def wiener_deconvolve(I: np.ndarray, geom: Geometry, eps: float) -> np.ndarray:
    """Re Filter(I, IOTF / (IOTF^2 + eps))."""
    W = iotf(geom)
    return Filter(I, W / (W * W + eps)).real


def diffuser_from_reference(I_ref: np.ndarray, geom: Geometry, eps: float) -> np.ndarray:
    """t = P(-L2){ sqrt(max(I_coh, 0)) } with I_coh the Wiener-deconvolved
    reference speckle and its phase set to zero at the detector."""
    I_coh = np.clip(wiener_deconvolve(I_ref, geom, eps), 0.0, None)
    return FreePropagation(np.sqrt(I_coh), geom, -geom.L2)
