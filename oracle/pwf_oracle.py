"""FP64 CPU oracle of preconditioned Wirtinger flow (PWF), arXiv 2503.20146.

TEST INFRASTRUCTURE ONLY. This module is imported by ``tests/``, by
``__graft_entry__.smoke()`` and by the CPU-baseline / reference leg of
``bench.py``. The CUDA library never calls it, links it or imports it, and it
shares no code with the CUDA path: only the seeded input generators of
``paper_2503_20146_gb300.synth`` serve both.

How it is organised (every array complex128 / float64; numpy's FFT is the one
library primitive):

* The forward model of Eq. (1) is a chain of linear operators and one
  point-wise nonlinearity,

      psi --exp--> x --P(L1)--> u1 --(t .)--> u2 --P(L2)--> v --|.|^2--> I --K--> f,

  with P(L) the angular-spectrum propagator and K the IPSF convolution, both
  Fourier multipliers on the periodic grid (transfer function Q of the
  propagation; IOTF of Eq. (5)), and (t .) the diffuser. Each linear operator
  knows its adjoint.
* The loss is Eq. (2). Its gradient is the reverse sweep through the same
  chain (the Wirtinger calculus of Results, "Preconditioned Wirtinger flow"):
  for a real functional l of f, dl/dconj(psi) = conj(x) P1^H{conj(t) P2^H{v K^H{dl/df}}}.
  The search direction g the paper iterates with is that derivative for
  l = Eq. (2) with the factor 2 dropped (Methods, "Preconditioning filter")
  and divided by max|t|^2.
* The preconditioner of Eq. (11) acts on Im g, the regularization window of
  Eqs. (14)-(15) on psi; Nesterov's accelerated step (Results; Algorithm S1)
  is a separate state update. The stopping rule is the field correlation of
  Methods, "Reconstruction procedure".
* The K-mode source variant (a workload option, reading R13) is a second
  forward model with the same evaluate / pull-back interface, so the solver
  loop is shared.

Readings where the paper is silent or ambiguous (R1 onwards, the numbering the design notes use):
  R1  The transfer function Q = exp(i 2 pi w L) carries the constant piston
      exp(i 2 pi L / lambda). It is a global phase that cancels in |v|^2 and in
      the back-propagation, so it is dropped, and w - 1/lambda is evaluated in
      the cancellation-free form -rho^2 / (1/lambda + w).
  R2  Bins with rho^2 > lambda^-2 (evanescent) get Q = 0. None occur at the
      geometries used here, so the back-propagation P(-L) = conj(Q) is the
      exact adjoint.
  R3  Frequencies u, v are numpy fftfreq in cycles per metre for Q, IOTF and
      STF (they multiply lengths in metres). For the preconditioner P^-1 =
      1/(u^2 + v^2) the units are not stated; it is evaluated in cycles per
      PIXEL, so P^-1 ranges over [2, N^2]. The overall scale is the step size's.
  R4  x_coh = y_coh = 0 means a fully coherent beam: IOTF = 1, STF = 1 and the
      regularization window Gamma^2 = 0 (the regularizer vanishes).
  R5  Filtering a real field (the intensity, the residual, Im g) keeps the
      real part of the inverse transform.
  R6  The stopping test compares the object fields x = exp(psi) of successive
      iterations by |<x_k, x_{k-1}>| / (||x_k|| ||x_{k-1}||); the threshold is
      10^(-0.00001) (Methods, "Reconstruction procedure").
  R7  The gradient w.r.t. the diffuser (simultaneous retrieval, Methods and
      Fig. S12) is not printed; it is the t-branch of the same reverse sweep.
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
      update rule is not printed. Reading: after each PWF iteration over the
      whole series, t <- t - eta_t sum_b g_t,b, a plain gradient step (no
      preconditioner, no momentum) with g_t the t-branch of the reverse sweep
      in the same normalisation as g (factor 2 dropped, divided by max|t|^2
      of the current t), evaluated at the same point as the sample gradient.
      Fixed iteration count (no stopping rule).
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

STOP_CORRELATION = 10.0 ** (-0.00001)


@dataclass(frozen=True)
class Geometry:
    """Problem constants: grid, pixel pitch, wavelength, the two distances and
    the solver parameters gamma, alpha, eta (Results, "Preconditioned Wirtinger
    flow"). Lengths in metres. ``xcoh``/``ycoh`` are the coherence lengths of
    Eqs. (4), (5) and (14); zero means fully coherent (reading R4)."""
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
# Spatial frequencies and the Fourier-domain windows
# ----------------------------------------------------------------------------
def frequencies(geom: Geometry):
    """(u, v) grids in cycles/m, u along x (columns), v along y (rows)."""
    u = np.fft.fftfreq(geom.nx, d=geom.pixel)[None, :]
    v = np.fft.fftfreq(geom.ny, d=geom.pixel)[:, None]
    return u, v


def transfer_function(geom: Geometry, L: float) -> np.ndarray:
    """Angular-spectrum transfer function over distance L, piston removed (R1).

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
    """Q = exp(i 2 pi w L) with the piston kept (for the R1 pin)."""
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
# Linear operators on the periodic grid
# ----------------------------------------------------------------------------
def fourier_filter(x: np.ndarray, W: np.ndarray) -> np.ndarray:
    """F^-1{ W F{x} }: multiplication by W on the 2-D DFT spectrum (circular,
    no padding), the way every Fourier-domain window of the paper is applied."""
    return np.fft.ifft2(np.fft.fft2(x) * W)


class FourierMultiplier:
    """x -> F^-1{W F{x}}; its adjoint multiplies by conj(W) (the DFT is
    unitary up to the 1/N factor that the pair F, F^-1 cancels)."""

    def __init__(self, W: np.ndarray):
        self.W = W

    def __call__(self, x):
        return fourier_filter(x, self.W)

    def H(self, x):
        return fourier_filter(x, np.conj(self.W))


class Pointwise:
    """x -> m x; its adjoint multiplies by conj(m)."""

    def __init__(self, m: np.ndarray):
        self.m = m

    def __call__(self, x):
        return self.m * x

    def H(self, x):
        return np.conj(self.m) * x


def propagator(geom: Geometry, L: float) -> FourierMultiplier:
    """Free-space propagation over L by the angular-spectrum method (Results,
    "Preconditioned Wirtinger flow"): the Fourier multiplier Q of
    ``transfer_function``. Its adjoint is propagation over -L (R2)."""
    return FourierMultiplier(transfer_function(geom, L))


def propagate(x: np.ndarray, geom: Geometry, L: float) -> np.ndarray:
    """x propagated over distance L (negative L: back-propagation)."""
    return propagator(geom, L)(x)


# ----------------------------------------------------------------------------
# Forward model, Eq. (1), and its reverse sweep
# ----------------------------------------------------------------------------
@dataclass
class Trace:
    """Intermediate fields of one evaluation of the forward chain."""
    x: np.ndarray          # e^psi
    u1: np.ndarray         # P1{x}, the field arriving at the diffuser
    v: np.ndarray          # P2{t u1}, the detector field
    f: np.ndarray          # modelled intensity


class SpeckleModel:
    """f(psi) = |P2{t P1{e^psi}}|^2 * IPSF, Eq. (1), for one diffuser t."""

    def __init__(self, geom: Geometry, t: np.ndarray):
        self.geom = geom
        self.P1 = propagator(geom, geom.L1)
        self.P2 = propagator(geom, geom.L2)
        self.T = Pointwise(t)
        self.K = FourierMultiplier(iotf(geom))
        self.maxt2 = float(np.max(np.abs(t) ** 2))

    def evaluate(self, psi: np.ndarray) -> Trace:
        x = np.exp(psi)
        u1 = self.P1(x)
        v = self.P2(self.T(u1))
        f = self.K(np.abs(v) ** 2).real             # R5
        return Trace(x, u1, v, f)

    def pullback(self, tr: Trace, df: np.ndarray):
        """(dl/dconj(psi), dl/dconj(t)) for a real functional l of f with
        dl/df = df, by the reverse sweep of the chain: I = v conj(v) gives
        dl/dconj(v) = (dl/dI) v; the linear maps pass their adjoints; x = e^psi
        is holomorphic, so dl/dconj(psi) = conj(x) dl/dconj(x)."""
        dI = self.K.H(df).real                      # R5
        dv = dI * tr.v
        du2 = self.P2.H(dv)
        dt = np.conj(tr.u1) * du2
        dx = self.P1.H(self.T.H(du2))
        return np.conj(tr.x) * dx, dt


def intensity(psi, t, geom: Geometry) -> np.ndarray:
    """The modelled intensity f(psi) of Eq. (1)."""
    return SpeckleModel(geom, t).evaluate(psi).f


def loss(y: np.ndarray, f: np.ndarray) -> float:
    """Sum_r (y_r - f_r)^2, Eq. (2)."""
    return float(np.sum((y - f) ** 2))


def search_direction(model, tr: Trace, y: np.ndarray) -> np.ndarray:
    """g: dL/dconj(psi) of Eq. (2) with the factor 2 dropped (Methods,
    "Preconditioning filter") and divided by max|t|^2. Since dL/df = -2 e,
    e = y - f, this is pullback(-2 e) / (2 max|t|^2)."""
    dpsi, _ = model.pullback(tr, -2.0 * (y - tr.f))
    return dpsi / (2.0 * model.maxt2)


def wirtinger_gradient(psi, t, y, geom: Geometry):
    """(g, loss) at psi: the search direction above and Eq. (2)."""
    m = SpeckleModel(geom, t)
    tr = m.evaluate(psi)
    return search_direction(m, tr, y), loss(y, tr.f)


def loss_gradient_real(psi, t, y, geom: Geometry):
    """dL/dRe(psi) + i dL/dIm(psi) of Eq. (2) = 2 dL/dconj(psi) = 4 max|t|^2 g."""
    g, L = wirtinger_gradient(psi, t, y, geom)
    return 4.0 * np.max(np.abs(t) ** 2) * g, L


def forward_vjp(psi, t, grad_f, geom: Geometry):
    """Vector-Jacobian product of f for a real cotangent grad_f, in the
    convention dl/dRe + i dl/dIm = 2 dl/dconj: (grad_psi, grad_t)."""
    m = SpeckleModel(geom, t)
    dpsi, dt = m.pullback(m.evaluate(psi), grad_f)
    return 2.0 * dpsi, 2.0 * dt


def diffuser_gradient(psi, t, y, geom: Geometry):
    """g_t: the t-branch of the sweep for Eq. (2) in g's normalisation (R16),
    so that dL/dRe t + i dL/dIm t = 4 max|t|^2 g_t."""
    m = SpeckleModel(geom, t)
    tr = m.evaluate(psi)
    _, dt = m.pullback(tr, -2.0 * (y - tr.f))
    return dt / (2.0 * m.maxt2)


# ----------------------------------------------------------------------------
# Preconditioner, regularizer, momentum, stopping rule
# ----------------------------------------------------------------------------
def precondition(g: np.ndarray, Pinv: np.ndarray) -> np.ndarray:
    """Eq. (11): the inverse-Laplacian filter applied to the phase part Im g;
    the attenuation part Re g is left as it is."""
    return g.real + 1j * fourier_filter(g.imag, Pinv).real      # R5


def regularization(psi: np.ndarray, Gamma2: np.ndarray, alpha: complex) -> np.ndarray:
    """The regularizer's contribution to the direction: psi filtered by the
    window Gamma^2 of Eq. (15), with Re(alpha) weighting the attenuation and
    Im(alpha) the phase separately (Results, "Preconditioned Wirtinger flow")."""
    rho = fourier_filter(psi, Gamma2)
    return alpha.real * rho.real + 1j * alpha.imag * rho.imag


def nesterov_mu(mu: float) -> float:
    """Nesterov's sequence mu <- (1 + sqrt(1 + 4 mu^2)) / 2, from mu = 1."""
    return (1.0 + np.sqrt(1.0 + 4.0 * mu * mu)) / 2.0


@dataclass
class Momentum:
    """State of Nesterov's accelerated step: the previous plain step phi and mu."""
    phi: np.ndarray
    mu: float = 1.0

    def advance(self, psi: np.ndarray, direction: np.ndarray, eta: float) -> np.ndarray:
        """phi' = psi - eta d; psi' = phi' + ((mu - 1)/mu') (phi' - phi)."""
        phi_new = psi - eta * direction
        mu_new = nesterov_mu(self.mu)
        psi_new = phi_new + ((self.mu - 1.0) / mu_new) * (phi_new - self.phi)
        self.phi, self.mu = phi_new, mu_new
        return psi_new


def correlation(x_new: np.ndarray, x_old: np.ndarray) -> float:
    """Normalised correlation of successive fields (reading R6)."""
    num = np.abs(np.vdot(x_old, x_new))
    den = np.sqrt(np.vdot(x_new, x_new).real * np.vdot(x_old, x_old).real)
    return float(num / den)


# ----------------------------------------------------------------------------
# The PWF solver
# ----------------------------------------------------------------------------
@dataclass
class PWFResult:
    psi: np.ndarray
    iterations: int
    losses: list = field(default_factory=list)        # loss of the model at the start of each iteration
    correlations: list = field(default_factory=list)  # correlation after each iteration


class PWFSolver:
    """Preconditioned Wirtinger flow on one projection: a forward model with
    the evaluate / pullback interface, the two windows and the step size.
    ``Pinv`` may be overridden (all ones: no preconditioner, Fig. S3)."""

    def __init__(self, model, geom: Geometry, Pinv=None, Gamma2=None):
        self.model = model
        self.geom = geom
        self.Pinv = precond_filter(geom) if Pinv is None else Pinv
        self.Gamma2 = reg_window(geom) if Gamma2 is None else Gamma2

    def direction(self, psi, y):
        """(total direction, loss at psi): precondition(g) + regularization(psi)."""
        tr = self.model.evaluate(psi)
        g = search_direction(self.model, tr, y)
        d = precondition(g, self.Pinv) + regularization(psi, self.Gamma2, self.geom.alpha)
        return d, loss(y, tr.f)

    def step(self, psi, y, mom: Momentum):
        """One iteration from psi: (new psi, loss at psi)."""
        d, L = self.direction(psi, y)
        return mom.advance(psi, d, self.geom.eta), L

    def solve(self, y, max_iter: int, corr_tol=None, psi0=None) -> PWFResult:
        """From psi = 0 (or psi0) for max_iter iterations, stopping earlier once
        the correlation of successive fields exceeds corr_tol (None: never)."""
        g = self.geom
        psi = np.zeros((g.ny, g.nx), np.complex128) if psi0 is None else psi0.astype(np.complex128)
        mom = Momentum(np.zeros_like(psi))
        res = PWFResult(psi, 0)
        while res.iterations < max_iter:
            x_old = np.exp(psi)
            psi, L = self.step(psi, y, mom)
            res.iterations += 1
            res.losses.append(L)
            c = correlation(np.exp(psi), x_old)
            res.correlations.append(c)
            if corr_tol is not None and c > corr_tol:
                break
        res.psi = psi
        return res


def solve(y: np.ndarray, t: np.ndarray, geom: Geometry, max_iter: int,
          corr_tol: float | None = None, psi0: np.ndarray | None = None, Pinv=None) -> PWFResult:
    """PWF with the paper's forward model (Eq. (1))."""
    return PWFSolver(SpeckleModel(geom, t), geom, Pinv=Pinv).solve(y, max_iter, corr_tol, psi0)


@dataclass
class JointResult:
    psi: np.ndarray       # [B][ny][nx]
    t: np.ndarray         # refined diffuser
    losses: list          # total loss of the series at the start of each iteration


def joint_solve(y_b, t0, geom: Geometry, max_iter: int, eta_t: float) -> JointResult:
    """PWF over a series of projections that share the diffuser, with t refined
    after every iteration (reading R16). The Nesterov sequence mu is common to
    the series (every projection takes the same number of steps)."""
    B = len(y_b)
    psi = np.zeros((B, geom.ny, geom.nx), np.complex128)
    moms = [Momentum(np.zeros((geom.ny, geom.nx), np.complex128)) for _ in range(B)]
    t = np.asarray(t0, np.complex128).copy()
    Pinv, Gamma2 = precond_filter(geom), reg_window(geom)
    losses = []
    for _ in range(max_iter):
        solver = PWFSolver(SpeckleModel(geom, t), geom, Pinv, Gamma2)
        gt = np.zeros_like(t)
        total = 0.0
        for b in range(B):
            gt = gt + diffuser_gradient(psi[b], t, y_b[b], geom)
            psi[b], L = solver.step(psi[b], y_b[b], moms[b])
            total += L
        t = t - eta_t * gt
        losses.append(total)
    return JointResult(psi, t, losses)


# ----------------------------------------------------------------------------
# Batched helpers (independent projections, shared diffuser)
# ----------------------------------------------------------------------------
def intensity_batch(psi_b, t, geom: Geometry) -> np.ndarray:
    m = SpeckleModel(geom, t)
    return np.stack([m.evaluate(p).f for p in psi_b])


def gradient_batch(psi_b, t, y_b, geom: Geometry):
    gs, Ls = zip(*[wirtinger_gradient(p, t, y, geom) for p, y in zip(psi_b, y_b)])
    return np.stack(gs), np.array(Ls)


def forward_vjp_batch(psi_b, t, grad_f_b, geom: Geometry):
    """grad_t is summed over the batch: the diffuser is shared."""
    gp, gt = zip(*[forward_vjp(p, t, gf, geom) for p, gf in zip(psi_b, grad_f_b)])
    return np.stack(gp), np.sum(np.stack(gt), axis=0)


def solve_batch(y_b, t, geom: Geometry, max_iter: int, corr_tol=None):
    return [solve(y, t, geom, max_iter, corr_tol) for y in y_b]


# ----------------------------------------------------------------------------
# K-mode partial-coherence variant (a workload option, not the paper's form)
# ----------------------------------------------------------------------------
# The paper models partial coherence by the IPSF convolution of Eq. (1). The
# variant sums the intensities of K mutually incoherent source modes instead:
# tilted plane waves s_j(r) = exp(i 2 pi q_j . r) with weights w_j,
#   f = sum_j w_j |P2{ t P1{ x s_j } }|^2,
# the tilts on a tensor Gauss-Hermite grid of a Gaussian source whose walk-off
# over L1 + L2 has standard deviation sigma pixels at the detector (reading
# R13). Tilts are rounded to whole frequency bins so that s_j is periodic on
# the grid. The reverse sweep runs per mode and sums.
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


@dataclass
class ModalTrace:
    x: np.ndarray
    u1: list               # P1{x s_j} per mode
    v: list                # detector field per mode
    f: np.ndarray


class ModalSpeckleModel:
    """f = sum_j w_j |P2{t P1{x s_j}}|^2 (reading R13), same interface as
    SpeckleModel."""

    def __init__(self, geom: Geometry, t: np.ndarray, modes):
        self.geom = geom
        self.P1 = propagator(geom, geom.L1)
        self.P2 = propagator(geom, geom.L2)
        self.T = Pointwise(t)
        self.modes = [(Pointwise(mode_wave(geom, mx, my)), w) for mx, my, w in modes]
        self.maxt2 = float(np.max(np.abs(t) ** 2))

    def evaluate(self, psi) -> ModalTrace:
        x = np.exp(psi)
        f = np.zeros(psi.shape)
        u1s, vs = [], []
        for S, w in self.modes:
            u1 = self.P1(S(x))
            v = self.P2(self.T(u1))
            f += w * np.abs(v) ** 2
            u1s.append(u1)
            vs.append(v)
        return ModalTrace(x, u1s, vs, f)

    def pullback(self, tr: ModalTrace, df):
        dx = np.zeros(tr.x.shape, complex)
        dt = np.zeros(tr.x.shape, complex)
        for (S, w), u1, v in zip(self.modes, tr.u1, tr.v):
            du2 = self.P2.H(w * df * v)
            dt += np.conj(u1) * du2
            dx += S.H(self.P1.H(self.T.H(du2)))
        return np.conj(tr.x) * dx, dt


def modal_intensity(psi, t, geom: Geometry, modes) -> np.ndarray:
    return ModalSpeckleModel(geom, t, modes).evaluate(psi).f


def modal_gradient(psi, t, y, geom: Geometry, modes):
    """(g, loss) of the modal model in g's normalisation."""
    m = ModalSpeckleModel(geom, t, modes)
    tr = m.evaluate(psi)
    return search_direction(m, tr, y), loss(y, tr.f)


def modal_solve(y, t, geom: Geometry, modes, max_iter: int, corr_tol=None) -> PWFResult:
    """PWF with the modal forward model (the preconditioner, regularizer and
    momentum are unchanged; Gamma^2 uses x_coh, y_coh of geom)."""
    return PWFSolver(ModalSpeckleModel(geom, t, modes), geom).solve(y, max_iter, corr_tol)


def modal_forward_vjp(psi, t, grad_f, geom: Geometry, modes):
    """VJP of the modal f for a real cotangent, convention dl/dRe + i dl/dIm."""
    m = ModalSpeckleModel(geom, t, modes)
    dpsi, dt = m.pullback(m.evaluate(psi), grad_f)
    return 2.0 * dpsi, 2.0 * dt


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
    """Re F^-1{ IOTF / (IOTF^2 + eps) F{I} }."""
    W = iotf(geom)
    return fourier_filter(I, W / (W * W + eps)).real


def diffuser_from_reference(I_ref: np.ndarray, geom: Geometry, eps: float) -> np.ndarray:
    """t = P(-L2){ sqrt(max(I_coh, 0)) } with I_coh the Wiener-deconvolved
    reference speckle and its phase set to zero at the detector."""
    I_coh = np.clip(wiener_deconvolve(I_ref, geom, eps), 0.0, None)
    return propagate(np.sqrt(I_coh), geom, -geom.L2)
