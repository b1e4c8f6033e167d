"""Pins of the FP64 oracle to facts other than itself (CPU only).

Each test checks the oracle against something the paper or the mathematics
fixes: brute-force DFT sums, the closed-form paraxial Gaussian beam, the
IPSF/IOTF Fourier pair of Eqs. (4)-(5), closed-form filter responses,
unitarity / semigroup / adjointness of the propagator, central finite
differences of the loss of Eq. (2), the stationary point at the true object,
energy conservation, and noise-free recovery.
"""
import json
import math
import os

import numpy as np
import pytest

from oracle import pwf_oracle as O
from paper_2503_20146_gb300 import synth as S

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def geom(ny=16, nx=12, xcoh=0.0, ycoh=0.0, L1=0.1, L2=0.4, eta=1.0, pixel=1e-6,
         wavelength=S.WAVELENGTH_20KEV_M):
    return O.Geometry(ny, nx, pixel, wavelength, L1, L2, xcoh, ycoh, 1.0, 0.1 + 0.01j, eta)


def crandn(rng, shape):
    return rng.standard_normal(shape) + 1j * rng.standard_normal(shape)


def dft_matrix(n, sign):
    j = np.arange(n)
    return np.exp(sign * 2j * np.pi * np.outer(j, j) / n)


# ----------------------------------------------------------------------------
# Fourier-domain filtering against the DFT definition and direct convolution
# ----------------------------------------------------------------------------
@pytest.mark.parametrize("ny,nx", [(16, 16), (12, 12), (12, 16), (9, 8)])
def test_filter_matches_bruteforce_dft(ny, nx):
    rng = np.random.default_rng(0)
    x = crandn(rng, (ny, nx))
    W = rng.standard_normal((ny, nx)) + 0.3j * rng.standard_normal((ny, nx))
    Fy, Fx = dft_matrix(ny, -1), dft_matrix(nx, -1)
    X = Fy @ x @ Fx.T                                  # sum_{r} x_r e^{-2 pi i k.r / N}
    back = dft_matrix(ny, +1) @ (X * W) @ dft_matrix(nx, +1).T / (ny * nx)
    got = O.fourier_filter(x, W)
    assert np.max(np.abs(got - back)) <= 1e-12 * np.max(np.abs(back))


def test_filter_is_circular_convolution():
    rng = np.random.default_rng(1)
    ny, nx = 6, 5
    x = crandn(rng, (ny, nx))
    h = crandn(rng, (ny, nx))
    conv = np.zeros((ny, nx), complex)
    for r in range(ny):
        for c in range(nx):
            for a in range(ny):
                for b in range(nx):
                    conv[r, c] += x[a, b] * h[(r - a) % ny, (c - b) % nx]
    got = O.fourier_filter(x, np.fft.fft2(h))
    assert np.max(np.abs(got - conv)) <= 1e-12 * np.max(np.abs(conv))


# ----------------------------------------------------------------------------
# Free-space propagation (angular spectrum)
# ----------------------------------------------------------------------------
def test_propagation_identity_unitarity_semigroup_adjoint():
    rng = np.random.default_rng(2)
    g = geom(32, 24)
    x, y = crandn(rng, (32, 24)), crandn(rng, (32, 24))
    assert np.max(np.abs(O.propagate(x, g, 0.0) - x)) <= 1e-14 * np.max(np.abs(x))
    px = O.propagate(x, g, 0.3)
    assert abs(np.linalg.norm(px) - np.linalg.norm(x)) <= 1e-13 * np.linalg.norm(x)
    back = O.propagate(px, g, -0.3)
    assert np.max(np.abs(back - x)) <= 1e-13 * np.max(np.abs(x))
    two = O.propagate(O.propagate(x, g, 0.1), g, 0.25)
    one = O.propagate(x, g, 0.35)
    assert np.max(np.abs(two - one)) <= 1e-12 * np.max(np.abs(one))
    lhs = np.vdot(y, O.propagate(x, g, 0.4))
    rhs = np.vdot(O.propagate(y, g, -0.4), x)
    assert abs(lhs - rhs) <= 1e-12 * abs(lhs)


def test_propagation_matches_paraxial_gaussian_beam():
    """exp(-r^2/w0^2) propagated over z equals exp(-r^2/q)/(1 + i z/zR),
    q = w0^2 (1 + i z/zR), zR = pi w0^2 / lambda (paraxial closed form; the
    angular-spectrum correction is ~1e-12 rad here)."""
    n, p, lam, w0, z = 256, 1e-6, S.WAVELENGTH_20KEV_M, 5e-6, 0.4
    g = geom(n, n, pixel=p, wavelength=lam)
    c = (np.arange(n) - n // 2) * p
    c = np.fft.ifftshift(c)
    r2 = c[:, None] ** 2 + c[None, :] ** 2
    zr = math.pi * w0 ** 2 / lam
    q = w0 ** 2 * (1 + 1j * z / zr)
    expect = np.exp(-r2 / q) / (1 + 1j * z / zr)
    got = O.propagate(np.exp(-r2 / w0 ** 2), g, z)
    assert np.max(np.abs(got - expect)) <= 1e-9
    # and the beam really changed (z/zR ~ 0.3)
    assert np.max(np.abs(expect - np.exp(-r2 / w0 ** 2))) > 0.1


def test_piston_reading_matches_literal_transfer_function():
    """Reading R1: dropping exp(i 2 pi L / lambda) leaves |v|^2 unchanged."""
    w = S.WORKLOADS["blob128_coherent"]
    psi, t = S.blob_case(w)
    g = O.Geometry(w.ny, w.nx, w.pixel_m, w.wavelength_m, w.L1_m, w.L2_m)
    v1 = O.fourier_filter(O.fourier_filter(np.exp(psi), O.transfer_function_literal(g, g.L1)) * t,
                  O.transfer_function_literal(g, g.L2))
    f_lit = np.abs(v1) ** 2
    f = O.intensity(psi, t, g)
    # The literal phase 2 pi w L is ~4e10 rad; fp64 keeps it to ~1e-5 rad.
    assert np.linalg.norm(f - f_lit) <= 2e-5 * np.linalg.norm(f)


def test_no_evanescent_bins_and_exact_adjoint_at_workload_geometry():
    """Reading R2: rho^2 < lambda^-2 everywhere, so P(-L) = conj(Q)."""
    for w in S.WORKLOADS.values():
        sizes = [(w.ny, w.nx)] if w.ny else [(n, n) for n in S.MIXED_SIZES]
        for ny, nx in sizes:
            g = O.Geometry(ny, nx, w.pixel_m, w.wavelength_m, w.L1_m, w.L2_m)
            Q = O.transfer_function(g, g.L2)
            assert np.all(np.abs(np.abs(Q) - 1) < 1e-15)
            assert np.max(np.abs(O.transfer_function(g, -g.L2) - np.conj(Q))) < 1e-15


# ----------------------------------------------------------------------------
# IOTF / IPSF (Eqs. (4)-(5)), STF / regularization window (Eqs. (14)-(15))
# ----------------------------------------------------------------------------
def test_iotf_is_fourier_pair_of_ipsf():
    ny, nx, p = 96, 64, 1e-6
    xc, yc = 7.09e-6, 8.0e-6        # IOTF < 3e-9 at Nyquist: no spectral truncation
    g = geom(ny, nx, xcoh=xc, ycoh=yc, pixel=p)
    delta = np.zeros((ny, nx))
    delta[0, 0] = 1.0
    blur = O.fourier_filter(delta, O.iotf(g)).real
    yy = np.fft.fftfreq(ny, 1.0 / ny)[:, None] * p        # signed periodic offsets
    xx = np.fft.fftfreq(nx, 1.0 / nx)[None, :] * p
    ipsf = 2.0 / (xc * yc) * np.exp(-2 * np.pi * (xx ** 2 / xc ** 2 + yy ** 2 / yc ** 2))
    assert np.max(np.abs(blur - ipsf * p * p)) <= 1e-9 * np.max(ipsf * p * p)
    assert abs(np.sum(ipsf) * p * p - 1.0) < 1e-9           # integral of IPSF = 1
    assert O.iotf(g)[0, 0] == 1.0


def test_stf_is_iotf_power_and_window_vanishes_at_dc():
    g = O.Geometry(40, 40, 1e-6, 6.2e-11, 0.1, 0.4, 7e-6, 5e-6, 1.7)
    assert np.allclose(O.stf(g), O.iotf(g) ** (2 * g.gamma), rtol=0, atol=1e-15)
    G2 = O.reg_window(g)
    assert G2[0, 0] == 0.0 and np.all(G2 >= 0) and np.all(G2 <= 1)
    coh = O.Geometry(40, 40, 1e-6, 6.2e-11, 0.1, 0.4)        # reading R4
    assert np.all(O.reg_window(coh) == 0) and np.all(O.iotf(coh) == 1)


# ----------------------------------------------------------------------------
# Preconditioner (Eq. (11)) and regularization window (Eqs. (14)-(15))
# ----------------------------------------------------------------------------
def test_preconditioner_closed_form_on_a_cosine():
    ny, nx, ky, kx = 32, 48, 3, 5
    g = geom(ny, nx)
    yy, xx = np.mgrid[0:ny, 0:nx]
    c = np.cos(2 * np.pi * (ky * yy / ny + kx * xx / nx))
    gin = 0.7 * c + 1j * (c + 2.5)            # Re part untouched, DC of Im dropped
    out = O.precondition(gin, O.precond_filter(g))
    scale = 1.0 / ((ky / ny) ** 2 + (kx / nx) ** 2)    # cycles per pixel (R3)
    assert np.max(np.abs(out.real - 0.7 * c)) < 1e-12
    assert np.max(np.abs(out.imag - scale * c)) < 1e-9 * scale


def test_regularizer_special_cases():
    rng = np.random.default_rng(3)
    psi = crandn(rng, (16, 20))
    ones = np.ones((16, 20))
    assert np.max(np.abs(O.regularization(psi, ones, 1 + 1j) - psi)) < 1e-13
    r = O.regularization(psi, ones, 0.1 + 0.01j)
    assert np.max(np.abs(r - (0.1 * psi.real + 0.01j * psi.imag))) < 1e-13
    g = geom(16, 20, xcoh=7e-6, ycoh=7e-6)
    const = np.full((16, 20), 2.0 - 3.0j)      # DC only: Gamma^2(0) = 0
    assert np.max(np.abs(O.regularization(const, O.reg_window(g), 0.1 + 0.01j))) < 1e-13


# ----------------------------------------------------------------------------
# Forward model invariants (Eq. (1))
# ----------------------------------------------------------------------------
def test_forward_flat_and_energy_conservation():
    rng = np.random.default_rng(4)
    g = geom(32, 32, xcoh=6e-6, ycoh=6e-6)
    t = np.exp(1j * rng.standard_normal((32, 32)))
    f0 = O.intensity(np.zeros((32, 32), complex), t, O.Geometry(32, 32, 1e-6, 6.2e-11, 0.0, 0.0, 6e-6, 6e-6))
    assert np.max(np.abs(f0 - 1.0)) < 1e-13                  # P_0 = I, |t| = 1, IOTF(0) = 1
    psi = 0.2 * crandn(rng, (32, 32))
    f = O.intensity(psi, t, g)
    assert abs(np.sum(f) - np.sum(np.exp(2 * psi.real))) < 1e-11 * np.sum(f)


# ----------------------------------------------------------------------------
# Loss and gradient (Eq. (2); the Wirtinger derivative of Results)
# ----------------------------------------------------------------------------
def _fd_case(seed=5, n=32, coherent=False):
    rng = np.random.default_rng(seed)
    xc = 0.0 if coherent else 5e-6
    g = geom(n, n, xcoh=xc, ycoh=0.8 * xc)
    psi = 0.3 * crandn(rng, (n, n))
    t = 1.3 * np.exp(1j * rng.standard_normal((n, n))) * (1 + 0.2 * rng.standard_normal((n, n)))
    y = rng.uniform(0.5, 1.5, (n, n))
    return rng, g, psi, t, y


@pytest.mark.parametrize("coherent", [False, True])
def test_gradient_matches_central_differences(coherent):
    rng, g, psi, t, y = _fd_case(coherent=coherent)
    G, L = O.loss_gradient_real(psi, t, y, g)
    for _ in range(3):
        d = crandn(rng, psi.shape)
        an = np.sum(G.real * d.real + G.imag * d.imag)
        for eps, tol in ((1e-3, 1e-4), (1e-6, 1e-7)):
            Lp = O.loss(y, O.intensity(psi + eps * d, t, g))
            Lm = O.loss(y, O.intensity(psi - eps * d, t, g))
            assert abs((Lp - Lm) / (2 * eps) - an) <= tol * abs(an)


def test_vjp_matches_central_differences_for_psi_and_diffuser():
    rng, g, psi, t, _ = _fd_case(seed=6)
    gf = rng.standard_normal(psi.shape)
    gp, gt = O.forward_vjp(psi, t, gf, g)
    eps = 1e-6
    for grad, which in ((gp, "psi"), (gt, "t")):
        d = crandn(rng, psi.shape)
        if which == "psi":
            Fp = np.sum(gf * O.intensity(psi + eps * d, t, g))
            Fm = np.sum(gf * O.intensity(psi - eps * d, t, g))
        else:
            Fp = np.sum(gf * O.intensity(psi, t + eps * d, g))
            Fm = np.sum(gf * O.intensity(psi, t - eps * d, g))
        an = np.sum(grad.real * d.real + grad.imag * d.imag)
        assert abs((Fp - Fm) / (2 * eps) - an) <= 1e-7 * abs(an)


def test_truth_is_stationary():
    w = S.WORKLOADS["blob128_coherent"]
    psi, t = S.blob_case(w)
    g = O.Geometry(w.ny, w.nx, w.pixel_m, w.wavelength_m, w.L1_m, w.L2_m, 5e-6, 5e-6)
    y = O.intensity(psi, t, g)
    gr, L = O.wirtinger_gradient(psi, t, y, g)
    assert L < 1e-20 and np.max(np.abs(gr)) < 1e-12


# ----------------------------------------------------------------------------
# The PWF loop (Algorithm S1): Nesterov's step, recovery, stopping rule
# ----------------------------------------------------------------------------
def test_nesterov_sequence_and_first_step():
    mu1 = O.nesterov_mu(1.0)
    assert abs(mu1 - (1 + math.sqrt(5)) / 2) < 1e-15              # golden ratio
    rng, g, psi, t, y = _fd_case(seed=7, n=16)
    g = O.Geometry(**{**g.__dict__, "eta": 0.01})
    zero = np.zeros_like(psi)
    solver = O.PWFSolver(O.SpeckleModel(g, t), g)
    mom = O.Momentum(np.zeros_like(psi))
    psi1, _ = solver.step(zero, y, mom)
    phi1, m1 = mom.phi, mom.mu
    assert np.array_equal(psi1, phi1)                              # (mu_prev - 1) = 0
    gr, _ = O.wirtinger_gradient(zero, t, y, g)
    step = O.precondition(gr, O.precond_filter(g))               # the regularizer of psi = 0 is 0
    assert np.max(np.abs(psi1 + 0.01 * step)) < 1e-15 + 1e-12 * np.max(np.abs(psi1))
    psi2, _ = solver.step(psi1, y, mom)
    phi2, m2 = mom.phi, mom.mu
    beta = (m1 - 1) / m2
    assert abs(beta - ((1 + math.sqrt(5)) / 2 - 1) / O.nesterov_mu(mu1)) < 1e-15
    assert np.max(np.abs(psi2 - (phi2 + beta * (phi2 - phi1)))) < 1e-14


def test_noise_free_recovery_blob128():
    """y = f(psi_true), psi_0 = 0: the loss falls >= 1e3 in 200 iterations and
    the iterate reproduces the data. (It need not equal psi_true: with a
    complex unknown per pixel and one intensity per pixel the forward model is
    not injective here, and this coherent case has no regularizer.)"""
    w = S.WORKLOADS["blob128_coherent"]
    psi_true, t = S.blob_case(w)
    g = O.Geometry(w.ny, w.nx, w.pixel_m, w.wavelength_m, w.L1_m, w.L2_m, eta=2.0 ** -10)
    y = O.intensity(psi_true, t, g)
    r = O.solve(y, t, g, 200)
    assert r.losses[0] / r.losses[-1] > 1e3
    f = O.intensity(r.psi, t, g)
    assert np.linalg.norm(f - y) < 1e-3 * np.linalg.norm(y)
    assert np.linalg.norm(O.intensity(np.zeros_like(psi_true), t, g) - y) > 0.03 * np.linalg.norm(y)


def test_stop_rule_reading():
    assert abs(O.STOP_CORRELATION - 0.99997697) < 1e-8
    x = np.exp(1j * np.linspace(0, 1, 50))
    assert abs(O.correlation(x, x) - 1.0) < 1e-15
    assert abs(O.correlation(3.0 * x, x) - 1.0) < 1e-15             # scale-free


def test_correlation_is_phase_blind_and_matches_a_hand_computed_pair():
    # a global phase rotation leaves the field unchanged up to its phase: the
    # modulus of the inner product (not its real part) makes the correlation 1
    rng = np.random.default_rng(40)
    x = crandn(rng, (8, 6))
    for theta in (0.3, 1.5, math.pi):
        assert abs(O.correlation(x * np.exp(1j * theta), x) - 1.0) < 1e-14
    # x_old = (1, i), x_new = (1, 1): <x_old, x_new> = 1 - i, |.| = sqrt 2, norms sqrt 2 each
    c = O.correlation(np.array([1.0, 1.0]), np.array([1.0, 1j]))
    assert abs(c - math.sqrt(2.0) / 2.0) < 1e-15
    # orthogonal fields correlate to 0; the measure is symmetric
    assert O.correlation(np.array([1.0, 0.0]), np.array([0.0, 1.0])) == 0.0
    y = crandn(rng, (8, 6))
    assert abs(O.correlation(x, y) - O.correlation(y, x)) < 1e-15


# ----------------------------------------------------------------------------
# Printed constants (golden fixture with citations)
# ----------------------------------------------------------------------------
def test_paper_constants_golden():
    with open(os.path.join(GOLDEN, "paper_constants.json")) as fh:
        c = json.load(fh)
    g = O.Geometry(8, 8, 1e-6, 1e-10, 0.0, 0.0)
    assert g.gamma == c["gamma"]["value"]
    assert g.alpha == complex(c["alpha"]["re"], c["alpha"]["im"])
    assert O.STOP_CORRELATION == 10.0 ** c["stop_exponent"]["value"]
    lam_10kev = 1.23984198e-6 / 1.0e4
    assert abs(lam_10kev - c["wavelength_10keV_nm"]["value"] * 1e-9) < 0.001e-9


# ----------------------------------------------------------------------------
# K-mode variant (reading R13)
# ----------------------------------------------------------------------------
def test_gauss_hermite_rules_integrate_normal_moments():
    for k1, exact_to in ((3, 5), (5, 9)):
        x, w = O.gauss_hermite(k1)
        for m in range(exact_to + 1):
            moment = 0.0 if m % 2 else float(np.prod(np.arange(m - 1, 0, -2))) if m else 1.0
            assert abs(np.sum(w * x ** m) - moment) < 1e-12


def test_single_mode_is_the_coherent_model():
    rng = np.random.default_rng(12)
    g = geom(32, 48)
    psi = 0.3 * crandn(rng, (32, 48))
    t = np.exp(1j * rng.standard_normal((32, 48)))
    f1 = O.modal_intensity(psi, t, g, [(0, 0, 1.0)])
    assert np.max(np.abs(f1 - O.intensity(psi, t, g))) < 1e-13


@pytest.mark.parametrize("mx,my", [(3, -2), (-5, 7), (0, 31), (47, 0)])
def test_a_mode_shifts_the_2d_spectrum_by_its_bins(mx, my):
    # DFT shift theorem: F{x s}(kx, ky) = F{x}(kx - mx, ky - my), indices mod (nx, ny);
    # the product with a tilted mode is an index shift of the exit wave's spectrum
    rng = np.random.default_rng(abs(mx) * 100 + abs(my))
    g = geom(32, 48)
    x = crandn(rng, (32, 48))
    lhs = np.fft.fft2(x * O.mode_wave(g, mx, my))
    rhs = np.roll(np.fft.fft2(x), (my, mx), axis=(0, 1))
    assert np.max(np.abs(lhs - rhs)) < 1e-10 * np.max(np.abs(rhs))


def test_tilted_modes_shift_the_field_by_lambda_L2_q():
    """With L1 = 0, a mode tilted by m bins propagates to
    v_m(r) = s_m(r) exp(-i pi lambda L2 |q|^2) v_0(r - lambda L2 q), q = m/(N p)
    (the Fresnel shift theorem; exact on the grid for the paraxial kernel up to
    spectral content that wraps past Nyquist, here on periodic smooth inputs;
    the angular-spectrum correction is ~1e-8 rad)."""
    n = 64
    g = O.Geometry(n, n, 1e-6, S.WAVELENGTH_20KEV_M, 0.0, 0.4)
    rng = S.rng_for(1, 5)
    psi = 0.4j * np.angle(S.diffuser(n, n, rng, corr_px=6.0, std_rad=1.0)) - 0.02
    t = S.diffuser(n, n, rng, corr_px=6.0, std_rad=0.5)
    v0 = O.ModalSpeckleModel(g, t, [(0, 0, 1.0)]).evaluate(psi).v[0]
    V0 = np.fft.fft2(v0)
    kx = np.fft.fftfreq(n)[None, :]
    ky = np.fft.fftfreq(n)[:, None]
    for mx, my in ((3, 0), (-2, 5)):
        vm = O.ModalSpeckleModel(g, t, [(mx, my, 1.0)]).evaluate(psi).v[0]
        qx, qy = mx / (n * g.pixel), my / (n * g.pixel)
        dx, dy = g.wavelength * g.L2 * qx / g.pixel, g.wavelength * g.L2 * qy / g.pixel   # pixels
        shifted = np.fft.ifft2(V0 * np.exp(-2j * np.pi * (kx * dx + ky * dy)))
        expect = O.mode_wave(g, mx, my) * np.exp(-1j * np.pi * g.wavelength * g.L2 * (qx * qx + qy * qy)) * shifted
        assert np.max(np.abs(vm - expect)) < 1e-6 * np.max(np.abs(v0))     # 2-4e-7 seen; a sign error gives > 0.3
        assert np.max(np.abs(np.abs(vm) - np.abs(v0))) > 1e-2 * np.max(np.abs(v0))   # the pattern moved


def test_modal_gradient_matches_central_differences():
    rng = np.random.default_rng(13)
    g = geom(32, 32, xcoh=4e-6, ycoh=4e-6)
    modes = O.source_modes(O.Geometry(32, 32, 1e-6, S.WAVELENGTH_20KEV_M, 0.1, 0.4), 9, 1.5)
    assert len({(mx, my) for mx, my, _ in modes}) == 9
    psi = 0.3 * crandn(rng, (32, 32))
    t = np.exp(1j * rng.standard_normal((32, 32))) * (1 + 0.2 * rng.standard_normal((32, 32)))
    y = rng.uniform(0.5, 1.5, (32, 32))
    gr, L = O.modal_gradient(psi, t, y, g, modes)
    G = 4.0 * np.max(np.abs(t) ** 2) * gr
    for _ in range(2):
        d = crandn(rng, psi.shape)
        an = np.sum(G.real * d.real + G.imag * d.imag)
        eps = 1e-6
        Lp = O.loss(y, O.modal_intensity(psi + eps * d, t, g, modes))
        Lm = O.loss(y, O.modal_intensity(psi - eps * d, t, g, modes))
        assert abs((Lp - Lm) / (2 * eps) - an) <= 1e-7 * abs(an)


def test_modal_vjp_matches_central_differences():
    rng = np.random.default_rng(14)
    g = geom(32, 32)
    modes = O.source_modes(O.Geometry(32, 32, 1e-6, S.WAVELENGTH_20KEV_M, 0.1, 0.4), 9, 1.5)
    psi = 0.3 * crandn(rng, (32, 32))
    t = np.exp(1j * rng.standard_normal((32, 32))) * (1 + 0.2 * rng.standard_normal((32, 32)))
    gf = rng.standard_normal((32, 32))
    gp, gt = O.modal_forward_vjp(psi, t, gf, g, modes)
    eps = 1e-6
    for grad, which in ((gp, "psi"), (gt, "t")):
        d = crandn(rng, psi.shape)
        a = (psi + eps * d, t) if which == "psi" else (psi, t + eps * d)
        b = (psi - eps * d, t) if which == "psi" else (psi, t - eps * d)
        Fp = np.sum(gf * O.modal_intensity(a[0], a[1], g, modes))
        Fm = np.sum(gf * O.modal_intensity(b[0], b[1], g, modes))
        an = np.sum(grad.real * d.real + grad.imag * d.imag)
        assert abs((Fp - Fm) / (2 * eps) - an) <= 1e-7 * abs(an)


def test_without_preconditioner_the_phase_is_underestimated():
    """Fig. S3: without the preconditioner the retrieved phase is much too
    small. Same data, same step size, 60 iterations each."""
    w = S.WORKLOADS["blob128_coherent"]
    psi_true, t = S.blob_case(w)
    g = O.Geometry(w.ny, w.nx, w.pixel_m, w.wavelength_m, w.L1_m, w.L2_m, S.xcoh_from_blur_sigma(2.0),
                   S.xcoh_from_blur_sigma(2.0), eta=2.0 ** -9)
    y = O.intensity(psi_true, t, g)
    with_p = O.solve(y, t, g, 60).psi

    psi = O.solve(y, t, g, 60, Pinv=np.ones((w.ny, w.nx))).psi
    rms = lambda a: float(np.sqrt(np.mean((a.imag - a.imag.mean()) ** 2)))  # noqa: E731
    assert rms(psi) < 0.1 * rms(with_p)
    assert rms(with_p) > 0.2 * rms(psi_true)


# ----------------------------------------------------------------------------
# Calibration (Methods: IOTF from the reference speckle; diffuser)
# ----------------------------------------------------------------------------
def _gaussian_speckle(n, xc_px, seed):
    """Fully developed speckle whose field has the power spectrum
    exp(-2 pi xc^2 u^2): then |g1(D)|^2 = exp(-pi D^2 / xc^2) exactly in the
    ensemble (Siegert: g2 = 1 + |g1|^2)."""
    rng = np.random.default_rng(seed)
    u = np.fft.fftfreq(n)
    A = np.exp(-np.pi * xc_px ** 2 * (u[:, None] ** 2 + u[None, :] ** 2))
    E = np.fft.ifft2(A * np.exp(2j * np.pi * rng.uniform(size=(n, n))))
    return np.abs(E) ** 2


def test_autocorrelation_fit_recovers_the_coherence_length():
    I = _gaussian_speckle(512, 4.0, 3)
    g2x = O.intensity_autocorrelation(I, 1)
    assert abs(g2x[0] - 2.0) < 0.05                      # fully developed: <I^2>/<I>^2 = 2
    # lags 1..3: beyond them g2 - 1 < 0.05 and the +-0.01 baseline fluctuation of
    # one 512^2 realisation dominates the logarithm
    xc, A = O.fit_coherence_length(g2x, 3)
    assert abs(xc - 4.0) < 0.16 and abs(A - 1.0) < 0.1
    xcm, ycm = O.calibrate_coherence(I, 1e-6, 3)
    assert abs(xcm - 4e-6) < 0.16e-6 and abs(ycm - 4e-6) < 0.16e-6
    # brute-force autocorrelation on a small image
    J = _gaussian_speckle(16, 2.0, 4)
    bf = np.array([np.mean(J * np.roll(J, -d, axis=1)) for d in range(16)]) / np.mean(J) ** 2
    assert np.max(np.abs(O.intensity_autocorrelation(J, 1) - bf)) < 1e-12


def test_wiener_inverts_a_noise_free_blur_and_the_diffuser_reproduces_the_reference():
    n = 64
    g = O.Geometry(n, n, 1e-6, S.WAVELENGTH_20KEV_M, 0.1, 0.4, 3e-6, 3.5e-6)
    t_true = S.diffuser(n, n, S.rng_for(1, 6))
    I_coh = np.abs(O.propagate(t_true, g, g.L2)) ** 2     # coherent reference speckle
    I_ref = O.fourier_filter(I_coh, O.iotf(g)).real                     # partial coherence (Eq. (1), no sample)
    assert np.max(np.abs(O.wiener_deconvolve(I_ref, g, 1e-14) - I_coh)) < 1e-8
    t = O.diffuser_from_reference(I_ref, g, 1e-14)
    v = O.propagate(t, g, g.L2)
    assert np.max(np.abs(np.abs(v) ** 2 - I_coh)) < 1e-7         # reproduces the reference
    assert np.max(np.abs(v.imag)) < 1e-7                         # zero phase at the detector


@pytest.mark.parametrize("coherent", [False, True])
def test_diffuser_gradient_matches_central_differences(coherent):
    # dL/dRe t + i dL/dIm t = 4 max|t|^2 g_t (g's normalisation: factor 2 dropped, / max|t|^2)
    rng, g, psi, t, y = _fd_case(seed=21, coherent=coherent)
    gt = 4.0 * np.max(np.abs(t) ** 2) * O.diffuser_gradient(psi, t, y, g)
    for _ in range(3):
        d = crandn(rng, t.shape)
        an = np.sum(gt.real * d.real + gt.imag * d.imag)
        eps = 1e-6
        Lp = O.loss(y, O.intensity(psi, t + eps * d, g))
        Lm = O.loss(y, O.intensity(psi, t - eps * d, g))
        assert abs((Lp - Lm) / (2 * eps) - an) <= 1e-7 * abs(an)


def _joint_case(n=32, B=3):
    w = S.WORKLOADS["blob512_iotf"]
    g = O.Geometry(n, n, w.pixel_m, w.wavelength_m, w.L1_m, w.L2_m, w.xcoh_m, w.ycoh_m, w.gamma, w.alpha, w.eta)
    t = S.diffuser(n, n, S.rng_for(w.config, 99))
    psi_true = np.stack([S.complex_phase_from(S.blob_phase(n, n, S.rng_for(w.config, b))) for b in range(B)])
    f = O.intensity_batch(psi_true, t, g)
    y = np.stack([S.poisson_measurement(f[b], 1e4, S.rng_for(w.config, 50 + b)) for b in range(B)])
    return g, t, y


def test_joint_refinement_with_zero_step_is_algorithm_s1_per_projection():
    g, t, y = _joint_case()
    r = O.joint_solve(y, t, g, 6, 0.0)
    plain = O.solve_batch(y, t, g, 6)
    for b in range(len(y)):
        assert np.max(np.abs(r.psi[b] - plain[b].psi)) < 1e-12
    assert np.array_equal(r.t, t)
    assert abs(r.losses[0] - sum(p.losses[0] for p in plain)) < 1e-9 * r.losses[0]


def test_joint_refinement_lowers_the_loss_from_a_perturbed_diffuser():
    g, t, y = _joint_case(n=48, B=3)
    t0 = t * np.exp(0.3j * np.angle(S.diffuser(48, 48, np.random.default_rng(5))))
    fixed = O.joint_solve(y, t0, g, 25, 0.0)
    joint = O.joint_solve(y, t0, g, 25, 3e-3)
    assert joint.losses[-1] < 0.97 * fixed.losses[-1]
    assert not np.array_equal(joint.t, t0)


def test_linear_pieces_are_adjoint_to_1e_12():
    # <A x, y> = <x, A^H y> for every linear piece of the forward chain: the Fourier windows
    # with the real, even windows (IOTF, P^-1, Gamma^2; self-adjoint), the
    # propagations (adjoint P(-L)), the multiplication by t (adjoint conj(t))
    rng = np.random.default_rng(31)
    g = geom(24, 20, xcoh=6e-6, ycoh=5e-6)
    x, y = crandn(rng, (24, 20)), crandn(rng, (24, 20))
    t = crandn(rng, (24, 20))

    def check(A, AH):
        lhs, rhs = np.vdot(y, A(x)), np.vdot(AH(y), x)
        assert abs(lhs - rhs) <= 1e-12 * max(abs(lhs), 1.0), (lhs, rhs)

    for W in (O.iotf(g), O.precond_filter(g), O.reg_window(g)):
        check(lambda v, W=W: O.fourier_filter(v, W), lambda v, W=W: O.fourier_filter(v, W))
    for L in (g.L1, g.L2):
        check(lambda v, L=L: O.propagate(v, g, L), lambda v, L=L: O.propagate(v, g, -L))
    check(lambda v: t * v, lambda v: np.conj(t) * v)
    # the back-propagation (propagation over -L, conj(t)) is the adjoint of the forward chain
    fwd = lambda v: O.propagate(t * O.propagate(v, g, g.L1), g, g.L2)
    bwd = lambda v: O.propagate(np.conj(t) * O.propagate(v, g, -g.L2), g, -g.L1)
    check(fwd, bwd)
    # the operator objects the forward model is built from carry the same adjoints
    Wc = crandn(rng, (24, 20))
    check(O.FourierMultiplier(Wc), O.FourierMultiplier(Wc).H)
    check(O.Pointwise(t), O.Pointwise(t).H)
    P1 = O.propagator(g, g.L1)
    assert np.max(np.abs(P1.H(x) - O.propagate(x, g, -g.L1))) < 1e-13 * np.max(np.abs(x))


@pytest.mark.parametrize("modal", [False, True])
def test_pullback_is_the_adjoint_of_the_linearised_forward_model(modal):
    # For real df: sum df . (J dpsi) = 2 Re <pullback(df), dpsi>, with J the
    # derivative of f at psi, formed here by forward-mode perturbation of the
    # chain (dx = x dpsi, du1 = P1 dx, dv = P2(t du1) [+ P2(dt u1)],
    # dI = 2 Re(conj(v) dv), df = K dI), independently of the reverse sweep.
    rng = np.random.default_rng(41)
    g = geom(20, 24, xcoh=5e-6, ycoh=4e-6)
    psi = 0.3 * crandn(rng, (20, 24))
    t = np.exp(1j * rng.standard_normal((20, 24))) * (1 + 0.2 * rng.standard_normal((20, 24)))
    df = rng.standard_normal((20, 24))
    dpsi_in, dt_in = crandn(rng, (20, 24)), crandn(rng, (20, 24))
    if modal:
        modes = [(0, 0, 0.5), (2, -1, 0.3), (-3, 4, 0.2)]
        m = O.ModalSpeckleModel(g, t, modes)
    else:
        modes = [(0, 0, 1.0)]
        m = O.SpeckleModel(g, t)
    tr = m.evaluate(psi)
    gp, gt = m.pullback(tr, df)
    x = np.exp(psi)
    Q1, Q2, K = O.transfer_function(g, g.L1), O.transfer_function(g, g.L2), O.iotf(g)
    jp = np.zeros((20, 24))
    jt = np.zeros((20, 24))
    for mx, my, w in modes:
        s = O.mode_wave(g, mx, my)
        u1 = np.fft.ifft2(np.fft.fft2(x * s) * Q1)
        v = np.fft.ifft2(np.fft.fft2(t * u1) * Q2)
        dv_p = np.fft.ifft2(np.fft.fft2(t * np.fft.ifft2(np.fft.fft2(x * s * dpsi_in) * Q1)) * Q2)
        dv_t = np.fft.ifft2(np.fft.fft2(dt_in * u1) * Q2)
        jp += w * 2.0 * np.real(np.conj(v) * dv_p)
        jt += w * 2.0 * np.real(np.conj(v) * dv_t)
    if not modal:
        jp = np.fft.ifft2(np.fft.fft2(jp) * K).real
        jt = np.fft.ifft2(np.fft.fft2(jt) * K).real
    for grad, d, j in ((gp, dpsi_in, jp), (gt, dt_in, jt)):
        lhs = np.sum(df * j)
        rhs = 2.0 * np.real(np.vdot(grad, d))
        assert abs(lhs - rhs) <= 1e-12 * abs(lhs)


# ----------------------------------------------------------------------------
# Source-mode bins and weights (reading R13): the walk-off distribution
# ----------------------------------------------------------------------------
def _walk_off(g, n_modes, sigma_px):
    """(s_x, s_y, w): detector walk-off of every mode in pixels, s = lambda (L1 +
    L2) q / p with q = m / (N p) the tilt of bin m, and the mode weights."""
    modes = O.source_modes(g, n_modes, sigma_px)
    z = g.wavelength * (g.L1 + g.L2)
    sx = np.array([mx / (g.nx * g.pixel) for mx, _, _ in modes]) * z / g.pixel
    sy = np.array([my / (g.ny * g.pixel) for _, my, _ in modes]) * z / g.pixel
    return sx, sy, np.array([w for _, _, w in modes]), modes


@pytest.mark.parametrize("n,n_modes", [(1024, 9), (1024, 25), (512, 9), (2048, 25), (768, 25)])
def test_source_mode_walk_off_has_the_gaussian_moments(n, n_modes):
    """The K tilts and weights discretise a Gaussian source whose walk-off at
    the detector has standard deviation sigma pixels per axis, the axes
    independent: mean 0, second moment sigma^2, fourth moment 3 sigma^4
    (exact for the 3- and 5-point rules), cross moment 0 and
    E[s_x^2 s_y^2] = sigma^4, each within the bound that rounding the tilt to
    whole bins (at most half a bin, Delta / 2 pixels) allows."""
    sigma = 2.0
    g = O.Geometry(n, n, 1e-6, S.WAVELENGTH_20KEV_M, 0.1, 0.4)
    sx, sy, w, modes = _walk_off(g, n_modes, sigma)
    assert len({(mx, my) for mx, my, _ in modes}) == n_modes
    assert all(isinstance(mx, int) and isinstance(my, int) for mx, my, _ in modes)
    delta = g.wavelength * (g.L1 + g.L2) / (n * g.pixel ** 2)        # one bin in pixels
    assert delta < 0.1                                                # fine enough for 4th moments
    h = delta / 2
    smax = np.max(np.abs(sx)) + h
    assert abs(np.sum(w) - 1.0) < 1e-14
    for s in (sx, sy):
        assert abs(np.sum(w * s)) <= h + 1e-12                        # symmetric rule
        assert abs(np.sum(w * s ** 2) - sigma ** 2) <= 2 * smax * h + h * h
        assert abs(np.sum(w * s ** 4) - 3 * sigma ** 4) <= 4 * smax ** 3 * h + 1e-9
    assert abs(np.sum(w * sx * sy)) <= 2 * smax * h
    assert abs(np.sum(w * sx ** 2 * sy ** 2) - sigma ** 4) <= 4 * smax ** 3 * h
    # the marginal of each axis is the 1-D rule: weights of equal s_x sum to the 1-D weights
    nodes, weights = O.gauss_hermite(int(round(math.sqrt(n_modes))))
    for node, wt in zip(nodes, weights):
        sel = np.abs(sx - sigma * node) <= h + 1e-12
        assert abs(np.sum(w[sel]) - wt) < 1e-14


def test_source_modes_degenerate_cases():
    g = O.Geometry(256, 256, 1e-6, S.WAVELENGTH_20KEV_M, 0.1, 0.4)
    assert O.source_modes(g, 1, 2.0) == [(0, 0, 1.0)]                 # one mode: the coherent model
    assert all(mx == 0 and my == 0 for mx, my, _ in O.source_modes(g, 9, 0.0))
    with pytest.raises(ValueError):
        O.source_modes(g, 8, 2.0)
