"""Planted mistakes in the oracle must be caught by its pins (CPU only).

Each case replaces one piece of the FP64 oracle with a plausible wrong
version (a flipped sign, a dropped factor, a transposed operand, wrong units,
a missing conjugate) for the duration of the test, then runs the pins that
should notice. A case passes when at least one of its pins fails.
"""
import numpy as np
import pytest

from oracle import pwf_oracle as O

import test_oracle_pins as pins

_tf = O.transfer_function
_iotf = O.iotf
_pullback = O.SpeckleModel.pullback
_mpullback = O.ModalSpeckleModel.pullback
_reg = O.regularization
_mwave = O.mode_wave
_modes = O.source_modes


def flipped_propagation(geom, L):
    return np.conj(_tf(geom, L))


def propagation_without_2pi(geom, L):
    Q = _tf(geom, L)
    return np.exp(1j * np.angle(Q) / (2 * np.pi))


def iotf_wrong_constant(geom):
    return _iotf(geom) ** 2            # pi instead of pi/2


def pinv_cycles_per_metre(geom):
    u, v = O.frequencies(geom)
    r2 = u * u + v * v
    out = np.zeros_like(r2)
    out[r2 > 0] = 1.0 / r2[r2 > 0]
    return out


def pullback_without_conj_x(self, tr, df):
    dpsi, dt = _pullback(self, tr, df)
    return dpsi * tr.x / np.conj(tr.x), dt        # x dx instead of conj(x) dx


def pullback_forward_instead_of_back(self, tr, df):
    dI = self.K(df).real
    du2 = self.P2(dI * tr.v)                      # P2 where P2^H belongs
    return np.conj(tr.x) * self.P1(self.T.H(du2)), np.conj(tr.u1) * du2


def pullback_without_conj_t(self, tr, df):
    dI = self.K.H(df).real
    du2 = self.P2.H(dI * tr.v)
    return np.conj(tr.x) * self.P1.H(self.T(du2)), np.conj(tr.u1) * du2


def pullback_without_conj_u1(self, tr, df):
    dpsi, dt = _pullback(self, tr, df)
    return dpsi, dt * tr.u1 / np.conj(tr.u1)


def modal_pullback_without_mode_conj(self, tr, df):
    dx = np.zeros(tr.x.shape, complex)
    dt = np.zeros(tr.x.shape, complex)
    for (S, w), u1, v in zip(self.modes, tr.u1, tr.v):
        du2 = self.P2.H(w * df * v)
        dt += np.conj(u1) * du2
        dx += S(self.P1.H(self.T.H(du2)))        # S where S^H belongs
    return np.conj(tr.x) * dx, dt


def filter_unnormalised(x, W):
    return np.fft.ifft2(np.fft.fft2(x) * W) * x.size


def filter_swapped(x, W):
    return np.fft.fft2(np.fft.ifft2(x) * W)


def regularizer_swapped(psi, Gamma2, alpha):
    return _reg(psi, Gamma2, complex(alpha.imag, alpha.real))


def mu_without_sqrt(mu):
    return (1.0 + 1.0 + 4.0 * mu * mu) / 2.0


def mode_wave_conj(geom, mx, my):
    return np.conj(_mwave(geom, mx, my))


def mode_wave_axes_swapped(geom, mx, my):
    y = np.arange(geom.ny)[:, None]
    x = np.arange(geom.nx)[None, :]
    return np.exp(2j * np.pi * (my * x / geom.nx + mx * y / geom.ny))


def modes_with_halved_bins(geom, n_modes, sigma_px):
    return [(int(mx / 2), int(my / 2), w) for mx, my, w in _modes(geom, n_modes, sigma_px)]


def modes_with_uniform_weights(geom, n_modes, sigma_px):
    return [(mx, my, 1.0 / n_modes) for mx, my, _ in _modes(geom, n_modes, sigma_px)]


def modes_with_L2_only(geom, n_modes, sigma_px):
    g = O.Geometry(**{**geom.__dict__, "L1": 0.0})       # walk-off over L2 instead of L1 + L2
    return _modes(g, n_modes, sigma_px)


def correlation_real_part(x_new, x_old):
    num = np.vdot(x_old, x_new).real
    return float(num / np.sqrt(np.vdot(x_new, x_new).real * np.vdot(x_old, x_old).real))


def correlation_unnormalised(x_new, x_old):
    return float(np.abs(np.vdot(x_old, x_new)) / np.vdot(x_old, x_old).real)


_WALK = "test_source_mode_walk_off_has_the_gaussian_moments"
_CORR = ["test_correlation_is_phase_blind_and_matches_a_hand_computed_pair", "test_stop_rule_reading"]

MUTATIONS = [
    (O, "transfer_function", flipped_propagation, ["test_propagation_matches_paraxial_gaussian_beam"]),
    (O, "transfer_function", propagation_without_2pi, ["test_propagation_matches_paraxial_gaussian_beam",
                                                        "test_piston_reading_matches_literal_transfer_function"]),
    (O, "iotf", iotf_wrong_constant, ["test_iotf_is_fourier_pair_of_ipsf"]),
    (O, "precond_filter", pinv_cycles_per_metre, ["test_preconditioner_closed_form_on_a_cosine"]),
    (O.SpeckleModel, "pullback", pullback_without_conj_x, ["test_gradient_matches_central_differences"]),
    (O.SpeckleModel, "pullback", pullback_forward_instead_of_back, ["test_gradient_matches_central_differences"]),
    (O.SpeckleModel, "pullback", pullback_without_conj_t, ["test_gradient_matches_central_differences"]),
    (O.SpeckleModel, "pullback", pullback_without_conj_u1, ["test_diffuser_gradient_matches_central_differences"]),
    (O.ModalSpeckleModel, "pullback", modal_pullback_without_mode_conj,
     ["test_modal_gradient_matches_central_differences"]),
    (O, "fourier_filter", filter_unnormalised, ["test_filter_matches_bruteforce_dft"]),
    (O, "fourier_filter", filter_swapped, ["test_filter_matches_bruteforce_dft"]),
    (O, "regularization", regularizer_swapped, ["test_regularizer_special_cases"]),
    (O, "nesterov_mu", mu_without_sqrt, ["test_nesterov_sequence_and_first_step"]),
    (O, "mode_wave", mode_wave_conj, ["test_tilted_modes_shift_the_field_by_lambda_L2_q"]),
    (O, "mode_wave", mode_wave_conj, ["test_a_mode_shifts_the_2d_spectrum_by_its_bins"]),
    (O, "mode_wave", mode_wave_axes_swapped, ["test_a_mode_shifts_the_2d_spectrum_by_its_bins"]),
    (O, "source_modes", modes_with_halved_bins, [_WALK]),
    (O, "source_modes", modes_with_uniform_weights, [_WALK]),
    (O, "source_modes", modes_with_L2_only, [_WALK]),
    (O, "correlation", correlation_real_part, _CORR),
    (O, "correlation", correlation_unnormalised, _CORR),
]


def _run_pin(name):
    fn = getattr(pins, name)
    if name == "test_filter_matches_bruteforce_dft":
        fn(12, 16)
    elif name == "test_a_mode_shifts_the_2d_spectrum_by_its_bins":
        fn(3, -2)
    elif name == _WALK:
        fn(1024, 9)
        fn(1024, 25)
    elif name in ("test_gradient_matches_central_differences", "test_diffuser_gradient_matches_central_differences"):
        fn(False)
    else:
        fn()


@pytest.mark.parametrize("owner,target,bad,pin_names", MUTATIONS,
                         ids=[f"{t}-{b.__name__}" for _, t, b, _ in MUTATIONS])
def test_planted_mistake_is_caught(monkeypatch, owner, target, bad, pin_names):
    monkeypatch.setattr(owner, target, bad)
    caught = []
    for name in pin_names:
        try:
            _run_pin(name)
        except AssertionError:
            caught.append(name)
    assert caught, f"no pin caught the planted mistake in {target} ({bad.__name__})"
