"""Planted mistakes in the oracle must be caught by its pins (CPU only).

Each case replaces one piece of the FP64 oracle with a plausible wrong
version (a flipped sign, a dropped factor, a transposed operand, wrong units)
for the duration of the test, then runs the pins that should notice. A case
passes when at least one of its pins fails.
"""
import numpy as np
import pytest

from oracle import pwf_oracle as O

import test_oracle_pins as pins

_tf = O.transfer_function
_iotf = O.iotf
_wd = O.WirtingerDerivative
_filter = O.Filter
_reg = O.Regularizer
_pinv = O.precond_filter
_mu = O.nesterov_mu
_mwave = O.mode_wave


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


def wd_without_conj_x(e, x, v, t, geom):
    return _wd(e, np.conj(x), v, t, geom)


def wd_forward_instead_of_back(e, x, v, t, geom):
    g = O.Filter(-e, O.iotf(geom)).real
    g = O.FreePropagation(v * g, geom, geom.L2)
    g = O.FreePropagation(np.conj(t) * g, geom, geom.L1)
    return np.conj(x) * g / np.max(np.abs(t) ** 2)


def wd_without_conj_t(e, x, v, t, geom):
    g = O.Filter(-e, O.iotf(geom)).real
    g = O.FreePropagation(v * g, geom, -geom.L2)
    g = O.FreePropagation(t * g, geom, -geom.L1)
    return np.conj(x) * g / np.max(np.abs(t) ** 2)


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


def diffuser_gradient_without_conj_u1(psi, t, y, geom):
    f, x, v = O.PhysicalModel(psi, t, geom)
    G = O.Filter(-(y - f), O.iotf(geom)).real
    g2 = O.FreePropagation(v * G, geom, -geom.L2)
    return O.FreePropagation(x, geom, geom.L1) * g2 / np.max(np.abs(t) ** 2)


MUTATIONS = [
    ("transfer_function", flipped_propagation, ["test_propagation_matches_paraxial_gaussian_beam"]),
    ("transfer_function", propagation_without_2pi, ["test_propagation_matches_paraxial_gaussian_beam",
                                                     "test_piston_reading_matches_literal_transfer_function"]),
    ("iotf", iotf_wrong_constant, ["test_iotf_is_fourier_pair_of_ipsf"]),
    ("precond_filter", pinv_cycles_per_metre, ["test_preconditioner_closed_form_on_a_cosine"]),
    ("WirtingerDerivative", wd_without_conj_x, ["test_gradient_matches_central_differences"]),
    ("WirtingerDerivative", wd_forward_instead_of_back, ["test_gradient_matches_central_differences"]),
    ("WirtingerDerivative", wd_without_conj_t, ["test_gradient_matches_central_differences"]),
    ("Filter", filter_unnormalised, ["test_filter_matches_bruteforce_dft"]),
    ("Filter", filter_swapped, ["test_filter_matches_bruteforce_dft"]),
    ("Regularizer", regularizer_swapped, ["test_regularizer_special_cases"]),
    ("nesterov_mu", mu_without_sqrt, ["test_nesterov_sequence_and_first_step"]),
    ("mode_wave", mode_wave_conj, ["test_tilted_modes_shift_the_field_by_lambda_L2_q"]),
    ("mode_wave", mode_wave_conj, ["test_a_mode_shifts_the_2d_spectrum_by_its_bins"]),
    ("mode_wave", mode_wave_axes_swapped, ["test_a_mode_shifts_the_2d_spectrum_by_its_bins"]),
    ("diffuser_gradient", diffuser_gradient_without_conj_u1, ["test_diffuser_gradient_matches_central_differences"]),
]


def _run_pin(name):
    fn = getattr(pins, name)
    if name in ("test_filter_matches_bruteforce_dft",):
        fn(12, 16)
    elif name == "test_a_mode_shifts_the_2d_spectrum_by_its_bins":
        fn(3, -2)
    elif name in ("test_gradient_matches_central_differences", "test_diffuser_gradient_matches_central_differences"):
        fn(False)
    else:
        fn()


@pytest.mark.parametrize("target,bad,pin_names", MUTATIONS,
                         ids=[f"{t}-{b.__name__}" for t, b, _ in MUTATIONS])
def test_planted_mistake_is_caught(monkeypatch, target, bad, pin_names):
    monkeypatch.setattr(O, target, bad)
    caught = []
    for name in pin_names:
        try:
            _run_pin(name)
        except AssertionError:
            caught.append(name)
    assert caught, f"no pin caught the planted mistake in {target} ({bad.__name__})"
