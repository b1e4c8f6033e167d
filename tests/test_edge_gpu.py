"""Degenerate and limit cases on the CUDA path: zero iterations leave the
state untouched, a single projection angle in FBP, and the largest supported
grid (2048 x 2048) against the FP64 oracle."""
import math

import numpy as np
import pytest

from oracle import fbp_oracle as F
from oracle import pwf_oracle as O
from paper_2503_20146_gb300 import synth as S

from _cases import blob_batch, geometry, rel_l2, to_c64, to_f32

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

W2 = S.WORKLOADS["blob512_iotf"]


@pytest.fixture(scope="module")
def pwf():
    from paper_2503_20146_gb300 import _build
    _build.build()
    from paper_2503_20146_gb300 import pwf as P
    P.load()
    return P


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def plan_for(P, g, batch):
    return P.Plan(P.PlanDesc(batch, g.ny, g.nx, g.pixel, g.wavelength, g.L1, g.L2, g.xcoh, g.ycoh, g.gamma,
                             g.alpha.real, g.alpha.imag, g.eta))


def test_zero_iterations_change_nothing(pwf):
    g = geometry(W2, 128, 96)
    psi0, t = blob_batch(W2, 2, 128, 96)
    y = dev(to_f32(np.ones((2, 128, 96))))
    with plan_for(pwf, g, 2) as plan:
        psi = dev(to_c64(psi0))
        td = dev(to_c64(t))
        before_psi, before_t = psi.clone(), td.clone()
        it, _ = plan.solve(y, td, psi, 0)
        assert list(it) == [0, 0]
        plan.solve_joint(y, td, psi, 0, 1e-3)
        torch.cuda.synchronize()
        assert torch.equal(psi, before_psi) and torch.equal(td, before_t)


def test_fbp_single_angle_matches_oracle(pwf):
    rng = np.random.default_rng(11)
    psi = (rng.standard_normal((1, 2, 64)) + 1j * rng.standard_normal((1, 2, 64))).astype(np.complex64)
    angles = np.array([0.3])
    vol = pwf.pwf_fbp(dev(psi), angles, S.WAVELENGTH_20KEV_M, S.PIXEL_M).cpu().numpy()
    ref = F.fbp_volume(psi.astype(np.complex128), angles, S.WAVELENGTH_20KEV_M, S.PIXEL_M)
    assert rel_l2(vol, ref) < max(1e-5, 64 * 2.0 ** -22)


def test_largest_grid_forward_and_gradient_match_oracle(pwf):
    n = 2048
    g = geometry(W2, n, n)
    psi, t = blob_batch(W2, 1, n, n)
    psi, t = to_c64(psi), to_c64(t)
    y = to_f32(np.clip(1.0 + 0.1 * np.random.default_rng(2).standard_normal((1, n, n)), 0, None))
    with plan_for(pwf, g, 1) as plan:
        f = plan.forward(dev(psi), dev(t)).cpu().numpy()[0]
        gr, _ = plan.gradient(dev(psi), dev(t), dev(y))
        gr = gr.cpu().numpy()[0]
    P64, T64 = psi[0].astype(np.complex128), t.astype(np.complex128)
    assert rel_l2(f, O.intensity(P64, T64, g)) <= 1e-5
    assert rel_l2(gr, O.wirtinger_gradient(P64, T64, y[0].astype(np.float64), g)[0]) <= 1e-4


def test_large_phase_and_strong_attenuation_match_oracle(pwf):
    # phases wrapped many times over (|Im psi| up to ~400 rad) and log-amplitudes
    # from about -4 to 1: the complex exponential's phase reduction and modulus
    n = 256
    g = geometry(W2, n, n)
    psi, t = blob_batch(W2, 2, n, n)
    yy, xx = np.mgrid[0:n, 0:n] / n
    psi = (30.0 * psi.real - 2.0) + 1j * (psi.imag + 2.0 * np.pi * (40.0 * xx + 23.0 * yy))
    psi[1] = np.conj(psi[1])
    psi, t = to_c64(psi), to_c64(t)
    assert np.abs(psi.imag).max() > 350 and psi.real.min() < -3
    y = to_f32(np.clip(1.0 + 0.1 * np.random.default_rng(4).standard_normal((2, n, n)), 0, None))
    with plan_for(pwf, g, 2) as plan:
        f = plan.forward(dev(psi), dev(t)).cpu().numpy()
        gr, _ = plan.gradient(dev(psi), dev(t), dev(y))
        gr = gr.cpu().numpy()
    T64 = t.astype(np.complex128)
    for b in range(2):
        P64 = psi[b].astype(np.complex128)
        assert rel_l2(f[b], O.intensity(P64, T64, g)) <= 1e-5
        assert rel_l2(gr[b], O.wirtinger_gradient(P64, T64, y[b].astype(np.float64), g)[0]) <= 1e-4


def test_misaligned_device_arrays_are_rejected_before_any_work(pwf):
    g = geometry(W2, 64, 64)
    _, t = blob_batch(W2, 1, 64, 64)
    n = 64 * 64
    with plan_for(pwf, g, 1) as plan:
        td = dev(to_c64(t))
        psi_bad = torch.zeros(n + 1, dtype=torch.complex64, device="cuda")[1:].view(1, 64, 64)  # 8 B off
        y = torch.ones((1, 64, 64), dtype=torch.float32, device="cuda")
        with pytest.raises(pwf.PWFError):
            plan.forward(psi_bad, td)
        with pytest.raises(pwf.PWFError):
            plan.solve(y, td, psi_bad, 2)
        y_bad = torch.ones(n + 1, dtype=torch.float32, device="cuda")[1:].view(1, 64, 64)  # 4 B off
        psi = torch.zeros((1, 64, 64), dtype=torch.complex64, device="cuda")
        with pytest.raises(pwf.PWFError):
            plan.gradient(psi, td, y_bad)
        # nothing was queued: the plan still solves
        it, _ = plan.solve(y, td, psi, 2)
        assert list(it) == [2]


# ---------------------------------------------------------------------------
# debug aids: the non-finite scan and the allocation-failure hook
# ---------------------------------------------------------------------------
def _flagged_plan(P, g, batch, flags):
    return P.Plan(P.PlanDesc(batch, g.ny, g.nx, g.pixel, g.wavelength, g.L1, g.L2, g.xcoh, g.ycoh, g.gamma,
                             g.alpha.real, g.alpha.imag, g.eta, flags))


@pytest.mark.parametrize("where,first", [("t", "row_mul_t"), ("psi", "row_exp_fft")])
def test_check_finite_names_the_first_pass_with_bad_output(pwf, where, first):
    # one NaN pixel in the diffuser first shows in the output of the diffuser
    # multiply; one in the starting iterate, in exp(psi) of the first pass
    g = geometry(W2, 128, 128)
    psi0, t = blob_batch(W2, 1, 128, 128)
    psi0, t = to_c64(psi0).copy(), to_c64(t).copy()
    if where == "t":
        t[40, 17] = np.nan
    else:
        psi0[0, 40, 17] = np.nan
    y = dev(to_f32(np.ones((1, 128, 128))))
    with _flagged_plan(pwf, g, 1, pwf.FLAG_CHECK_FINITE) as plan:
        with pytest.raises(pwf.PWFError) as e:
            plan.solve(y, dev(t), dev(psi0), 2)
        assert e.value.status == 5 and f"pass {first}" in str(e.value)
    with _flagged_plan(pwf, g, 1, 0) as plan:      # without the scan: only that something went non-finite
        with pytest.raises(pwf.PWFError) as e:
            plan.solve(y, dev(t), dev(psi0), 2)
        assert e.value.status == 5 and "pass" not in str(e.value)


def test_check_finite_passes_clean_input_bitwise(pwf):
    g = geometry(W2, 128, 128)
    psi0, t = blob_batch(W2, 1, 128, 128)
    y = dev(to_f32(np.ones((1, 128, 128))))
    out = []
    for flags in (pwf.FLAG_CHECK_FINITE, pwf.FLAG_GRAPH):   # both graphs on the untuned column shapes
        with _flagged_plan(pwf, g, 1, flags | pwf.FLAG_NO_TUNE) as plan:
            psi = torch.zeros((1, 128, 128), dtype=torch.complex64, device="cuda")
            plan.solve(y, dev(to_c64(t)), psi, 4)
            out.append(psi.cpu())
    assert torch.equal(out[0], out[1])


def test_failed_allocation_returns_nomem_and_frees_the_rest(pwf):
    g = geometry(W2, 256, 256)
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    for k in (0, 3, 9):
        pwf.pwf_debug_fail_alloc(k)
        with pytest.raises(pwf.PWFError) as e:
            _flagged_plan(pwf, g, 4, 0)
        assert e.value.status == 3
    pwf.pwf_debug_fail_alloc(-1)
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] >= free0 - (8 << 20)   # nothing of the failed plans is left
    with _flagged_plan(pwf, g, 4, 0) as plan:                  # and the next plan is whole
        assert plan.handle
