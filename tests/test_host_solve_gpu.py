"""pwf_solve_host: Algorithm S1 from host buffers, the batch streamed through
the device in chunks with the copies overlapping the solve. Checked against
the device-buffer solve, the FP64 oracle, and for its argument rules."""
import numpy as np
import pytest

from oracle import pwf_oracle as O
from paper_2503_20146_gb300 import synth as S

from _cases import blob_batch, geometry, measurement, phase_rms, rel_l2, to_c64, to_f32

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

W1 = S.WORKLOADS["blob128_coherent"]
W2 = S.WORKLOADS["blob512_iotf"]


@pytest.fixture(scope="module")
def pwf():
    from paper_2503_20146_gb300 import _build
    _build.build()
    from paper_2503_20146_gb300 import pwf as P
    P.load()
    return P


def plan_for(P, g, batch, n_modes=0, sigma=0.0):
    return P.Plan(P.PlanDesc(batch, g.ny, g.nx, g.pixel, g.wavelength, g.L1, g.L2, g.xcoh, g.ycoh, g.gamma,
                             g.alpha.real, g.alpha.imag, g.eta, 0, n_modes, sigma))


def case(w, batch, ny, nx):
    g = geometry(w, ny, nx)
    psi_true, t = blob_batch(w, batch, ny, nx)
    t = to_c64(t)
    y = to_f32(measurement(psi_true, t.astype(np.complex128), g, w.photons, w.config))
    return g, t, y


def pinned(a):
    return torch.from_numpy(np.ascontiguousarray(a)).pin_memory()


def device_solve(plan, y, t, psi0, iters, corr_tol=0.0):
    psi = torch.from_numpy(np.ascontiguousarray(psi0)).cuda()
    it, loss = plan.solve(torch.from_numpy(y).cuda(), torch.from_numpy(t).cuda(), psi, iters, corr_tol)
    return psi.cpu().numpy(), it, loss


@pytest.mark.parametrize("w,batch,ny,nx,chunk", [(W2, 6, 128, 96, 0), (W2, 5, 64, 64, 1), (W1, 4, 64, 64, 4),
                                                 (W2, 8, 256, 128, 2)])
def test_host_solve_matches_device_solve(pwf, w, batch, ny, nx, chunk):
    g, t, y = case(w, batch, ny, nx)
    iters = 12
    psi_h = pinned(np.zeros((batch, ny, nx), np.complex64))
    with plan_for(pwf, g, batch) as plan:
        it_h, loss_h = plan.solve_host(pinned(y), pinned(t), psi_h, iters, chunk=chunk)
        ref, it_d, loss_d = device_solve(plan, y, t, np.zeros((batch, ny, nx), np.complex64), iters)
    got = psi_h.numpy()
    assert (it_h == iters).all() and (it_d == iters).all()
    # chunk-sized plans may pick other column-pass shapes: rounding-level differences only
    assert rel_l2(got, ref) <= 1e-5, rel_l2(got, ref)
    np.testing.assert_allclose(loss_h, loss_d, rtol=1e-5)


def test_host_solve_matches_oracle(pwf):
    g, t, y = case(W2, 3, 128, 128)
    n = 20
    refs = [O.solve(y[b].astype(np.float64), t.astype(np.complex128), g, n) for b in range(3)]
    psi_h = np.zeros((3, 128, 128), np.complex64)             # pageable numpy buffers work too
    with plan_for(pwf, g, 3) as plan:
        it, loss = plan.solve_host(y, t, psi_h, n, psi_is_input=False, chunk=1)
    for b in range(3):
        assert it[b] == n
        assert phase_rms(psi_h[b], refs[b].psi) <= 1e-3
        assert abs(loss[b] - refs[b].losses[-1]) <= 1e-3 * refs[b].losses[-1]


def test_host_solve_continues_from_the_given_psi_and_stops_on_correlation(pwf):
    g, t, y = case(W2, 4, 64, 64)
    with plan_for(pwf, g, 4) as plan:
        start, _, _ = device_solve(plan, y, t, np.zeros((4, 64, 64), np.complex64), 5)
        ref, it_d, _ = device_solve(plan, y, t, start, 40, corr_tol=0.999999)
        psi_h = pinned(start)
        it_h, _ = plan.solve_host(pinned(y), pinned(t), psi_h, 40, corr_tol=0.999999, chunk=2)
    assert list(it_h) == list(it_d)
    assert rel_l2(psi_h.numpy(), ref) <= 1e-5


def test_host_solve_with_source_modes_matches_device_solve(pwf):
    g, t, y = case(W2, 4, 128, 128)
    psi_h = pinned(np.zeros((4, 128, 128), np.complex64))
    with plan_for(pwf, g, 4, n_modes=9, sigma=1.5) as plan:
        plan.solve_host(pinned(y), pinned(t), psi_h, 6, chunk=2)
        ref, _, _ = device_solve(plan, y, t, np.zeros((4, 128, 128), np.complex64), 6)
    assert rel_l2(psi_h.numpy(), ref) <= 1e-5


def test_host_solve_argument_rules(pwf):
    g, t, y = case(W2, 6, 64, 64)
    psi = np.zeros((6, 64, 64), np.complex64)
    with plan_for(pwf, g, 6) as plan:
        with pytest.raises(pwf.PWFError):
            plan.solve_host(y, t, psi, 2, chunk=4)                 # 4 does not divide 6
        with pytest.raises(pwf.PWFError):
            plan.solve_host(y, t, psi, 2, chunk=7)
        with pytest.raises(ValueError):
            plan.solve_host(y[:5], t, psi, 2)                      # wrong size
        with pytest.raises(TypeError):
            plan.solve_host(torch.from_numpy(y).cuda(), t, psi, 2)  # device tensor
        it, _ = plan.solve_host(y, t, psi, 0)                      # zero iterations: psi unchanged
        assert (it == 0).all() and not psi.any()
