"""Joint refinement of the shared diffuser on the CUDA path (pwf_solve_joint)
against the FP64 oracle's joint_pwf: refined t, retrieved psi and losses."""
import numpy as np
import pytest

from oracle import pwf_oracle as O
from paper_2503_20146_gb300 import synth as S

from _cases import blob_batch, geometry, measurement, phase_rms, rel_l2, to_c64, to_f32

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pwf():
    from paper_2503_20146_gb300 import _build
    _build.build()
    from paper_2503_20146_gb300 import pwf as P
    P.load()
    return P


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def plan_for(P, g, batch, flags=0):
    return P.Plan(P.PlanDesc(batch, g.ny, g.nx, g.pixel, g.wavelength, g.L1, g.L2, g.xcoh, g.ycoh, g.gamma,
                             g.alpha.real, g.alpha.imag, g.eta, flags))


def perturbed_case(wname, batch, ny, nx):
    w = S.WORKLOADS[wname]
    g = geometry(w, ny=ny, nx=nx)
    psi_true, t = blob_batch(w, batch, ny=ny, nx=nx)
    y = measurement(psi_true, t, g, 1e4, w.config)
    t0 = t * np.exp(0.3j * np.angle(S.diffuser(ny, nx, np.random.default_rng(5))))
    return g, y, t0


@pytest.mark.parametrize("wname,batch,ny,nx,iters", [("blob512_iotf", 3, 64, 64, 10),
                                                      ("blob512_iotf", 2, 96, 128, 8),
                                                      ("blob128_coherent", 2, 128, 128, 8)])
def test_joint_refinement_matches_oracle(pwf, wname, batch, ny, nx, iters):
    g, y, t0 = perturbed_case(wname, batch, ny, nx)
    eta_t = 3e-3
    ref = O.joint_solve(y, t0, g, iters, eta_t)
    with plan_for(pwf, g, batch) as plan:
        t = dev(to_c64(t0))
        psi = torch.zeros((batch, ny, nx), dtype=torch.complex64, device="cuda")
        it, loss = plan.solve_joint(dev(to_f32(y)), t, psi, iters, eta_t)
        t_g, psi_g = t.cpu().numpy(), psi.cpu().numpy()
    assert (it == iters).all()
    assert rel_l2(t_g, ref.t) < 1e-5, rel_l2(t_g, ref.t)
    assert rel_l2(t_g - t0, ref.t - t0) < 1e-3          # the refinement step itself
    assert rel_l2(psi_g, ref.psi) < 1e-4, rel_l2(psi_g, ref.psi)
    assert abs(loss.sum() - ref.losses[-1]) < 1e-4 * ref.losses[-1]


def test_joint_with_zero_step_equals_solve(pwf):
    # the joint refinement runs on the graph replay, so pwf_solve is held to it
    g, y, t0 = perturbed_case("blob512_iotf", 3, 64, 64)
    with plan_for(pwf, g, 3, pwf.FLAG_GRAPH) as plan:
        yd, t = dev(to_f32(y)), dev(to_c64(t0))
        p1 = torch.zeros((3, 64, 64), dtype=torch.complex64, device="cuda")
        p2 = torch.zeros_like(p1)
        plan.solve(yd, t, p1, 7)
        plan.solve_joint(yd, t, p2, 7, 0.0)
        assert torch.equal(p1, p2)
        assert torch.equal(t, dev(to_c64(t0)))


def test_joint_full_size_sample_matches_oracle(pwf):
    w = S.WORKLOADS["tomo180x1024_iotf"]
    g, y, t0 = perturbed_case("tomo180x1024_iotf", 4, w.ny, w.nx)
    ref = O.joint_solve(y, t0, g, 2, 1e-3)
    with plan_for(pwf, g, 4) as plan:
        t = dev(to_c64(t0))
        psi = torch.zeros((4, w.ny, w.nx), dtype=torch.complex64, device="cuda")
        plan.solve_joint(dev(to_f32(y)), t, psi, 2, 1e-3)
        assert rel_l2(t.cpu().numpy(), ref.t) < 1e-5
        # at 1024^2, P^-1 reaches N^2 at the lowest bins and lifts FP32 rounding
        # there: compare with the retrieved-phase criterion (RMS, radians)
        got = psi.cpu().numpy()
        assert phase_rms(got, ref.psi) < 1e-3
        assert np.sqrt(np.mean((got.real - ref.psi.real) ** 2)) < 1e-3


def test_joint_rejects_unsupported_plans(pwf):
    g, y, t0 = perturbed_case("blob512_iotf", 2, 64, 64)
    yd, t = dev(to_f32(y)), dev(to_c64(t0))
    psi = torch.zeros((2, 64, 64), dtype=torch.complex64, device="cuda")
    with plan_for(pwf, g, 2) as plan:
        with pytest.raises(pwf.PWFError):
            plan.solve_joint(yd, t, psi, 2, -1.0)
    with plan_for(pwf, g, 2, pwf.FLAG_PLAIN) as plan:
        with pytest.raises(pwf.PWFError):
            plan.solve_joint(yd, t, psi, 2, 1e-3)
