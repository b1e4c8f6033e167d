"""Differentiation through torch.autograd: the hand-written adjoint (VJP)
against central finite differences and against the FP64 oracle's VJP."""
import numpy as np
import pytest

from oracle import pwf_oracle as O
from paper_2503_20146_gb300 import synth as S

from _cases import blob_batch, geometry, rel_l2, to_c64

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    from paper_2503_20146_gb300 import _build
    _build.build()
    from paper_2503_20146_gb300 import pwf
    pwf.load()
    return pwf


def make_plan(P, geom, batch):
    return P.Plan(P.PlanDesc(batch, geom.ny, geom.nx, geom.pixel, geom.wavelength, geom.L1, geom.L2, geom.xcoh,
                             geom.ycoh, geom.gamma, geom.alpha.real, geom.alpha.imag, geom.eta))


def _inputs(w, batch, n, seed=3):
    psi, t = blob_batch(w, batch, n, n)
    rng = np.random.default_rng(seed)
    t = t * (1.0 + 0.1 * rng.standard_normal(t.shape))
    return to_c64(psi), to_c64(t), rng


def test_autograd_matches_oracle_vjp(P):
    from paper_2503_20146_gb300.autograd import physical_model
    w = S.WORKLOADS["blob512_iotf"]
    geom = geometry(w, 128, 128)
    psi, t, rng = _inputs(w, 2, 128)
    wts = rng.standard_normal((2, 128, 128)).astype(np.float32)
    with make_plan(P, geom, 2) as plan:
        ps = torch.from_numpy(psi).cuda().requires_grad_(True)
        ts = torch.from_numpy(t).cuda().requires_grad_(True)
        f = physical_model(ps, ts, plan)
        L = (f * torch.from_numpy(wts).cuda()).sum()
        L.backward()
        gp, gt = ps.grad.cpu().numpy(), ts.grad.cpu().numpy()
    ep, et = O.forward_vjp_batch(psi.astype(np.complex128), t.astype(np.complex128), wts.astype(np.float64), geom)
    assert rel_l2(gp, ep) <= 1e-4
    assert rel_l2(gt, et) <= 1e-4


def _fd_check(P, geom, batch, n, steps=(1e-3,), tol=2e-2, ndir=2):
    """Central differences of L = sum(w f) along reweighted-gradient directions vs the autograd gradient."""
    from paper_2503_20146_gb300.autograd import physical_model
    w = S.WORKLOADS["blob512_iotf"]
    psi, t, rng = _inputs(w, batch, n, seed=9)
    wts = torch.from_numpy(rng.standard_normal((batch, n, n)).astype(np.float32)).cuda()
    with make_plan(P, geom, batch) as plan:
        ps = torch.from_numpy(psi).cuda().requires_grad_(True)
        ts = torch.from_numpy(t).cuda().requires_grad_(True)
        (physical_model(ps, ts, plan) * wts).sum().backward()
        for which, grad in (("psi", ps.grad), ("t", ts.grad)):
            for k in range(ndir):
                # Directions along a random reweighting of the gradient: the
                # directional derivative then dominates the float32 rounding of
                # sum(w (f+ - f-)) / (2 eps), which is ~1e-4 / eps here.
                m = torch.from_numpy(rng.uniform(0.5, 1.5, grad.shape).astype(np.float32)).cuda()
                d = (grad * m).contiguous()
                d = d / d.abs().max()
                an = float((grad.real.double() * d.real.double() + grad.imag.double() * d.imag.double()).sum())
                for eps in steps:
                    with torch.no_grad():
                        if which == "psi":
                            fp = plan.forward((ps + eps * d).contiguous(), ts.detach())
                            fm = plan.forward((ps - eps * d).contiguous(), ts.detach())
                        else:
                            fp = plan.forward(ps.detach(), (ts + eps * d).contiguous())
                            fm = plan.forward(ps.detach(), (ts - eps * d).contiguous())
                        fd = float(((fp.double() - fm.double()) * wts.double()).sum()) / (2 * eps)
                    assert abs(fd - an) <= tol * abs(an), (which, k, eps, fd, an)


def test_finite_differences_small(P):
    w = S.WORKLOADS["blob512_iotf"]
    _fd_check(P, geometry(w, 256, 256), 2, 256)


def test_differentiation_workload_2048_batch16(P):
    """16 projections at 2048^2: forward + backward through autograd w.r.t. psi
    and t; central differences (step 1e-3) along a reweighted gradient, and two
    sampled projections against the oracle's VJP."""
    from paper_2503_20146_gb300.autograd import physical_model
    w = S.WORKLOADS["grad16x2048_iotf"]
    geom = geometry(w)
    _fd_check(P, geom, w.batch, w.ny, ndir=1)
    psi, t, rng = _inputs(w, w.batch, w.ny, seed=21)
    wts = rng.standard_normal((w.batch, w.ny, w.nx)).astype(np.float32)
    with make_plan(P, geom, w.batch) as plan:
        torch.cuda.reset_peak_memory_stats()
        base = torch.cuda.memory_allocated()
        ps = torch.from_numpy(psi).cuda().requires_grad_(True)
        ts = torch.from_numpy(t).cuda().requires_grad_(True)
        f = physical_model(ps, ts, plan)
        (f * torch.from_numpy(wts).cuda()).sum().backward()
        gp = ps.grad.cpu().numpy()
        gt = ts.grad.cpu().numpy()
        # torch-side memory: psi, t, f, weights and the two gradients; the
        # propagated fields live only in the plan's fixed workspace
        field = w.batch * w.ny * w.nx * 8
        assert torch.cuda.max_memory_allocated() - base <= 5 * field
    # grad_t sums all 16 projections: compare with the oracle on the same sum
    ep, et = O.forward_vjp_batch(psi.astype(np.complex128), t.astype(np.complex128), wts.astype(np.float64), geom)
    for b in (0, 11):
        assert rel_l2(gp[b], ep[b]) <= 1e-4
    assert rel_l2(gt, et) <= 1e-4
