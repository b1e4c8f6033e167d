"""The bounds-checked build (PWF_BOUNDS_CHECK) and the debug aid that drives
it: every pass checks the projection index of each CTA against the plan's
batch before it touches memory. The checked library is built beside the
normal one; a row pass over one projection more than the plan holds is caught
(PWF_ERR_BOUNDS, nothing accessed), the checked build computes the same bits
as the normal one (both on the untuned column shapes), and the normal build refuses the overrun without
launching anything."""
import ctypes

import numpy as np
import pytest

from paper_2503_20146_gb300 import synth as S

from _cases import blob_batch, geometry, to_c64, to_f32

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


def _desc(P, g, batch):
    return P.PlanDesc(batch, g.ny, g.nx, g.pixel, g.wavelength, g.L1, g.L2, g.xcoh, g.ycoh, g.gamma,
                      g.alpha.real, g.alpha.imag, g.eta, P.FLAG_GRAPH | P.FLAG_NO_TUNE)


def _inputs(g, batch):
    psi0, t = blob_batch(W2, batch, g.ny, g.nx)
    y = np.abs(np.asarray(psi0)) ** 2 + 1.0
    return (torch.from_numpy(to_f32(y)).cuda(), torch.from_numpy(to_c64(t)).cuda())


def test_normal_build_refuses_the_overrun(pwf):
    g = geometry(W2, 128, 128)
    with pwf.Plan(_desc(pwf, g, 2)) as plan:
        assert pwf.load().pwf_debug_overrun(plan.handle) == 2


def test_checked_build_catches_the_overrun_and_computes_the_same_bits(pwf):
    from paper_2503_20146_gb300 import _build
    lib = pwf.open_library(_build.build(bounds_check=True))
    g = geometry(W2, 128, 128)
    y, t = _inputs(g, 2)
    n = 6
    with pwf.Plan(_desc(pwf, g, 2)) as plan:
        ref = torch.zeros((2, 128, 128), dtype=torch.complex64, device="cuda")
        plan.solve(y, t, ref, n)
    torch.cuda.synchronize()
    d = pwf._desc_struct(_desc(pwf, g, 2))
    h = ctypes.c_void_p()
    assert lib.pwf_plan_create(ctypes.byref(d), ctypes.byref(h)) == 0
    try:
        assert lib.pwf_debug_overrun(h) == 8                  # PWF_ERR_BOUNDS: caught, not accessed
        psi = torch.zeros_like(ref)
        ptr = lambda x: ctypes.c_void_p(x.data_ptr())
        assert lib.pwf_solve(h, ptr(y), ptr(t), ptr(psi), n, 0.0, None, None) == 0
        torch.cuda.synchronize()
        assert torch.equal(psi, ref)
    finally:
        lib.pwf_plan_destroy(h)
