"""Calibration from the reference speckle on the CUDA path against the FP64
oracle: coherence lengths from the intensity autocorrelation, and the diffuser
recovered by Wiener deconvolution and back-propagation (Methods, IOTF and
diffuser transmission function)."""
import numpy as np
import pytest

from oracle import pwf_oracle as O
from paper_2503_20146_gb300 import synth as S

from _cases import rel_l2, to_f32

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


def plan_for(P, g):
    return P.Plan(P.PlanDesc(1, g.ny, g.nx, g.pixel, g.wavelength, g.L1, g.L2, g.xcoh, g.ycoh, g.gamma,
                             g.alpha.real, g.alpha.imag, g.eta))


def reference_speckle(g, seed):
    """Partially coherent reference speckle without the sample (Eq. (1), psi = 0)."""
    t = S.diffuser(g.ny, g.nx, S.rng_for(7, seed))
    I_coh = np.abs(O.propagate(t, g, g.L2)) ** 2
    return O.fourier_filter(I_coh, O.iotf(g)).real


@pytest.mark.parametrize("ny,nx,max_lag", [(256, 256, 3), (128, 512, 3), (1024, 1024, 4)])
def test_coherence_lengths_match_oracle(pwf, ny, nx, max_lag):
    g = O.Geometry(ny, nx, 1e-6, S.WAVELENGTH_20KEV_M, 0.1, 0.4, 3e-6, 4e-6)
    I = reference_speckle(g, ny + nx)
    xo, yo = O.calibrate_coherence(I, g.pixel, max_lag)
    with plan_for(pwf, g) as plan:
        xg, yg = plan.calibrate_coherence(dev(to_f32(I)), max_lag)
    # the fit is a smooth function of a few fp32 autocorrelation sums
    assert abs(xg - xo) / xo < 1e-4 and abs(yg - yo) / yo < 1e-4, (xg, xo, yg, yo)


def test_coherence_rejects_bad_lags(pwf):
    g = O.Geometry(64, 64, 1e-6, S.WAVELENGTH_20KEV_M, 0.1, 0.4, 3e-6, 3e-6)
    I = dev(to_f32(reference_speckle(g, 1)))
    with plan_for(pwf, g) as plan:
        for lag in (0, 32):
            with pytest.raises(pwf.PWFError):
                plan.calibrate_coherence(I, lag)


@pytest.mark.parametrize("ny,nx,eps", [(128, 128, 1e-3), (96, 256, 1e-2), (1024, 1024, 1e-3)])
def test_diffuser_from_reference_matches_oracle(pwf, ny, nx, eps):
    g = O.Geometry(ny, nx, 1e-6, S.WAVELENGTH_20KEV_M, 0.1, 0.4, 3e-6, 3.5e-6)
    I = reference_speckle(g, 3 * ny + nx)
    t_o = O.diffuser_from_reference(I, g, eps)
    with plan_for(pwf, g) as plan:
        t_g = plan.diffuser_from_reference(dev(to_f32(I)), eps).cpu().numpy()
    assert rel_l2(t_g, t_o) < 1e-5
