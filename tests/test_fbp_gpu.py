"""Filtered back projection on the CUDA path against the FP64 oracle: random
complex sinograms at assorted sizes (ragged tiles, odd row counts), phantom
projections, and sampled slices of the full 180 x 1024^2 series."""
import math

import numpy as np
import pytest

from oracle import fbp_oracle as F
from paper_2503_20146_gb300 import synth as S

from _cases import rel_l2

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

TOL = 1e-5


def noise_tol(nx):
    """White-noise rows are the worst case for the FP32 back projection: the
    detector position u = x cos + z sin + nx/2 is rounded to ~2 ulp(nx) =
    nx 2^-22, and the interpolated value moves by that times |q1 - q0| <= 2 max|q|
    (smooth rows, like retrieved phases, keep the 1e-5 bound)."""
    return max(TOL, nx * 2.0 ** -22)


@pytest.fixture(scope="module")
def pwf():
    from paper_2503_20146_gb300 import _build
    _build.build()
    from paper_2503_20146_gb300 import pwf as P
    P.load()
    return P


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


@pytest.mark.parametrize("n_angles,ny,nx", [(37, 3, 16), (30, 5, 48), (90, 2, 128), (61, 1, 384), (180, 3, 64),
                                           (45, 2, 96), (20, 1, 192)])
def test_fbp_matches_oracle_on_random_fields(pwf, n_angles, ny, nx):
    rng = np.random.default_rng(n_angles * 1000 + nx)
    psi = (rng.standard_normal((n_angles, ny, nx)) + 1j * rng.standard_normal((n_angles, ny, nx))).astype(np.complex64)
    angles = np.sort(rng.uniform(0.0, math.pi, n_angles))
    vol = pwf.pwf_fbp(dev(psi), angles, S.WAVELENGTH_20KEV_M, S.PIXEL_M).cpu().numpy()
    ref = F.fbp_volume(psi.astype(np.complex128), angles, S.WAVELENGTH_20KEV_M, S.PIXEL_M)
    assert rel_l2(vol, ref) < noise_tol(nx), rel_l2(vol, ref)


def test_fbp_of_phantom_projections_matches_oracle(pwf):
    ph = S.ellipsoid_phantom(S.rng_for(3, 0), size=96, n_ellipsoids=12)
    n = 96
    angles = np.deg2rad(np.arange(180.0))
    xd, yd = S.detector_grid(n, n)
    psi = np.zeros((180, n, n), dtype=np.complex64)
    for a, th in enumerate(angles):
        re, im = S.ellipsoid_projection(ph, th, xd, yd, S.WAVELENGTH_20KEV_M, S.PIXEL_M)
        psi[a] = re + 1j * im
    vol = pwf.pwf_fbp(dev(psi), angles, S.WAVELENGTH_20KEV_M, S.PIXEL_M).cpu().numpy()
    rows = [0, 17, 48, 95]
    ref = F.fbp_volume(psi[:, rows, :].astype(np.complex128), angles, S.WAVELENGTH_20KEV_M, S.PIXEL_M)
    assert rel_l2(vol[rows], ref) < TOL, rel_l2(vol[rows], ref)


def test_fbp_rejects_bad_sizes_and_workspace(pwf):
    psi = torch.zeros((4, 2, 100), dtype=torch.complex64, device="cuda")
    with pytest.raises(pwf.PWFError):
        pwf.pwf_fbp(psi, np.linspace(0, 3, 4), 1e-10, 1e-6)          # 2 nx = 200 is not a transform length
    assert pwf.pwf_fbp_workspace_bytes(4, 2, 100) == 0
    assert pwf.pwf_fbp_workspace_bytes(0, 2, 64) == 0
    psi = torch.zeros((4, 2, 64), dtype=torch.complex64, device="cuda")
    small = torch.empty(16, dtype=torch.uint8, device="cuda")
    with pytest.raises(pwf.PWFError):
        pwf.pwf_fbp(psi, np.linspace(0, 3, 4), 1e-10, 1e-6, workspace=small)


def test_fbp_full_series_sampled_slices(pwf):
    w = S.WORKLOADS["tomo180x1024_iotf"]
    angles = S.tomo_angles(w.batch)
    ph = S.ellipsoid_phantom(S.rng_for(w.config, 999), size=w.nx)
    xd, yd = S.detector_grid(w.ny, w.nx, xp=torch)
    xd, yd = xd.cuda(), yd.cuda()
    psi = torch.empty((w.batch, w.ny, w.nx), dtype=torch.complex64, device="cuda")
    for a in range(w.batch):
        re, im = S.ellipsoid_projection(ph, float(angles[a]), xd, yd, w.wavelength_m, w.pixel_m)
        psi[a] = torch.complex(re.float(), im.float())
    vol = pwf.pwf_fbp(psi, angles, w.wavelength_m, w.pixel_m)
    torch.cuda.synchronize()
    for y in (300, 511):
        ref = F.fbp_slice(psi[:, y, :].cpu().numpy().astype(np.complex128), angles) * \
            (-w.wavelength_m / (2 * math.pi * w.pixel_m))
        got = vol[y].cpu().numpy()
        assert rel_l2(got, ref) < TOL, (y, rel_l2(got, ref))
