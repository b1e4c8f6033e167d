"""Source-mode partial-coherence variant (K tilted plane-wave modes) on the
CUDA path against the FP64 oracle: forward, gradient, VJP and iterations."""
import numpy as np
import pytest

from oracle import pwf_oracle as O
from paper_2503_20146_gb300 import synth as S

from _cases import blob_batch, geometry, measurement, phase_rms, rel_l2, to_c64, to_f32

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

FWD_TOL, GRAD_TOL, PHASE_TOL = 1e-5, 1e-4, 1e-3
W2 = S.WORKLOADS["blob512_iotf"]
SIGMA = 2.0


@pytest.fixture(scope="module")
def pwf():
    from paper_2503_20146_gb300 import _build
    _build.build()
    from paper_2503_20146_gb300 import pwf as P
    P.load()
    return P


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def modal_plan(P, geom, batch, K):
    d = P.PlanDesc(batch, geom.ny, geom.nx, geom.pixel, geom.wavelength, geom.L1, geom.L2, geom.xcoh, geom.ycoh,
                   geom.gamma, geom.alpha.real, geom.alpha.imag, geom.eta, 0, K, SIGMA)
    return P.Plan(d)


CASES = [("k9_128", 9, 2, 128, 128), ("k25_96x128", 25, 2, 96, 128), ("k9_256x1024", 9, 1, 256, 1024),
         ("k9_1024x64", 9, 2, 1024, 64), ("k9_2048x32", 9, 1, 2048, 32),
         # radix-3 column lengths (24 values per thread: the one-column mode kernels)
         ("k9_768x96", 9, 1, 768, 96), ("k25_1536x32", 25, 1, 1536, 32)]


@pytest.mark.parametrize("name,K,batch,ny,nx", CASES, ids=[c[0] for c in CASES])
def test_modal_forward_gradient_vjp(pwf, name, K, batch, ny, nx):
    geom = geometry(W2, ny, nx)
    modes = O.source_modes(geom, K, SIGMA)
    psi, t = blob_batch(W2, batch, ny, nx)
    psi, t = to_c64(psi), to_c64(t)
    rng = np.random.default_rng(21)
    y = to_f32(np.clip(1.0 + 0.1 * rng.standard_normal((batch, ny, nx)), 0, None))
    gf = to_f32(rng.standard_normal((batch, ny, nx)))
    with modal_plan(pwf, geom, batch, K) as plan:
        f = plan.forward(dev(psi), dev(t)).cpu().numpy()
        g, L = plan.gradient(dev(psi), dev(t), dev(y))
        g, L = g.cpu().numpy(), L.cpu().numpy()
        gp, gt = plan.vjp(dev(psi), dev(t), dev(gf))
        gp, gt = gp.cpu().numpy(), gt.cpu().numpy()
    T64 = t.astype(np.complex128)
    gt_ref = np.zeros_like(T64)
    for b in range(batch):
        P64 = psi[b].astype(np.complex128)
        assert rel_l2(f[b], O.modal_intensity(P64, T64, geom, modes)) <= FWD_TOL
        ge, le = O.modal_gradient(P64, T64, y[b].astype(np.float64), geom, modes)
        assert rel_l2(g[b], ge) <= GRAD_TOL
        assert abs(L[b] - le) <= 1e-5 * le
        vp, vt = O.modal_forward_vjp(P64, T64, gf[b].astype(np.float64), geom, modes)
        assert rel_l2(gp[b], vp) <= GRAD_TOL
        gt_ref += vt
    assert rel_l2(gt, gt_ref) <= GRAD_TOL


@pytest.mark.parametrize("K,n,iters", [(9, 128, 30), (25, 128, 10), (9, 512, 20)], ids=["k9_128", "k25_128", "k9_512"])
def test_modal_solve_matches_oracle(pwf, K, n, iters):
    geom = geometry(W2, n, n)
    modes = O.source_modes(geom, K, SIGMA)
    psi_true, t = blob_batch(W2, 1, n, n)
    t = to_c64(t)
    f_true = O.modal_intensity(psi_true[0], t.astype(np.complex128), geom, modes)
    y = to_f32(S.poisson_measurement(f_true, W2.photons, S.rng_for(W2.config, 77))[None])
    ref = O.modal_solve(y[0].astype(np.float64), t.astype(np.complex128), geom, modes, iters)
    with modal_plan(pwf, geom, 1, K) as plan:
        p = torch.zeros((1, n, n), dtype=torch.complex64, device="cuda")
        it, loss = plan.solve(dev(y), dev(t), p, iters)
    assert int(it[0]) == iters
    assert phase_rms(p.cpu().numpy()[0], ref.psi) <= PHASE_TOL
    assert abs(loss[0] - ref.losses[-1]) <= 1e-3 * ref.losses[-1]


# every mode-pass shape of both radix schedules (passes 6 and 7 of the shape
# control), forward and gradient against the oracle
SHAPE_CASES = [("k9_1024x64", 9, 2, 1024, 64), ("k9_2048x32", 9, 1, 2048, 32), ("k9_768x96", 9, 1, 768, 96),
               ("k9_256x128", 9, 2, 256, 128), ("k9_1536x32", 9, 1, 1536, 32)]


@pytest.mark.parametrize("name,K,batch,ny,nx", SHAPE_CASES, ids=[c[0] for c in SHAPE_CASES])
def test_every_mode_shape_matches_oracle(pwf, name, K, batch, ny, nx):
    geom = geometry(W2, ny, nx)
    modes = O.source_modes(geom, K, SIGMA)
    psi, t = blob_batch(W2, batch, ny, nx)
    psi, t = to_c64(psi), to_c64(t)
    y = to_f32(np.clip(1.0 + 0.1 * np.random.default_rng(22).standard_normal((batch, ny, nx)), 0, None))
    b = batch - 1
    P64, T64 = psi[b].astype(np.complex128), t.astype(np.complex128)
    f_ref = O.modal_intensity(P64, T64, geom, modes)
    g_ref, _ = O.modal_gradient(P64, T64, y[b].astype(np.float64), geom, modes)
    with modal_plan(pwf, geom, batch, K) as plan:
        counts = [pwf.pwf_plan_column_shapes(plan.handle, m) for m in (7, 8)]
        assert min(counts) >= 2
        for k in range(max(counts)):
            for m, c in zip((7, 8), counts):
                pwf.pwf_plan_set_column_shape(plan.handle, m, min(k, c - 1))
            f = plan.forward(dev(psi), dev(t)).cpu().numpy()
            g, _ = plan.gradient(dev(psi), dev(t), dev(y))
            desc = pwf.pwf_plan_describe(plan.handle)
            assert rel_l2(f[b], f_ref) <= FWD_TOL, (k, desc)
            assert rel_l2(g.cpu().numpy()[b], g_ref) <= GRAD_TOL, (k, desc)
