"""The workloads at their own sizes and iteration counts, CUDA path against the
FP64 oracle on sampled projections.

* 512^2 single projection with K = 9 source modes, 100 iterations;
* the 180 x 1024^2 tomographic series, 20 iterations over the whole series in
  the benchmark's launch configuration, IOTF form and K = 9 form, sampled
  projections against the oracle;
* differentiation of 16 x 2048^2 with K = 25 modes: VJP w.r.t. psi and t on
  two sampled projections against the oracle's VJP, and central differences
  (step 1e-3, FP64 oracle) along the oracle's gradient;
* the uneven batch (16 each of 256^2, 768^2, 1536^2, 2048^2, K = 25) in one
  group, one sampled projection per class against the oracle.

The measurements are made by the oracle's forward model (never by the CUDA
path). The oracle's work runs in a spawn process pool started before the GPU
work, so the host cores and the GPU work at the same time.

Tolerances (as the other parity tests): forward 1e-5, gradient relative L2
1e-4, retrieved phase (and log-amplitude) RMS 1e-3 rad.
"""
import numpy as np
import pytest

import _oracle_jobs as J
from oracle import pwf_oracle as O
from paper_2503_20146_gb300 import synth as S

from _cases import geometry, phase_rms, rel_l2

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

GRAD_TOL, PHASE_TOL = 1e-4, 1e-3
TOMO_ITERS = 20
TOMO_SAMPLES = (5, 150)
TOMO_K9_SAMPLE = 97
MIXED_ITERS = 4
MIXED_SAMPLE = 5
FD_EPS = 1e-3


@pytest.fixture(scope="module")
def pwf():
    from paper_2503_20146_gb300 import _build
    _build.build()
    from paper_2503_20146_gb300 import pwf as P
    P.load()
    return P


@pytest.fixture(scope="module")
def jobs():
    """Every independent oracle job of this module, submitted at once."""
    ex = J.pool()
    fut = {
        "modal512": ex.submit(J.blob_modal_solve, 512, 9, 100),
        "tomo_y": [ex.submit(J.tomo_measurement, b) for b in range(180)],
        "tomo_iotf": {b: ex.submit(J.tomo_solve, b, TOMO_ITERS) for b in TOMO_SAMPLES},
        "tomo_k9": ex.submit(J.tomo_solve, TOMO_K9_SAMPLE, TOMO_ITERS, 9),
        "vjp": {b: ex.submit(J.grad_vjp, b) for b in (0, 11)},
        "mixed_y": {(k, b): ex.submit(J.mixed_measurement, k, n, b)
                    for k, n in enumerate(S.MIXED_SIZES) for b in range(S.MIXED_PER_SIZE)},
        "mixed": {k: ex.submit(J.mixed_solve, k, n, MIXED_SAMPLE, MIXED_ITERS)
                  for k, n in enumerate(S.MIXED_SIZES) if n >= 768},
    }
    yield ex, fut
    ex.shutdown(wait=False, cancel_futures=True)


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def desc(P, geom, batch, K=0, sigma=0.0):
    return P.PlanDesc(batch, geom.ny, geom.nx, geom.pixel, geom.wavelength, geom.L1, geom.L2, geom.xcoh,
                      geom.ycoh, geom.gamma, geom.alpha.real, geom.alpha.imag, geom.eta, 0, K, sigma)


def amp_rms(a, b):
    return float(np.sqrt(np.mean((np.asarray(a).real - np.asarray(b).real) ** 2)))


def test_single_512_k9_for_100_iterations(pwf, jobs):
    _, fut = jobs
    y, t = J.blob_modal_measurement(512, 9)
    geom = geometry(S.WORKLOADS["blob512_iotf"], 512, 512)
    with pwf.Plan(desc(pwf, geom, 1, 9, J.SIGMA)) as plan:
        p = torch.zeros((1, 512, 512), dtype=torch.complex64, device="cuda")
        it, loss = plan.solve(dev(y[None]), dev(t), p, 100)
    ref_psi, ref_losses = fut["modal512"].result()
    assert int(it[0]) == 100
    got = p.cpu().numpy()[0]
    assert phase_rms(got, ref_psi) <= PHASE_TOL
    assert amp_rms(got, ref_psi) <= PHASE_TOL
    assert abs(loss[0] - ref_losses[-1]) <= 1e-3 * ref_losses[-1]


@pytest.fixture(scope="module")
def tomo_y(jobs):
    _, fut = jobs
    return np.stack([f.result() for f in fut["tomo_y"]])


@pytest.mark.parametrize("K", [0, 9], ids=["iotf", "k9"])
def test_tomo_series_20_iterations_sampled(pwf, jobs, tomo_y, K):
    """All 180 projections iterate together (one plan, the captured iteration
    graph the benchmark times); sampled projections against the oracle."""
    _, fut = jobs
    w = S.WORKLOADS["tomo180x1024_iotf"]
    geom = geometry(w)
    t32 = J.tomo_t32()
    with pwf.Plan(desc(pwf, geom, 180, K, J.SIGMA if K else 0.0)) as plan:
        psi = torch.zeros((180, 1024, 1024), dtype=torch.complex64, device="cuda")
        iters, _ = plan.solve(dev(tomo_y), dev(t32), psi, TOMO_ITERS)
        assert list(iters) == [TOMO_ITERS] * 180
        samples = TOMO_SAMPLES if K == 0 else (TOMO_K9_SAMPLE,)
        got = {b: psi[b].cpu().numpy() for b in samples}
    for b in samples:
        ref = fut["tomo_iotf"][b].result() if K == 0 else fut["tomo_k9"].result()
        assert phase_rms(got[b], ref) <= PHASE_TOL, b
        assert amp_rms(got[b], ref) <= PHASE_TOL, b


def test_differentiation_16x2048_k25(pwf, jobs):
    """VJP of f(psi, t) with 25 source modes for 16 projections at 2048^2:
    grad_psi of projections 0 and 11 and grad_t (cotangent on those two
    projections) against the oracle; central differences of the FP64 oracle
    along its own gradient (reweighted) against the CUDA gradient."""
    ex, fut = jobs
    w = S.WORKLOADS["grad16x2048_k25"]
    geom = geometry(w)
    psi, t, wts = J.grad_inputs()
    two = np.zeros_like(wts)
    two[[0, 11]] = wts[[0, 11]]
    with pwf.Plan(desc(pwf, geom, w.batch, w.n_modes, w.mode_sigma_px)) as plan:
        gp, _ = plan.vjp(dev(psi), dev(t), dev(wts))              # the workload's call
        gp = gp.cpu().numpy()
        _, gt2 = plan.vjp(dev(psi), dev(t), dev(two))             # grad_t of projections 0 and 11
        gt2 = gt2.cpu().numpy()
    ref = {b: fut["vjp"][b].result() for b in (0, 11)}
    for b in (0, 11):
        assert rel_l2(gp[b], ref[b][0]) <= GRAD_TOL, b
    gt_ref = ref[0][1] + ref[11][1]
    assert rel_l2(gt2, gt_ref) <= GRAD_TOL
    # central differences along the oracle's gradient, reweighted by a seeded
    # factor in [0.5, 1.5] so that the direction is not the gradient itself
    rng = np.random.default_rng(5)
    d_psi = ref[0][0] * rng.uniform(0.5, 1.5, ref[0][0].shape)
    d_psi /= np.max(np.abs(d_psi))
    d_t = gt_ref * rng.uniform(0.5, 1.5, gt_ref.shape)
    d_t /= np.max(np.abs(d_t))
    fd = {}
    for s in (1, -1):
        fd[("p", s)] = ex.submit(J.grad_weighted_intensity, (0,), s * FD_EPS, d_psi, None)
        fd[("t", s)] = ex.submit(J.grad_weighted_intensity, (0, 11), s * FD_EPS, None, d_t)
    fd_psi = (fd[("p", 1)].result() - fd[("p", -1)].result()) / (2 * FD_EPS)
    fd_t = (fd[("t", 1)].result() - fd[("t", -1)].result()) / (2 * FD_EPS)
    an_psi = float(np.sum(gp[0].real * d_psi.real + gp[0].imag * d_psi.imag))
    an_t = float(np.sum(gt2.real * d_t.real + gt2.imag * d_t.imag))
    assert abs(fd_psi - an_psi) <= GRAD_TOL * abs(fd_psi), (fd_psi, an_psi)
    assert abs(fd_t - an_t) <= GRAD_TOL * abs(fd_t), (fd_t, an_t)


def test_uneven_batch_k25_sampled(pwf, jobs):
    """The 64-projection uneven batch with 25 source modes in one group; the
    same graph launch per iteration the benchmark times; projection 5 of the
    768^2, 1536^2 and 2048^2 classes against the oracle."""
    _, fut = jobs
    w = S.WORKLOADS["mixed64_k25"]
    plans, ys, ts, psis = [], [], [], []
    try:
        for k, n in enumerate(S.MIXED_SIZES):
            geom = geometry(w, n, n)
            plans.append(pwf.Plan(desc(pwf, geom, S.MIXED_PER_SIZE, w.n_modes, w.mode_sigma_px)))
            y = np.stack([fut["mixed_y"][(k, b)].result() for b in range(S.MIXED_PER_SIZE)])
            ys.append(dev(y))
            ts.append(dev(J.mixed_class_t32(n)))
            psis.append(torch.zeros((S.MIXED_PER_SIZE, n, n), dtype=torch.complex64, device="cuda"))
        g = pwf.pwf_group_create(plans)
        try:
            pwf.pwf_group_solve(g, ys, ts, psis, MIXED_ITERS)
            torch.cuda.synchronize()
            for k in range(len(plans)):
                _, it = pwf.pwf_group_read(g, k, S.MIXED_PER_SIZE)
                assert list(it) == [MIXED_ITERS] * S.MIXED_PER_SIZE
        finally:
            pwf.pwf_group_destroy(g)
        for k, n in enumerate(S.MIXED_SIZES):
            if n < 768:
                continue
            got = psis[k][MIXED_SAMPLE].cpu().numpy()
            ref = fut["mixed"][k].result()
            assert phase_rms(got, ref) <= PHASE_TOL, n
            assert amp_rms(got, ref) <= PHASE_TOL, n
    finally:
        for p in plans:
            p.close()
