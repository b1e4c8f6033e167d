"""CUDA path vs the FP64 oracle, element by element, through the C ABI.

Tolerances (float32 path against float64 oracle on identical, float32-rounded
inputs): forward intensity relative L2 <= 1e-5; gradient relative L2 <= 1e-4;
retrieved phase RMS difference <= 1e-3 rad after the workload's iterations.
"""
import numpy as np
import pytest

from oracle import pwf_oracle as O
from paper_2503_20146_gb300 import synth as S

from _cases import blob_batch, geometry, measurement, phase_rms, rel_l2, to_c64, to_f32

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

FWD_TOL = 1e-5
GRAD_TOL = 1e-4
PHASE_TOL = 1e-3

W1 = S.WORKLOADS["blob128_coherent"]
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


def plan_for(P, geom: O.Geometry, batch: int, flags: int = 0):
    d = P.PlanDesc(batch, geom.ny, geom.nx, geom.pixel, geom.wavelength, geom.L1, geom.L2, geom.xcoh,
                   geom.ycoh, geom.gamma, geom.alpha.real, geom.alpha.imag, geom.eta, flags)
    return P.Plan(d)


# (name, workload, batch, ny, nx, coherent)
CASES = [
    ("c128_coh", W1, 1, 128, 128, True),
    ("c128_iotf_b3", W2, 3, 128, 128, False),
    ("rect96x128_iotf", W2, 2, 96, 128, False),
    ("rect768x256_iotf", W2, 1, 768, 256, False),
    ("tiny16x32_coh", W1, 2, 16, 32, True),
    ("c512_iotf", W2, 1, 512, 512, False),
    ("rect64x2048_coh", W1, 1, 64, 2048, True),
    ("rect1536x64_iotf", W2, 1, 1536, 64, False),
]


def case_inputs(w, batch, ny, nx, coherent):
    geom = geometry(w, ny, nx, xcoh=0.0 if coherent else None)
    psi, t = blob_batch(w, batch, ny, nx)
    psi, t = to_c64(psi), to_c64(t)
    return geom, psi, t


@pytest.mark.parametrize("name,w,batch,ny,nx,coh", CASES, ids=[c[0] for c in CASES])
def test_forward_parity(pwf, name, w, batch, ny, nx, coh):
    geom, psi, t = case_inputs(w, batch, ny, nx, coh)
    expect = O.intensity_batch(psi.astype(np.complex128), t.astype(np.complex128), geom)
    with plan_for(pwf, geom, batch) as plan:
        f = plan.forward(dev(psi), dev(t)).cpu().numpy()
    assert rel_l2(f, expect) <= FWD_TOL


@pytest.mark.parametrize("name,w,batch,ny,nx,coh", CASES, ids=[c[0] for c in CASES])
def test_gradient_parity(pwf, name, w, batch, ny, nx, coh):
    geom, psi, t = case_inputs(w, batch, ny, nx, coh)
    psi_true, _ = blob_batch(w, batch, ny, nx, seed_proj0=7)
    y = to_f32(measurement(psi_true, t.astype(np.complex128), geom, w.photons, w.config))
    g_exp, L_exp = O.gradient_batch(psi.astype(np.complex128), t.astype(np.complex128), y.astype(np.float64), geom)
    with plan_for(pwf, geom, batch) as plan:
        g, L = plan.gradient(dev(psi), dev(t), dev(y))
        g, L = g.cpu().numpy(), L.cpu().numpy()
    assert rel_l2(g, g_exp) <= GRAD_TOL
    assert np.max(np.abs(L - L_exp) / np.abs(L_exp)) <= 1e-5


@pytest.mark.parametrize("name,w,batch,ny,nx,coh", CASES[:4], ids=[c[0] for c in CASES[:4]])
def test_vjp_parity_psi_and_diffuser(pwf, name, w, batch, ny, nx, coh):
    geom, psi, t = case_inputs(w, batch, ny, nx, coh)
    rng = np.random.default_rng(11)
    gf = to_f32(rng.standard_normal((batch, ny, nx)))
    # a diffuser with |t| != 1 exercises the conj(t) and max|t|^2 paths
    t = to_c64(t * (1.0 + 0.2 * rng.standard_normal(t.shape)))
    gp_exp, gt_exp = O.forward_vjp_batch(psi.astype(np.complex128), t.astype(np.complex128), gf.astype(np.float64), geom)
    with plan_for(pwf, geom, batch) as plan:
        gp, gt = plan.vjp(dev(psi), dev(t), dev(gf))
        gp, gt = gp.cpu().numpy(), gt.cpu().numpy()
    assert rel_l2(gp, gp_exp) <= GRAD_TOL
    assert rel_l2(gt, gt_exp) <= GRAD_TOL


def _solve_case(w, batch, ny=None, nx=None):
    geom = geometry(w, ny, nx)
    psi_true, t = blob_batch(w, batch, ny, nx)
    t = to_c64(t)
    y = to_f32(measurement(psi_true, t.astype(np.complex128), geom, w.photons, w.config))
    return geom, t, y


@pytest.mark.parametrize("w,batch", [(W1, 1), (W2, 1)], ids=["blob128_coherent_50it", "blob512_iotf_100it"])
def test_solve_parity(pwf, w, batch):
    geom, t, y = _solve_case(w, batch)
    ref = [O.solve(y[b].astype(np.float64), t.astype(np.complex128), geom, w.n_iter) for b in range(batch)]
    psi = torch.zeros((batch, w.ny, w.nx), dtype=torch.complex64, device="cuda")
    with plan_for(pwf, geom, batch) as plan:
        iters, loss = plan.solve(dev(y), dev(t), psi, w.n_iter)
    got = psi.cpu().numpy()
    for b in range(batch):
        assert iters[b] == w.n_iter
        assert phase_rms(got[b], ref[b].psi) <= PHASE_TOL
        assert abs(loss[b] - ref[b].losses[-1]) <= 1e-3 * ref[b].losses[-1]


def test_step_matches_solve_and_oracle_losses(pwf):
    w = W2
    geom, t, y = _solve_case(w, 2, 128, 128)
    n = 12
    ref = [O.solve(y[b].astype(np.float64), t.astype(np.complex128), geom, n) for b in range(2)]
    with plan_for(pwf, geom, 2) as plan:
        a = torch.zeros((2, 128, 128), dtype=torch.complex64, device="cuda")
        plan.solve(dev(y), dev(t), a, n)
        b = torch.zeros_like(a)
        plan.reset()
        for k in range(n):
            plan.step(dev(y), dev(t), b)
            loss, corr, iters, active = plan.read()
            for p in range(2):
                assert abs(loss[p] - ref[p].losses[k]) <= 1e-4 * ref[p].losses[k]
                assert abs(corr[p] - ref[p].correlations[k]) <= 1e-6
        assert list(iters) == [n, n]
    assert rel_l2(b.cpu().numpy(), a.cpu().numpy()) <= 1e-5


def test_device_side_loop_counts_and_replays(pwf):
    # The graph path runs the whole loop on the device (a conditional WHILE
    # node closed by a loop-control kernel): its iteration count follows the
    # limit passed to each solve, and the same captured loop replayed with
    # another limit, or again with the same one, gives the same iterates.
    w = W2
    geom, t, y = _solve_case(w, 2, 128, 128)
    Y, T = dev(y), dev(t)
    with plan_for(pwf, geom, 2, pwf.FLAG_GRAPH) as plan:
        out = {}
        for n in (7, 1, 7, 3):
            psi = torch.zeros((2, 128, 128), dtype=torch.complex64, device="cuda")
            iters, loss = plan.solve(Y, T, psi, n)
            assert list(iters) == [n, n]
            assert "loop=device" in pwf.pwf_plan_describe(plan.handle)
            if n in out:
                assert torch.equal(out[n], psi)
            out[n] = psi
    for n in (1, 3, 7):
        ref = O.solve(y[0].astype(np.float64), t.astype(np.complex128), geom, n)
        assert phase_rms(out[n].cpu().numpy()[0], ref.psi) <= PHASE_TOL


def test_programmatic_launch_changes_no_value(pwf):
    # passes launched with and without programmatic dependent launch run the
    # same arithmetic: the iterates agree bit for bit
    geom, t, y = _solve_case(W2, 2, 128, 128)
    out = []
    for flags in (pwf.FLAG_GRAPH, pwf.FLAG_GRAPH | pwf.FLAG_NO_PDL):   # untuned shapes in both plans
        with plan_for(pwf, geom, 2, flags | pwf.FLAG_NO_TUNE) as plan:
            psi = torch.zeros((2, 128, 128), dtype=torch.complex64, device="cuda")
            plan.solve(dev(y), dev(t), psi, 9)
            out.append(psi.cpu())
    assert torch.equal(out[0], out[1])


def test_plain_baseline_matches_fused(pwf):
    w = W2
    geom, t, y = _solve_case(w, 2, 128, 128)
    out = []
    for flags in (0, pwf.FLAG_PLAIN):
        with plan_for(pwf, geom, 2, flags) as plan:
            psi = torch.zeros((2, 128, 128), dtype=torch.complex64, device="cuda")
            plan.solve(dev(y), dev(t), psi, 10)
            out.append(psi.cpu().numpy())
    assert rel_l2(out[1], out[0]) <= 1e-5


@pytest.mark.parametrize("flags", [1, 2], ids=["no_precond", "no_reg"])
def test_ablation_flags_match_oracle(pwf, flags):
    w = W2
    geom, t, y = _solve_case(w, 1, 128, 128)
    n = 8
    if flags == 1:
        # Preconditioner off: P^-1 := 1 everywhere (Fig. S3 ablation)
        Pinv = np.ones((128, 128))
        Gamma2 = O.reg_window(geom)
        alpha = geom.alpha
    else:
        Pinv = O.precond_filter(geom)
        Gamma2 = O.reg_window(geom)
        alpha = 0j
    g2 = O.Geometry(**{**geom.__dict__, "alpha": alpha})
    solver = O.PWFSolver(O.SpeckleModel(g2, t.astype(np.complex128)), g2, Pinv, Gamma2)
    psi = solver.solve(y[0].astype(np.float64), n).psi
    with plan_for(pwf, geom, 1, flags) as plan:
        p = torch.zeros((1, 128, 128), dtype=torch.complex64, device="cuda")
        plan.solve(dev(y), dev(t), p, n)
    assert phase_rms(p.cpu().numpy()[0], psi) <= PHASE_TOL


def test_stopping_rule_matches_oracle(pwf):
    # The stopping iteration is an integer that floating point decides: the
    # threshold is put halfway across the widest step of the oracle's
    # correlation sequence (iterations 10..80, a step of 2e-6), so that the
    # FP32 path, whose correlations follow the oracle's far closer than the
    # 1e-6 half-step, must stop at exactly the same iteration; the retrieved
    # phase is then compared as usual.
    w = W1
    geom, t, y = _solve_case(w, 1)
    y64, t128 = y[0].astype(np.float64), t.astype(np.complex128)
    free = O.solve(y64, t128, geom, 80)
    c = np.array(free.correlations)
    best_k, margin = None, 0.0
    for k in range(10, len(c)):
        m = c[k] - np.max(c[:k])
        if m > margin:
            best_k, margin = k, m
    assert best_k is not None and margin >= 1e-6, margin
    tol = float(np.max(c[:best_k]) + margin / 2)
    ref = O.solve(y64, t128, geom, 200, corr_tol=tol)
    assert ref.iterations == best_k + 1
    with plan_for(pwf, geom, 1) as plan:
        psi = torch.zeros((1, w.ny, w.nx), dtype=torch.complex64, device="cuda")
        iters, _ = plan.solve(dev(y), dev(t), psi, 200, corr_tol=tol)
    assert int(iters[0]) == ref.iterations
    assert phase_rms(psi.cpu().numpy()[0], ref.psi) <= PHASE_TOL


def test_checkpoint_resume_is_bitwise(pwf):
    w = W2
    geom, t, y = _solve_case(w, 2, 128, 128)
    Y, T = dev(y), dev(t)
    with plan_for(pwf, geom, 2) as plan:
        a = torch.zeros((2, 128, 128), dtype=torch.complex64, device="cuda")
        plan.reset()
        for _ in range(6):
            plan.step(Y, T, a)
        b = torch.zeros_like(a)
        plan.reset()
        for _ in range(3):
            plan.step(Y, T, b)
        blob = pwf.pwf_state_save(plan.handle, plan.state)
        saved_psi = b.clone()
        plan.reset()                                 # wipe the state
        plan.step(Y, T, torch.zeros_like(b))         # and dirty it
        pwf.pwf_state_load(plan.handle, plan.state, blob)
        b.copy_(saved_psi)
        for _ in range(3):
            plan.step(Y, T, b)
        assert torch.equal(a, b)


def test_bad_checkpoint_rejected(pwf):
    geom = geometry(W2, 128, 128)
    with plan_for(pwf, geom, 2) as plan, plan_for(pwf, geometry(W2, 64, 64), 2) as other:
        blob = pwf.pwf_state_save(plan.handle, plan.state)
        with pytest.raises(pwf.PWFError) as e:
            pwf.pwf_state_load(other.handle, other.state, blob)
        assert e.value.status == 6


def test_nonfinite_iterate_reported_in_the_same_iteration(pwf):
    # a step size of 1e30 overflows the first update: the loss (taken at the
    # starting point) is finite, the new iterate is not, and the correlation
    # sums over exp(psi) flag it at once
    geom, t, y = _solve_case(W1, 1)
    g = O.Geometry(**{**geom.__dict__, "eta": 1e30})
    with plan_for(pwf, g, 1) as plan:
        psi = torch.zeros((1, 128, 128), dtype=torch.complex64, device="cuda")
        with pytest.raises(pwf.PWFError) as e:
            plan.solve(dev(y), dev(t), psi, 1)
        assert e.value.status == 5


def test_nonfinite_measurement_reported(pwf):
    geom, t, y = _solve_case(W1, 1)
    y = y.copy()
    y[0, 5, 5] = np.nan
    with plan_for(pwf, geom, 1) as plan:
        psi = torch.zeros((1, 128, 128), dtype=torch.complex64, device="cuda")
        with pytest.raises(pwf.PWFError) as e:
            plan.solve(dev(y), dev(t), psi, 3)
        assert e.value.status == 5


# ----------------------------------------------------------------------------
# batches large enough for the persistent, pipelined column kernel
# (used once a pass has at least two column tiles per SM)
# ----------------------------------------------------------------------------
BIG = [("b64_128_iotf", 64, 128, 128), ("b40_512_iotf", 40, 512, 512), ("b24_768x256_iotf", 24, 768, 256),
       ("b20_256x1536_iotf", 20, 256, 1536)]


@pytest.mark.parametrize("name,batch,ny,nx", BIG, ids=[c[0] for c in BIG])
def test_pipelined_column_passes_sampled(pwf, name, batch, ny, nx):
    w = W2
    geom = geometry(w, ny, nx)
    psi, t = blob_batch(w, batch, ny, nx)
    psi, t = to_c64(psi), to_c64(t)
    y = to_f32(np.clip(1.0 + 0.1 * np.random.default_rng(5).standard_normal((batch, ny, nx)), 0, None))
    with plan_for(pwf, geom, batch) as plan:
        f = plan.forward(dev(psi), dev(t)).cpu().numpy()
        g, L = plan.gradient(dev(psi), dev(t), dev(y))
        g, L = g.cpu().numpy(), L.cpu().numpy()
        p = torch.zeros((batch, ny, nx), dtype=torch.complex64, device="cuda")
        plan.solve(dev(y), dev(t), p, 3)
        p = p.cpu().numpy()
    for b in (0, batch // 2, batch - 1):
        P64, T64 = psi[b].astype(np.complex128), t.astype(np.complex128)
        assert rel_l2(f[b], O.intensity(P64, T64, geom)) <= FWD_TOL
        ge, le = O.wirtinger_gradient(P64, T64, y[b].astype(np.float64), geom)
        assert rel_l2(g[b], ge) <= GRAD_TOL
        assert abs(L[b] - le) <= 1e-5 * le
        ref = O.solve(y[b].astype(np.float64), T64, geom, 3)
        assert phase_rms(p[b], ref.psi) <= PHASE_TOL


# ----------------------------------------------------------------------------
# every column-pass shape the tuner may choose, forced one at a time
# ----------------------------------------------------------------------------
@pytest.mark.parametrize("ny,nx,batch", [(1024, 256, 6), (512, 128, 8), (128, 96, 4), (2048, 64, 2), (768, 128, 3),
                                           (256, 64, 5), (1536, 64, 2)],
                         ids=["1024x256", "512x128", "128x96", "2048x64", "768x128", "256x64", "1536x64"])
def test_every_column_shape_matches_oracle(pwf, ny, nx, batch):
    w = W2
    geom = geometry(w, ny, nx)
    psi, t = blob_batch(w, batch, ny, nx)
    psi, t = to_c64(psi), to_c64(t)
    y = to_f32(np.clip(1.0 + 0.1 * np.random.default_rng(6).standard_normal((batch, ny, nx)), 0, None))
    P64, T64 = psi.astype(np.complex128), t.astype(np.complex128)
    b = batch - 1
    f_ref = O.intensity(P64[b], T64, geom)
    g_ref, _ = O.wirtinger_gradient(P64[b], T64, y[b].astype(np.float64), geom)
    ref3 = O.solve(y[b].astype(np.float64), T64, geom, 2)
    with plan_for(pwf, geom, batch) as plan:
        nshape = max(pwf.pwf_plan_column_shapes(plan.handle, op) for op in range(7))
        assert nshape >= 3
        for k in range(nshape):
            for op in range(7):
                n_op = pwf.pwf_plan_column_shapes(plan.handle, op)
                pwf.pwf_plan_set_column_shape(plan.handle, op, min(k, n_op - 1))
            f = plan.forward(dev(psi), dev(t)).cpu().numpy()
            g, _ = plan.gradient(dev(psi), dev(t), dev(y))
            p = torch.zeros((batch, ny, nx), dtype=torch.complex64, device="cuda")
            plan.solve(dev(y), dev(t), p, 2)
            assert rel_l2(f[b], f_ref) <= FWD_TOL, (k, pwf.pwf_plan_describe(plan.handle))
            assert rel_l2(g.cpu().numpy()[b], g_ref) <= GRAD_TOL, (k, pwf.pwf_plan_describe(plan.handle))
            assert phase_rms(p.cpu().numpy()[b], ref3.psi) <= PHASE_TOL, (k, pwf.pwf_plan_describe(plan.handle))


# ----------------------------------------------------------------------------
# full-size tomographic series (180 x 1024^2), sampled projections
# ----------------------------------------------------------------------------
def tomo_inputs(n_angles=180, n=1024):
    w = S.WORKLOADS["tomo180x1024_iotf"]
    ph = S.ellipsoid_phantom(S.rng_for(w.config, 0), size=n)
    xd, yd = S.detector_grid(n, n, xp=torch)
    xd, yd = xd.cuda(), yd.cuda()
    psi = torch.empty((n_angles, n, n), dtype=torch.complex128, device="cuda")
    for i, ang in enumerate(S.tomo_angles(n_angles)):
        re, im = S.ellipsoid_projection(ph, float(ang), xd, yd, w.wavelength_m)
        psi[i] = torch.complex(re, im)
    t = S.diffuser(n, n, S.rng_for(w.config, 99))
    return w, psi, t


@pytest.fixture(scope="module")
def tomo(pwf):
    return tomo_inputs()


def test_full_size_tomo_forward_sampled(pwf, tomo):
    w, psi, t = tomo
    geom = geometry(w)
    psi32 = psi.to(torch.complex64)
    t32 = to_c64(t)
    with plan_for(pwf, geom, psi.shape[0]) as plan:
        f = plan.forward(psi32, dev(t32))
    for b in (0, 97, 179):
        expect = O.intensity(psi32[b].cpu().numpy().astype(np.complex128), t32.astype(np.complex128), geom)
        assert rel_l2(f[b].cpu().numpy(), expect) <= FWD_TOL


# ----------------------------------------------------------------------------
# packed residual passes (two real rows per complex row, bins 0..nx/2)
# ----------------------------------------------------------------------------
@pytest.mark.parametrize("ny,nx,batch", [(1024, 256, 3), (128, 96, 4), (768, 128, 3), (64, 16, 4), (2048, 64, 2),
                                           (1536, 64, 2)],
                         ids=["1024x256", "128x96", "768x128", "64x16", "2048x64", "1536x64"])
def test_packed_residual_matches_unpacked_and_oracle(pwf, ny, nx, batch):
    # The default IOTF iteration carries |v|^2 and the residual as packed real
    # rows and filters only bins kx = 0..nx/2 (the rest are their conjugates);
    # PWF_FLAG_UNPACKED_RESID runs the full complex form. Both against the
    # oracle: the first iteration's loss (the Parseval sum over the packed
    # residual, weight 2 for mirrored bins) to 1e-5, the losses and iterates
    # after 4 iterations to the usual tolerances. The 4-iteration iterates of
    # the two FP32 forms are also held to the same order of error against the
    # FP64 ones: their error there is low-frequency rounding that the
    # preconditioner amplifies by up to ny nx, one realization per rounding
    # order, so the two differ by small factors; a slip in the packing (a lost
    # half, a wrong conjugate, a mis-weighted bin) is O(1).
    w = W2
    geom, t, y = _solve_case(w, batch, ny, nx)
    n = 4
    ref = [O.solve(y[b].astype(np.float64), t.astype(np.complex128), geom, n) for b in range(batch)]
    out = {}
    for flags in (0, pwf.FLAG_UNPACKED_RESID):
        with plan_for(pwf, geom, batch, flags) as plan:
            desc = pwf.pwf_plan_describe(plan.handle)
            first = torch.zeros((batch, ny, nx), dtype=torch.complex64, device="cuda")
            plan.reset()
            plan.step(dev(y), dev(t), first)
            loss1, _, _, _ = plan.read()
            psi = torch.zeros((batch, ny, nx), dtype=torch.complex64, device="cuda")
            iters, loss = plan.solve(dev(y), dev(t), psi, n)
        out[flags] = psi.cpu().numpy()
        for b in range(batch):
            assert abs(loss1[b] - ref[b].losses[0]) <= 1e-5 * ref[b].losses[0], (flags, b, desc)
            assert iters[b] == n
            assert phase_rms(out[flags][b], ref[b].psi) <= PHASE_TOL, (flags, b, desc)
            assert abs(loss[b] - ref[b].losses[-1]) <= 1e-4 * ref[b].losses[-1], (flags, b, desc)
    exact = np.stack([r.psi for r in ref])
    err_pk = rel_l2(out[0], exact)
    err_un = rel_l2(out[pwf.FLAG_UNPACKED_RESID], exact)
    assert err_pk <= 4.0 * max(err_un, 5e-5) and err_un <= 4.0 * max(err_pk, 5e-5), (err_pk, err_un)
