"""The persistent solver: all iterations of a solve in one cooperative launch
(grid barriers between the passes, every wait bounded), against the FP64
oracle and against the graph replay of the same plan.

* the 128^2 coherent projection for 50 iterations and the 512^2 partially
  coherent one for 100 iterations, phase RMS <= 1e-3 rad against the oracle;
* a batch of 3 projections at 256^2 (reductions per projection);
* the stopping rule (same iteration count as the oracle);
* a wait limit of zero makes the first barrier time out: the call returns
  PWF_ERR_TIMEOUT without hanging, and the next solve on the same plan, with
  the limit restored, is correct;
* which plans take the persistent launch;
* the cluster-resident launch (one thread-block cluster per projection):
  against the oracle, bit for bit against the cooperative launch and across
  cluster sizes, the stopping rule per projection, and its plan rules.
"""
import numpy as np
import pytest

from oracle import pwf_oracle as O
from paper_2503_20146_gb300 import synth as S

from _cases import blob_batch, geometry, measurement, phase_rms, rel_l2, to_c64, to_f32

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

PHASE_TOL = 1e-3
W1 = S.WORKLOADS["blob128_coherent"]
W2 = S.WORKLOADS["blob512_iotf"]
TIMEOUT = 7


@pytest.fixture(scope="module")
def pwf():
    from paper_2503_20146_gb300 import _build
    _build.build()
    from paper_2503_20146_gb300 import pwf as P
    P.load()
    return P


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def desc_for(P, geom, batch, flags=0):
    return P.PlanDesc(batch, geom.ny, geom.nx, geom.pixel, geom.wavelength, geom.L1, geom.L2, geom.xcoh,
                      geom.ycoh, geom.gamma, geom.alpha.real, geom.alpha.imag, geom.eta, flags)


def case(w, batch, n=None):
    geom = geometry(w, n, n)
    psi_true, t = blob_batch(w, batch, n, n)
    t = to_c64(t)
    y = to_f32(measurement(psi_true, t.astype(np.complex128), geom, w.photons, w.config))
    return geom, t, y


@pytest.mark.parametrize("w", [W1, W2], ids=["blob128_coherent_50it", "blob512_iotf_100it"])
def test_persistent_solve_matches_oracle_and_graph(pwf, w):
    geom, t, y = case(w, 1)
    ref = O.solve(y[0].astype(np.float64), t.astype(np.complex128), geom, w.n_iter)
    out = {}
    for flags in (pwf.FLAG_PERSISTENT, pwf.FLAG_GRAPH):
        with pwf.Plan(desc_for(pwf, geom, 1, flags)) as plan:
            assert pwf.pwf_plan_uses_persistent(plan.handle) == (1 if flags == pwf.FLAG_PERSISTENT else 0)
            psi = torch.zeros((1, w.ny, w.nx), dtype=torch.complex64, device="cuda")
            iters, loss = plan.solve(dev(y), dev(t), psi, w.n_iter)
            out[flags] = psi.cpu().numpy()[0]
        assert int(iters[0]) == w.n_iter
        assert phase_rms(out[flags], ref.psi) <= PHASE_TOL
        assert abs(loss[0] - ref.losses[-1]) <= 1e-3 * ref.losses[-1]
    assert phase_rms(out[pwf.FLAG_PERSISTENT], out[pwf.FLAG_GRAPH]) <= PHASE_TOL


def test_persistent_batch_keeps_projections_apart(pwf):
    geom, t, y = case(W2, 3, 256)
    n = 8
    with pwf.Plan(desc_for(pwf, geom, 3, pwf.FLAG_PERSISTENT)) as plan:
        psi = torch.zeros((3, 256, 256), dtype=torch.complex64, device="cuda")
        iters, loss = plan.solve(dev(y), dev(t), psi, n)
        got = psi.cpu().numpy()
    for b in range(3):
        ref = O.solve(y[b].astype(np.float64), t.astype(np.complex128), geom, n)
        assert int(iters[b]) == n
        assert phase_rms(got[b], ref.psi) <= PHASE_TOL
        assert abs(loss[b] - ref.losses[-1]) <= 1e-4 * ref.losses[-1]


def test_persistent_stopping_rule_matches_oracle(pwf):
    # threshold halfway across the widest step of the oracle's correlation
    # sequence, as in the graph-path test, so the decision is unambiguous
    geom, t, y = case(W1, 1)
    y64, t128 = y[0].astype(np.float64), t.astype(np.complex128)
    c = np.array(O.solve(y64, t128, geom, 80).correlations)
    margins = [(c[k] - np.max(c[:k]), k) for k in range(10, len(c))]
    margin, k = max(margins)
    assert margin >= 1e-6
    tol = float(np.max(c[:k]) + margin / 2)
    ref = O.solve(y64, t128, geom, 200, corr_tol=tol)
    with pwf.Plan(desc_for(pwf, geom, 1, pwf.FLAG_PERSISTENT)) as plan:
        psi = torch.zeros((1, W1.ny, W1.nx), dtype=torch.complex64, device="cuda")
        iters, _ = plan.solve(dev(y), dev(t), psi, 200, corr_tol=tol)
    assert int(iters[0]) == ref.iterations == k + 1
    assert phase_rms(psi.cpu().numpy()[0], ref.psi) <= PHASE_TOL


def test_wait_limit_zero_times_out_and_the_plan_recovers(pwf):
    geom, t, y = case(W2, 1, 128)
    n = 5
    ref = O.solve(y[0].astype(np.float64), t.astype(np.complex128), geom, n)
    with pwf.Plan(desc_for(pwf, geom, 1, pwf.FLAG_PERSISTENT)) as plan:
        psi = torch.zeros((1, 128, 128), dtype=torch.complex64, device="cuda")
        pwf.pwf_plan_set_wait_limit(plan.handle, 0)
        with pytest.raises(pwf.PWFError) as e:
            plan.solve(dev(y), dev(t), psi, n)
        assert e.value.status == TIMEOUT
        torch.cuda.synchronize()                    # the context is still usable
        pwf.pwf_plan_set_wait_limit(plan.handle, 1 << 31)
        psi.zero_()
        iters, _ = plan.solve(dev(y), dev(t), psi, n)
        assert int(iters[0]) == n
        assert phase_rms(psi.cpu().numpy()[0], ref.psi) <= PHASE_TOL
        with pytest.raises(pwf.PWFError) as e:
            pwf.pwf_plan_set_wait_limit(plan.handle, -1)
        assert e.value.status == 1


def test_which_plans_take_the_persistent_launch(pwf):
    # by default the graph, except the cluster-resident solver at 128^2 for
    # batches one wave of clusters holds (where it measured faster); the
    # persistent launch on request, for square IOTF/coherent plans of the
    # built sizes only
    expect = [(geometry(W1), 1, 0, 2),
              (geometry(W1), 4, 0, 2),
              (geometry(W1), 64, 0, 0),
              (geometry(W2, 512, 512), 1, 0, 0),
              (geometry(W1), 1, pwf.FLAG_GRAPH, 0),
              (geometry(W1), 1, pwf.FLAG_CHECK_FINITE, 0),
              (geometry(W1), 1, pwf.FLAG_PERSISTENT, 1),
              (geometry(W2, 512, 512), 16, pwf.FLAG_PERSISTENT, 1),
              (geometry(W2, 512, 512), 1, pwf.FLAG_GRAPH, 0)]
    for geom, batch, flags, persistent in expect:
        with pwf.Plan(desc_for(pwf, geom, batch, flags)) as plan:
            assert pwf.pwf_plan_uses_persistent(plan.handle) == persistent, (geom.ny, geom.nx, batch, flags)
    for geom in (geometry(W2, 1024, 1024), geometry(W2, 96, 128)):      # not a built size / not square
        with pytest.raises(pwf.PWFError) as e:
            pwf.Plan(desc_for(pwf, geom, 1, pwf.FLAG_PERSISTENT))
        assert e.value.status == 2
    d = desc_for(pwf, geometry(W2, 512, 512), 1, pwf.FLAG_PERSISTENT | pwf.FLAG_GRAPH)
    with pytest.raises(pwf.PWFError) as e:
        pwf.Plan(d)
    assert e.value.status == 1


# ---------------------------------------------------------------------------
# cluster-resident launch: one thread-block cluster per projection
# ---------------------------------------------------------------------------
def _solve_with(pwf, geom, t, y, n, flags, cluster=None, corr_tol=0.0, sched=None):
    # untuned column shapes (F{y} takes one), so that plans compared bit for bit run the same arithmetic
    with pwf.Plan(desc_for(pwf, geom, y.shape[0], flags | pwf.FLAG_NO_TUNE)) as plan:
        if sched is not None:
            pwf.pwf_plan_set_cluster_schedule(plan.handle, sched)
        if cluster is not None:
            pwf.pwf_plan_set_cluster_size(plan.handle, cluster)
        psi = torch.zeros((y.shape[0], geom.ny, geom.nx), dtype=torch.complex64, device="cuda")
        iters, loss = plan.solve(dev(y), dev(t), psi, n, corr_tol=corr_tol)
        return psi.cpu().numpy(), iters, loss, pwf.pwf_plan_describe(plan.handle)


@pytest.mark.parametrize("w", [W1, W2], ids=["blob128_coherent_50it", "blob512_iotf_100it"])
def test_cluster_solve_matches_oracle_and_persistent(pwf, w):
    # the same passes as the cooperative launch, item for item: psi agrees
    # bit for bit; losses (FP64 sums in another order) to rounding
    geom, t, y = case(w, 1)
    ref = O.solve(y[0].astype(np.float64), t.astype(np.complex128), geom, w.n_iter)
    # the plan's choice of schedule (the alternative at 128^2) against the oracle
    alt, iters_a, loss_a, desc = _solve_with(pwf, geom, t, y, w.n_iter, pwf.FLAG_CLUSTER)
    assert "solver=cluster" in desc
    assert int(iters_a[0]) == w.n_iter
    assert phase_rms(alt[0], ref.psi) <= PHASE_TOL
    assert abs(loss_a[0] - ref.losses[-1]) <= 1e-3 * ref.losses[-1]
    # the default schedule: also bit for bit against the cooperative launch
    got, iters, loss, desc = _solve_with(pwf, geom, t, y, w.n_iter, pwf.FLAG_CLUSTER, sched=0)
    assert int(iters[0]) == w.n_iter
    assert phase_rms(got[0], ref.psi) <= PHASE_TOL
    assert abs(loss[0] - ref.losses[-1]) <= 1e-3 * ref.losses[-1]
    per, _, loss_p, _ = _solve_with(pwf, geom, t, y, w.n_iter, pwf.FLAG_PERSISTENT)
    assert np.array_equal(got, per)
    assert abs(loss[0] - loss_p[0]) <= 1e-9 * loss_p[0]


@pytest.mark.parametrize("sched", [0, 1], ids=["default_schedule", "alternative_schedule"])
def test_cluster_sizes_agree_bitwise(pwf, sched):
    # within one radix schedule set every cluster size computes the same bits;
    # both sets (256 = 16.16 and 4.8.8) against the oracle
    geom, t, y = case(W2, 2, 256)
    n = 6
    out = {}
    for cs in (1, 2, 4, 8, 16):
        try:
            out[cs] = _solve_with(pwf, geom, t, y, n, pwf.FLAG_CLUSTER, cluster=cs, sched=sched)[0]
        except pwf.PWFError as e:      # a shape the device cannot hold
            assert e.status == 2
    assert 1 in out and 8 in out
    for cs, psi in out.items():
        assert np.array_equal(psi, out[1]), cs
    for b in range(2):
        ref = O.solve(y[b].astype(np.float64), t.astype(np.complex128), geom, n)
        assert phase_rms(out[1][b], ref.psi) <= PHASE_TOL


def test_cluster_stopping_rule_matches_oracle(pwf):
    # a batch of two: each cluster applies the rule to its own projection
    geom, t, y = case(W1, 1)
    y64, t128 = y[0].astype(np.float64), t.astype(np.complex128)
    c = np.array(O.solve(y64, t128, geom, 80).correlations)
    margin, k = max((c[k] - np.max(c[:k]), k) for k in range(10, len(c)))
    assert margin >= 1e-6
    tol = float(np.max(c[:k]) + margin / 2)
    ref = O.solve(y64, t128, geom, 200, corr_tol=tol)
    y2 = np.concatenate([y, y])
    got, iters, _, _ = _solve_with(pwf, geom, t, y2, 200, pwf.FLAG_CLUSTER, corr_tol=tol)
    assert [int(i) for i in iters] == [ref.iterations, ref.iterations]
    assert phase_rms(got[0], ref.psi) <= PHASE_TOL
    # one projection capped earlier by a lower limit on a second solve
    few, iters, _, _ = _solve_with(pwf, geom, t, y, 5, pwf.FLAG_CLUSTER, corr_tol=tol)
    assert int(iters[0]) == 5


def test_cluster_plan_rules(pwf):
    g128 = geometry(W1)
    with pwf.Plan(desc_for(pwf, g128, 1, pwf.FLAG_CLUSTER)) as plan:
        assert pwf.pwf_plan_uses_persistent(plan.handle) == 2
        assert pwf.pwf_plan_cluster_size(plan.handle) in (8, 16)   # the largest cluster that fits
        assert pwf.pwf_plan_cluster_schedule(plan.handle) == 1     # 4.4.4.2 built for 128
        assert "cluster_schedule=4.4.4.2" in pwf.pwf_plan_describe(plan.handle)
        with pytest.raises(pwf.PWFError) as e:
            pwf.pwf_plan_set_cluster_schedule(plan.handle, 2)
        assert e.value.status == 1
        for bad in (-1, 17):
            with pytest.raises(pwf.PWFError) as e:
                pwf.pwf_plan_set_cluster_size(plan.handle, bad)
            assert e.value.status == 1
    with pwf.Plan(desc_for(pwf, g128, 1, pwf.FLAG_GRAPH)) as plan:
        assert pwf.pwf_plan_cluster_size(plan.handle) == 0
        with pytest.raises(pwf.PWFError) as e:
            pwf.pwf_plan_set_cluster_size(plan.handle, 2)
        assert e.value.status == 1
    for flags in (pwf.FLAG_CLUSTER | pwf.FLAG_GRAPH, pwf.FLAG_CLUSTER | pwf.FLAG_PERSISTENT):
        with pytest.raises(pwf.PWFError) as e:
            pwf.Plan(desc_for(pwf, g128, 1, flags))
        assert e.value.status == 1
    with pytest.raises(pwf.PWFError) as e:
        pwf.Plan(desc_for(pwf, geometry(W2, 1024, 1024), 1, pwf.FLAG_CLUSTER))
    assert e.value.status == 2
