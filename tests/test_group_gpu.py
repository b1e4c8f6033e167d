"""Mixed-size batches: plans of different sizes (and coherence models) solved
together from one graph match each plan solved alone and the oracle."""
import dataclasses

import numpy as np
import pytest

from oracle import pwf_oracle as O
from paper_2503_20146_gb300 import synth as S

from _cases import blob_batch, geometry, phase_rms, to_c64, to_f32

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


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


# (ny, nx, batch, n_modes)
CLASSES = [(256, 256, 3, 0), (96, 128, 2, 0), (768, 128, 1, 9), (128, 128, 4, 25)]


def _class_inputs(ny, nx, batch, seed):
    geom = geometry(W2, ny, nx)
    psi_true, t = blob_batch(W2, batch, ny, nx, seed_proj0=seed)
    rng = np.random.default_rng(seed)
    photons = np.exp(rng.uniform(np.log(1e3), np.log(1e5), batch))       # per projection
    f = np.stack([O.intensity(p, t, geom) for p in psi_true])
    y = np.stack([S.poisson_measurement(f[b], photons[b], S.rng_for(5, seed + b)) for b in range(batch)])
    return geom, to_c64(t), to_f32(y)


def test_group_matches_individual_solves_and_oracle(pwf):
    iters = 6
    plans, ys, ts, psis, refs = [], [], [], [], []
    for k, (ny, nx, batch, K) in enumerate(CLASSES):
        geom, t, y = _class_inputs(ny, nx, batch, 10 * k)
        d = pwf.PlanDesc(batch, ny, nx, geom.pixel, geom.wavelength, geom.L1, geom.L2, geom.xcoh, geom.ycoh,
                         geom.gamma, geom.alpha.real, geom.alpha.imag, geom.eta, pwf.FLAG_NO_TUNE, K, 2.0)
        plans.append(pwf.Plan(d))
        ys.append(dev(y))
        ts.append(dev(t))
        psis.append(torch.zeros((batch, ny, nx), dtype=torch.complex64, device="cuda"))
        refs.append((geom, t, y, K, d))
    g = pwf.pwf_group_create(plans)
    try:
        pwf.pwf_group_solve(g, ys, ts, psis, iters)
        torch.cuda.synchronize()
        for k, (geom, t, y, K, d) in enumerate(refs):
            loss, it = pwf.pwf_group_read(g, k, d.batch)
            assert list(it) == [iters] * d.batch
            # the same class solved on its own, through its own graph
            with pwf.Plan(dataclasses.replace(d, flags=d.flags | pwf.FLAG_GRAPH)) as alone:
                p = torch.zeros_like(psis[k])
                alone.solve(ys[k], ts[k], p, iters)
            assert torch.equal(p, psis[k])
            # and the oracle on the last projection of the class
            b = d.batch - 1
            if K > 1:
                ref = O.modal_solve(y[b].astype(np.float64), t.astype(np.complex128), geom,
                                  O.source_modes(geom, K, 2.0), iters)
            else:
                ref = O.solve(y[b].astype(np.float64), t.astype(np.complex128), geom, iters)
            assert phase_rms(psis[k].cpu().numpy()[b], ref.psi) <= 1e-3
    finally:
        pwf.pwf_group_destroy(g)
        for p in plans:
            p.close()


def test_group_chains_large_classes_and_matches_individual_solves(pwf):
    # two classes that fill the GPU on their own (>= 8 Mi pixels: solved one
    # after another in the graph) and one small class on a side branch
    iters = 3
    classes = [(1024, 1024, 8), (2048, 2048, 3), (128, 128, 2)]
    gen = torch.Generator(device="cuda").manual_seed(7)
    plans, ys, ts, psis, descs = [], [], [], [], []
    for ny, nx, batch in classes:
        geom = geometry(W2, ny, nx)
        d = pwf.PlanDesc(batch, ny, nx, geom.pixel, geom.wavelength, geom.L1, geom.L2, geom.xcoh, geom.ycoh,
                         geom.gamma, geom.alpha.real, geom.alpha.imag, geom.eta, pwf.FLAG_NO_TUNE)
        plans.append(pwf.Plan(d))
        ys.append(0.5 + torch.rand((batch, ny, nx), generator=gen, device="cuda"))
        ts.append(dev(to_c64(S.diffuser(ny, nx, S.rng_for(5, ny)))))
        psis.append(torch.zeros((batch, ny, nx), dtype=torch.complex64, device="cuda"))
        descs.append(d)
    g = pwf.pwf_group_create(plans)
    try:
        pwf.pwf_group_solve(g, ys, ts, psis, iters)
        torch.cuda.synchronize()
        for k, d in enumerate(descs):
            with pwf.Plan(dataclasses.replace(d, flags=d.flags | pwf.FLAG_GRAPH)) as alone:
                p = torch.zeros_like(psis[k])
                alone.solve(ys[k], ts[k], p, iters)
            assert torch.equal(p, psis[k]), k
    finally:
        pwf.pwf_group_destroy(g)
        for p in plans:
            p.close()
