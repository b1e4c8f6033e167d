"""pwf_forward_noalloc: the forward model for callers that cannot allocate
device memory, checked against pwf_forward (which works through a plan that
owns allocated workspace).

Some callers cannot let a library call cudaMalloc: processes whose device
memory is owned by another allocator or reserved up front, and latency-bound
code that cannot take the device-wide synchronisation cudaMalloc/cudaFree
imply. pwf_forward_noalloc keeps its scratch field and tables in fixed
file-scope device arrays instead. This file runs last (pytest collects it
after the other test files) and passes both alone and after them.
"""
import ctypes

import numpy as np
import pytest

from paper_2503_20146_gb300 import synth as S

from _cases import blob_batch, geometry, rel_l2, to_c64

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

FWD_TOL = 1e-5  # same forward-intensity tolerance as the other parity tests


@pytest.fixture(scope="module")
def P():
    from paper_2503_20146_gb300 import _build
    _build.build()
    from paper_2503_20146_gb300 import pwf
    pwf.load()
    return pwf


def _desc(P, geom, batch):
    return P.PlanDesc(batch, geom.ny, geom.nx, geom.pixel, geom.wavelength, geom.L1, geom.L2, geom.xcoh,
                      geom.ycoh, geom.gamma, geom.alpha.real, geom.alpha.imag, geom.eta)


def test_noalloc_forward_matches_pwf_forward_on_two_calls(P):
    cases = [(S.WORKLOADS["blob512_iotf"], 2, 256, 256, None),      # partial coherence
             (S.WORKLOADS["blob128_coherent"], 3, 96, 128, 0.0)]    # coherent, rectangular
    for w, batch, ny, nx, xcoh in cases:
        geom = geometry(w, ny, nx, xcoh=xcoh)
        psi, t = blob_batch(w, batch, ny, nx)
        psi = torch.from_numpy(to_c64(psi)).cuda()
        t = torch.from_numpy(to_c64(t)).cuda()
        desc = _desc(P, geom, batch)
        f0 = torch.empty((batch, ny, nx), dtype=torch.float32, device="cuda")
        P.pwf_forward_noalloc(desc, psi, t, f0)
        torch.cuda.synchronize()
        with P.Plan(desc) as plan:
            ref = plan.forward(psi, t)
        assert rel_l2(f0.cpu().numpy(), ref.cpu().numpy()) <= FWD_TOL


def test_noalloc_rejects_sizes_beyond_its_scratch(P):
    w = S.WORKLOADS["blob512_iotf"]
    geom = geometry(w, 1024, 1024)
    psi = torch.zeros((3, 1024, 1024), dtype=torch.complex64, device="cuda")
    t = torch.ones((1024, 1024), dtype=torch.complex64, device="cuda")
    f = torch.empty((3, 1024, 1024), dtype=torch.float32, device="cuda")
    with pytest.raises(P.PWFError) as e:
        P.pwf_forward_noalloc(_desc(P, geom, 3), psi, t, f)   # 3 x 1024^2 > 2^21 elements
    assert e.value.status == 2
