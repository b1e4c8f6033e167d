"""pwf_forward_noalloc: the forward model for callers that cannot allocate
device memory, checked against pwf_forward (which works through a plan that
owns allocated workspace) and against the FP64 oracle.

Some callers cannot let a library call cudaMalloc: processes whose device
memory is owned by another allocator or reserved up front, and latency-bound
code that cannot take the device-wide synchronisation cudaMalloc/cudaFree
imply. pwf_forward_noalloc keeps its scratch field and tables in fixed
file-scope device arrays instead. This file runs last (pytest collects it
after the other test files) and passes both alone and after them.
"""
import numpy as np
import pytest

from oracle import pwf_oracle as O
from paper_2503_20146_gb300 import synth as S

from _cases import blob_batch, geometry, rel_l2, to_c64

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

FWD_TOL = 1e-5  # same forward-intensity tolerance as the other parity tests
LIMIT = 1 << 21  # batch * ny * nx the fixed scratch holds


@pytest.fixture(scope="module")
def P():
    from paper_2503_20146_gb300 import _build
    _build.build()
    from paper_2503_20146_gb300 import pwf
    pwf.load()
    return pwf


def _desc(P, geom, batch, n_modes=0):
    return P.PlanDesc(batch, geom.ny, geom.nx, geom.pixel, geom.wavelength, geom.L1, geom.L2, geom.xcoh,
                      geom.ycoh, geom.gamma, geom.alpha.real, geom.alpha.imag, geom.eta,
                      n_modes=n_modes, mode_sigma_px=2.0 if n_modes > 1 else 0.0)


# (workload, batch, ny, nx, x_coh override): partial coherence and coherent,
# rectangular grids, radix-3 lengths, the 2048-point twiddle tables, and a
# problem of exactly the scratch limit
CASES = [(S.WORKLOADS["blob512_iotf"], 2, 256, 256, None),
         (S.WORKLOADS["blob128_coherent"], 3, 96, 128, 0.0),
         (S.WORKLOADS["blob512_iotf"], 1, 768, 768, None),
         (S.WORKLOADS["blob512_iotf"], 1, 1536, 1024, None),
         (S.WORKLOADS["blob512_iotf"], 1, 1024, 2048, None)]


def _inputs(w, batch, ny, nx, xcoh):
    geom = geometry(w, ny, nx, xcoh=xcoh)
    psi, t = blob_batch(w, batch, ny, nx)
    return geom, psi, t


@pytest.mark.parametrize("case", range(len(CASES)), ids=[f"{b}x{ny}x{nx}" for _, b, ny, nx, _ in CASES])
def test_noalloc_forward_matches_pwf_forward_on_two_calls(P, case):
    w, batch, ny, nx, xcoh = CASES[case]
    assert batch * ny * nx <= LIMIT
    geom, psi, t = _inputs(w, batch, ny, nx, xcoh)
    psi = torch.from_numpy(to_c64(psi)).cuda()
    t = torch.from_numpy(to_c64(t)).cuda()
    desc = _desc(P, geom, batch)
    with P.Plan(desc) as plan:
        ref = plan.forward(psi, t).cpu().numpy()
    outs = []
    for _ in range(2):             # two calls in a row share (and rewrite) the arrays
        f = torch.empty((batch, ny, nx), dtype=torch.float32, device="cuda")
        P.pwf_forward_noalloc(desc, psi, t, f)
        torch.cuda.synchronize()
        outs.append(f.cpu().numpy())
    for f in outs:
        assert rel_l2(f, ref) <= FWD_TOL
    assert np.array_equal(outs[0], outs[1])


def test_noalloc_forward_matches_the_oracle(P):
    w, batch, ny, nx, xcoh = CASES[0]
    geom, psi, t = _inputs(w, batch, ny, nx, xcoh)
    psi32, t32 = to_c64(psi), to_c64(t)
    f = torch.empty((batch, ny, nx), dtype=torch.float32, device="cuda")
    P.pwf_forward_noalloc(_desc(P, geom, batch), torch.from_numpy(psi32).cuda(), torch.from_numpy(t32).cuda(), f)
    torch.cuda.synchronize()
    expect = O.intensity_batch(psi32.astype(np.complex128), t32.astype(np.complex128), geom)
    assert rel_l2(f.cpu().numpy(), expect) <= FWD_TOL


def test_noalloc_call_leaves_free_device_memory_unchanged(P):
    w, batch, ny, nx, xcoh = CASES[0]
    geom, psi, t = _inputs(w, batch, ny, nx, xcoh)
    psi = torch.from_numpy(to_c64(psi)).cuda()
    t = torch.from_numpy(to_c64(t)).cuda()
    f = torch.empty((batch, ny, nx), dtype=torch.float32, device="cuda")
    desc = _desc(P, geom, batch)
    P.pwf_forward_noalloc(desc, psi, t, f)       # first call: one-time set-up, kernels loaded
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    P.pwf_forward_noalloc(desc, psi, t, f)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0


def test_noalloc_rejects_sizes_beyond_its_scratch(P):
    w = S.WORKLOADS["blob512_iotf"]
    geom = geometry(w, 1024, 1024)
    psi = torch.zeros((3, 1024, 1024), dtype=torch.complex64, device="cuda")
    t = torch.ones((1024, 1024), dtype=torch.complex64, device="cuda")
    f = torch.empty((3, 1024, 1024), dtype=torch.float32, device="cuda")
    with pytest.raises(P.PWFError) as e:
        P.pwf_forward_noalloc(_desc(P, geom, 3), psi, t, f)   # 3 x 1024^2 > 2^21 elements
    assert e.value.status == 2


def test_noalloc_rejects_source_mode_descriptors(P):
    w = S.WORKLOADS["blob512_iotf"]
    geom = geometry(w, 128, 128)
    psi = torch.zeros((1, 128, 128), dtype=torch.complex64, device="cuda")
    t = torch.ones((128, 128), dtype=torch.complex64, device="cuda")
    f = torch.empty((1, 128, 128), dtype=torch.float32, device="cuda")
    for n_modes, status in ((9, 2), (25, 2), (7, 1), (-1, 1)):
        with pytest.raises(P.PWFError) as e:
            P.pwf_forward_noalloc(_desc(P, geom, 1, n_modes), psi, t, f)
        assert e.value.status == status, n_modes
