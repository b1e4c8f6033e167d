"""The C-ABI library loads and exports every entry point include/pwf.h declares.

Runs on CPU: no compute call is made. Only argument validation that returns
before any CUDA call is exercised (null descriptors, unsupported sizes).
"""
import ctypes

import pytest

from paper_2503_20146_gb300 import _build, pwf


@pytest.fixture(scope="module")
def lib():
    _build.build()
    return pwf.load()


def test_every_declared_function_is_exported(lib):
    names = pwf.header_functions()
    assert len(names) >= 18
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing


def test_status_strings(lib):
    for code, name in pwf.STATUS.items():
        assert pwf.pwf_status_string(code) == name


def _desc(**kw):
    base = dict(batch=1, ny=128, nx=128, pixel_m=1e-6, wavelength_m=6.2e-11, L1_m=0.1, L2_m=0.4,
                xcoh_m=0.0, ycoh_m=0.0, gamma=1.0, alpha_re=0.1, alpha_im=0.01, eta=1e-3, flags=0,
                stream=None, n_modes=0, mode_sigma_px=0.0)
    base.update(kw)
    return pwf.pwf_plan_desc(**base)


@pytest.mark.parametrize("kw,status", [
    (dict(ny=100), 2),            # not a built transform length
    (dict(nx=4096), 2),
    (dict(batch=0), 1),
    (dict(eta=0.0), 1),
    (dict(pixel_m=-1.0), 1),
    (dict(flags=0x800), 1),        # not a flag
    (dict(flags=0x200 | 0x20), 2),  # scans follow the passes, not a single launch
    (dict(flags=0x80 | 0x40), 1),  # two ways to run pwf_solve
    (dict(flags=0x80 | 0x20), 1),
    (dict(wavelength_m=2e-6), 2),  # evanescent bins at this pixel pitch
    (dict(L2_m=5e3), 2),           # separable-propagator bound exceeded
    (dict(n_modes=4, mode_sigma_px=2.0), 1),   # mode count must be 0, 1, 9 or 25
    (dict(n_modes=9, mode_sigma_px=-1.0), 1),
])
def test_plan_validation_before_any_cuda_call(lib, kw, status):
    plan = ctypes.c_void_p()
    d = _desc(**kw)
    assert lib.pwf_plan_create(ctypes.byref(d), ctypes.byref(plan)) == status
    assert not plan.value


def test_null_arguments(lib):
    plan = ctypes.c_void_p()
    assert lib.pwf_plan_create(None, ctypes.byref(plan)) == 1
    assert lib.pwf_forward(None, None, None, None) == 1
    assert lib.pwf_solve_host(None, None, None, None, 0, 1, 0.0, 0, None, None) == 1
    assert lib.pwf_plan_destroy(None) == 1
    assert lib.pwf_state_bytes(None) == 0


def test_host_buffer_marshalling_checks_dtype_size_and_layout():
    import numpy as np
    torch = pytest.importorskip("torch")
    a = np.zeros((2, 4, 4), np.complex64)
    assert pwf._host_ptr(a, "complex64", 32).value == a.ctypes.data
    t = torch.zeros((2, 4, 4), dtype=torch.float32)
    assert pwf._host_ptr(t, "float32", 32).value == t.data_ptr()
    with pytest.raises(ValueError):
        pwf._host_ptr(a, "float32", 32)                       # dtype
    with pytest.raises(ValueError):
        pwf._host_ptr(a, "complex64", 31)                     # size
    with pytest.raises(ValueError):
        pwf._host_ptr(a[:, :, ::2], "complex64", 16)          # not contiguous
    with pytest.raises(ValueError):
        pwf._host_ptr(t.transpose(1, 2), "float32", 32)
    with pytest.raises(TypeError):
        pwf._host_ptr([0.0] * 4, "float32", 4)


def test_autograd_inputs_are_realigned_by_copy():
    torch = pytest.importorskip("torch")
    from paper_2503_20146_gb300.autograd import _aligned
    base = torch.arange(18, dtype=torch.float32).view(torch.complex64)
    view = base[1:]                                  # starts 8 bytes into the allocation
    assert view.data_ptr() % 16 == 8
    fixed = _aligned(view)
    assert fixed.data_ptr() % 16 == 0 and torch.equal(fixed, view)
    whole = base[:8]
    assert _aligned(whole).data_ptr() == whole.data_ptr()   # aligned input: no copy
    nc = torch.arange(16, dtype=torch.float32).view(4, 4).t()
    assert _aligned(nc).is_contiguous()


def test_every_declared_function_has_a_binding_signature(lib):
    # the binding sets argtypes/restype for exactly the functions the header declares
    names = set(pwf.header_functions())
    typed = {n for n in names if getattr(lib, n).argtypes is not None}
    assert typed == names, sorted(names - typed)
