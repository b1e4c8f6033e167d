"""Thin Python binding of the C ABI in include/pwf.h (argument marshalling only).

Every function here has the name of the C entry point it calls and does no
arithmetic of its own: device tensors (torch, CUDA) are passed by pointer,
and all work runs in libpwf's kernels on the tensors' current CUDA stream.
There is no CPU fallback: if libpwf.so has not been built, or no GPU is
present, calls raise.
"""
from __future__ import annotations

import ctypes
import os
import re
from dataclasses import dataclass

_PKG = os.path.dirname(os.path.abspath(__file__))
_LIB_PATH = os.path.join(_PKG, "lib", "libpwf.so")
_HEADER = os.path.join(os.path.dirname(_PKG), "include", "pwf.h")

FLAG_NO_PRECOND = 0x1
FLAG_NO_REG = 0x2
FLAG_PLAIN = 0x4
FLAG_NO_TUNE = 0x8
FLAG_PERSISTENT = 0x20
FLAG_GRAPH = 0x40
FLAG_CLUSTER = 0x80
FLAG_NO_PDL = 0x100
FLAG_CHECK_FINITE = 0x200
FLAG_UNPACKED_RESID = 0x400

STATUS = {0: "PWF_OK", 1: "PWF_ERR_INVALID_ARG", 2: "PWF_ERR_UNSUPPORTED", 3: "PWF_ERR_NOMEM",
          4: "PWF_ERR_CUDA", 5: "PWF_ERR_NONFINITE", 6: "PWF_ERR_STATE", 7: "PWF_ERR_TIMEOUT",
          8: "PWF_ERR_BOUNDS"}

SIZES = (16, 32, 64, 96, 128, 256, 512, 768, 1024, 1536, 2048)


class PWFError(RuntimeError):
    def __init__(self, status: int, where: str, detail: str = ""):
        self.status = status
        super().__init__(f"{where}: {STATUS.get(status, status)}" + (f" ({detail})" if detail else ""))


class pwf_plan_desc(ctypes.Structure):
    _fields_ = [
        ("batch", ctypes.c_int32), ("ny", ctypes.c_int32), ("nx", ctypes.c_int32),
        ("pixel_m", ctypes.c_double), ("wavelength_m", ctypes.c_double),
        ("L1_m", ctypes.c_double), ("L2_m", ctypes.c_double),
        ("xcoh_m", ctypes.c_double), ("ycoh_m", ctypes.c_double),
        ("gamma", ctypes.c_double), ("alpha_re", ctypes.c_double), ("alpha_im", ctypes.c_double),
        ("eta", ctypes.c_double), ("flags", ctypes.c_uint32), ("stream", ctypes.c_void_p),
        ("n_modes", ctypes.c_int32), ("mode_sigma_px", ctypes.c_double),
    ]


_lib = None
_P = ctypes.c_void_p


def header_functions():
    """Names of the functions declared in include/pwf.h."""
    with open(_HEADER) as fh:
        text = fh.read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(pwf_[a-z_0-9]+)\s*\(", text)))


def library_path() -> str:
    return _LIB_PATH


def load(path: str | None = None):
    """Loads libpwf.so (built by paper_2503_20146_gb300._build.build())."""
    global _lib
    if _lib is not None:
        return _lib
    _lib = open_library(path or _LIB_PATH)
    return _lib


def open_library(path: str):
    """A separately loaded build of the library (for instance the
    bounds-checked one), with the same signatures; the module's own calls keep
    using the library load() returns."""
    if not os.path.exists(path):
        raise RuntimeError(f"libpwf.so is not built ({path}); run __graft_entry__.build()")
    lib = ctypes.CDLL(path)
    i32, f64, sz = ctypes.c_int32, ctypes.c_double, ctypes.c_size_t
    sig = {
        "pwf_plan_create": ([ctypes.POINTER(pwf_plan_desc), ctypes.POINTER(_P)], i32),
        "pwf_plan_destroy": ([_P], i32),
        "pwf_plan_set_stream": ([_P, _P], i32),
        "pwf_plan_workspace_bytes": ([_P], sz),
        "pwf_forward": ([_P, _P, _P, _P], i32),
        "pwf_gradient": ([_P, _P, _P, _P, _P, _P], i32),
        "pwf_forward_vjp": ([_P, _P, _P, _P, _P, _P], i32),
        "pwf_state_create": ([_P, ctypes.POINTER(_P)], i32),
        "pwf_state_destroy": ([_P], i32),
        "pwf_state_reset": ([_P, _P], i32),
        "pwf_step": ([_P, _P, _P, _P, _P, f64], i32),
        "pwf_state_read": ([_P, _P, _P, _P, _P, _P], i32),
        "pwf_solve": ([_P, _P, _P, _P, i32, f64, _P, _P], i32),
        "pwf_state_bytes": ([_P], sz),
        "pwf_state_save": ([_P, _P, _P, sz], i32),
        "pwf_state_load": ([_P, _P, _P, sz], i32),
        "pwf_status_string": ([i32], ctypes.c_char_p),
        "pwf_plan_last_error": ([_P], ctypes.c_char_p),
        "pwf_plan_launch_count": ([_P], ctypes.c_longlong),
        "pwf_profile_iteration": ([_P, _P, _P, _P, i32, _P, _P, _P], i32),
        "pwf_forward_noalloc": ([ctypes.POINTER(pwf_plan_desc), _P, _P, _P], i32),
        "pwf_plan_describe": ([_P, ctypes.c_char_p, sz], sz),
        "pwf_plan_column_shapes": ([_P, i32], i32),
        "pwf_plan_set_column_shape": ([_P, i32, i32], i32),
        "pwf_group_create": ([_P, i32, ctypes.POINTER(_P)], i32),
        "pwf_group_destroy": ([_P], i32),
        "pwf_group_solve": ([_P, _P, _P, _P, _P, i32, f64], i32),
        "pwf_group_read": ([_P, i32, _P, _P], i32),
        "pwf_solve_joint": ([_P, _P, _P, _P, i32, f64, _P, _P], i32),
        "pwf_solve_host": ([_P, _P, _P, _P, i32, i32, f64, i32, _P, _P], i32),
        "pwf_fbp_workspace_bytes": ([i32, i32, i32], ctypes.c_size_t),
        "pwf_fbp": ([_P, i32, i32, i32, ctypes.POINTER(f64), f64, f64, _P, _P, ctypes.c_size_t, _P], i32),
        "pwf_calibrate_coherence": ([_P, _P, i32, ctypes.POINTER(f64), ctypes.POINTER(f64)], i32),
        "pwf_diffuser_from_reference": ([_P, _P, f64, _P], i32),
        "pwf_plan_set_wait_limit": ([_P, ctypes.c_int64], i32),
        "pwf_plan_uses_persistent": ([_P], i32),
        "pwf_plan_set_cluster_size": ([_P, i32], i32),
        "pwf_plan_cluster_size": ([_P], i32),
        "pwf_plan_set_cluster_schedule": ([_P, i32], i32),
        "pwf_plan_cluster_schedule": ([_P], i32),
        "pwf_debug_fail_alloc": ([i32], None),
        "pwf_debug_overrun": ([_P], i32),
    }
    for name, (args, res) in sig.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = res
    return lib


# ----------------------------------------------------------------------------
# helpers (marshalling)
# ----------------------------------------------------------------------------
def _ptr(x):
    if x is None:
        return None
    import torch
    if not isinstance(x, torch.Tensor):
        raise TypeError("expected a torch.Tensor")
    if not x.is_cuda:
        raise ValueError("libpwf takes CUDA device tensors")
    if not x.is_contiguous():
        raise ValueError("tensor must be contiguous")
    return ctypes.c_void_p(x.data_ptr())


def _host_ptr(x, dtype: str, numel: int):
    """Pointer to a contiguous HOST array (torch CPU tensor or numpy array) of
    `numel` elements of `dtype` ("float32" or "complex64")."""
    import numpy as np
    if isinstance(x, np.ndarray):
        if x.dtype != np.dtype(dtype) or not x.flags.c_contiguous or x.size != numel:
            raise ValueError(f"expected a C-contiguous {dtype} numpy array of {numel} elements")
        return ctypes.c_void_p(x.ctypes.data)
    import torch
    if not isinstance(x, torch.Tensor) or x.is_cuda:
        raise TypeError("expected a host (CPU) torch.Tensor or numpy array")
    if x.dtype != getattr(torch, dtype) or not x.is_contiguous() or x.numel() != numel:
        raise ValueError(f"expected a contiguous {dtype} tensor of {numel} elements")
    return ctypes.c_void_p(x.data_ptr())


def _stream_ptr():
    import torch
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


def _check(status: int, where: str, plan=None):
    if status != 0:
        detail = ""
        if plan is not None and plan.value:
            detail = (_lib.pwf_plan_last_error(plan) or b"").decode()
        raise PWFError(status, where, detail)


# ----------------------------------------------------------------------------
# entry points, same names as the C ABI
# ----------------------------------------------------------------------------
@dataclass
class PlanDesc:
    batch: int
    ny: int
    nx: int
    pixel_m: float
    wavelength_m: float
    L1_m: float
    L2_m: float
    xcoh_m: float = 0.0
    ycoh_m: float = 0.0
    gamma: float = 1.0
    alpha_re: float = 0.1
    alpha_im: float = 0.01
    eta: float = 1.0
    flags: int = 0
    n_modes: int = 0
    mode_sigma_px: float = 0.0


def _desc_struct(desc: PlanDesc) -> pwf_plan_desc:
    return pwf_plan_desc(desc.batch, desc.ny, desc.nx, desc.pixel_m, desc.wavelength_m, desc.L1_m, desc.L2_m,
                         desc.xcoh_m, desc.ycoh_m, desc.gamma, desc.alpha_re, desc.alpha_im, desc.eta,
                         desc.flags, _stream_ptr(), desc.n_modes, desc.mode_sigma_px)


def pwf_plan_create(desc: PlanDesc):
    lib = load()
    d = _desc_struct(desc)
    plan = ctypes.c_void_p()
    _check(lib.pwf_plan_create(ctypes.byref(d), ctypes.byref(plan)), "pwf_plan_create")
    return plan


def pwf_plan_destroy(plan):
    _check(load().pwf_plan_destroy(plan), "pwf_plan_destroy")


def pwf_plan_workspace_bytes(plan) -> int:
    return int(load().pwf_plan_workspace_bytes(plan))


def _on_current_stream(plan):
    _check(load().pwf_plan_set_stream(plan, _stream_ptr()), "pwf_plan_set_stream", plan)


def pwf_forward(plan, psi, t, f):
    _on_current_stream(plan)
    _check(load().pwf_forward(plan, _ptr(psi), _ptr(t), _ptr(f)), "pwf_forward", plan)


def pwf_forward_noalloc(desc: "PlanDesc", psi, t, f):
    """Forward model without any device allocation by the library (scratch in
    fixed device arrays); for callers that cannot allocate. Runs on the current
    torch stream."""
    d = _desc_struct(desc)
    _check(load().pwf_forward_noalloc(ctypes.byref(d), _ptr(psi), _ptr(t), _ptr(f)), "pwf_forward_noalloc")


def pwf_plan_set_wait_limit(plan, cycles: int):
    """Longest wait of one grid barrier of the persistent solver (SM cycles)."""
    _check(load().pwf_plan_set_wait_limit(plan, int(cycles)), "pwf_plan_set_wait_limit", plan)


def pwf_plan_uses_persistent(plan) -> int:
    return int(load().pwf_plan_uses_persistent(plan))


def pwf_plan_set_cluster_size(plan, ctas: int):
    """CTAs per cluster of a cluster-resident plan (0: the default)."""
    _check(load().pwf_plan_set_cluster_size(plan, int(ctas)), "pwf_plan_set_cluster_size", plan)


def pwf_plan_cluster_size(plan) -> int:
    return int(load().pwf_plan_cluster_size(plan))


def pwf_plan_set_cluster_schedule(plan, sched: int):
    """Radix schedule set of a cluster-resident plan (0, 1, or -1 for the plan's choice)."""
    _check(load().pwf_plan_set_cluster_schedule(plan, int(sched)), "pwf_plan_set_cluster_schedule", plan)


def pwf_plan_cluster_schedule(plan) -> int:
    return int(load().pwf_plan_cluster_schedule(plan))


def pwf_debug_fail_alloc(after: int):
    """Make the device allocation `after` allocations from now fail (< 0: off)."""
    load().pwf_debug_fail_alloc(int(after))


def pwf_gradient(plan, psi, t, y, g, loss=None):
    _on_current_stream(plan)
    _check(load().pwf_gradient(plan, _ptr(psi), _ptr(t), _ptr(y), _ptr(g), _ptr(loss)), "pwf_gradient", plan)


def pwf_forward_vjp(plan, psi, t, grad_f, grad_psi=None, grad_t=None):
    _on_current_stream(plan)
    _check(load().pwf_forward_vjp(plan, _ptr(psi), _ptr(t), _ptr(grad_f), _ptr(grad_psi), _ptr(grad_t)),
           "pwf_forward_vjp", plan)


def pwf_state_create(plan):
    st = ctypes.c_void_p()
    _on_current_stream(plan)
    _check(load().pwf_state_create(plan, ctypes.byref(st)), "pwf_state_create", plan)
    return st


def pwf_state_destroy(state):
    _check(load().pwf_state_destroy(state), "pwf_state_destroy")


def pwf_state_reset(plan, state):
    _on_current_stream(plan)
    _check(load().pwf_state_reset(plan, state), "pwf_state_reset", plan)


def pwf_step(plan, state, y, t, psi, corr_tol: float = 0.0):
    _on_current_stream(plan)
    _check(load().pwf_step(plan, state, _ptr(y), _ptr(t), _ptr(psi), float(corr_tol)), "pwf_step", plan)


def pwf_state_read(plan, state, batch: int):
    """Returns (loss, corr, iters, active) as Python lists of length batch."""
    import numpy as np
    loss = np.zeros(batch, np.float64)
    corr = np.zeros(batch, np.float64)
    iters = np.zeros(batch, np.int32)
    active = np.zeros(batch, np.int32)
    _on_current_stream(plan)
    _check(load().pwf_state_read(plan, state, loss.ctypes.data_as(_P), corr.ctypes.data_as(_P),
                                 iters.ctypes.data_as(_P), active.ctypes.data_as(_P)), "pwf_state_read", plan)
    return loss, corr, iters, active


def pwf_solve(plan, y, t, psi, max_iter: int, corr_tol: float = 0.0, batch: int | None = None):
    """Runs Algorithm S1 on psi in place. With ``batch`` given, returns
    (iters, loss) numpy arrays read back from the device."""
    import numpy as np
    _on_current_stream(plan)
    it = loss = None
    if batch is not None:
        it = np.zeros(batch, np.int32)
        loss = np.zeros(batch, np.float64)
    _check(load().pwf_solve(plan, _ptr(y), _ptr(t), _ptr(psi), int(max_iter), float(corr_tol),
                            None if it is None else it.ctypes.data_as(_P),
                            None if loss is None else loss.ctypes.data_as(_P)), "pwf_solve", plan)
    return (it, loss) if batch is not None else None


def pwf_solve_host(plan, desc: "PlanDesc", y, t, psi, max_iter: int, corr_tol: float = 0.0,
                   psi_is_input: bool = True, chunk: int = 0):
    """Algorithm S1 on host buffers (torch CPU tensors, ideally pinned, or numpy
    arrays): psi is read (psi_is_input) and written in place. Chunks of the
    batch stream through the device with the copies overlapping the solve.
    Returns (iters, loss) numpy arrays."""
    import numpy as np
    B, n = desc.batch, desc.ny * desc.nx
    it = np.zeros(B, np.int32)
    loss = np.zeros(B, np.float64)
    _on_current_stream(plan)
    _check(load().pwf_solve_host(plan, _host_ptr(y, "float32", B * n), _host_ptr(t, "complex64", n),
                                 _host_ptr(psi, "complex64", B * n), int(bool(psi_is_input)), int(max_iter),
                                 float(corr_tol), int(chunk), it.ctypes.data_as(_P), loss.ctypes.data_as(_P)),
           "pwf_solve_host", plan)
    return it, loss


def pwf_solve_joint(plan, y, t, psi, max_iter: int, eta_t: float, batch: int | None = None):
    """Algorithm S1 with the shared diffuser t refined in place after every
    iteration (fixed iteration count). With ``batch`` given, returns (iters, loss)."""
    import numpy as np
    _on_current_stream(plan)
    it = loss = None
    if batch is not None:
        it = np.zeros(batch, np.int32)
        loss = np.zeros(batch, np.float64)
    _check(load().pwf_solve_joint(plan, _ptr(y), _ptr(t), _ptr(psi), int(max_iter), float(eta_t),
                                  None if it is None else it.ctypes.data_as(_P),
                                  None if loss is None else loss.ctypes.data_as(_P)), "pwf_solve_joint", plan)
    return (it, loss) if batch is not None else None


def pwf_state_bytes(state) -> int:
    return int(load().pwf_state_bytes(state))


def pwf_state_save(plan, state) -> bytes:
    n = pwf_state_bytes(state)
    buf = ctypes.create_string_buffer(n)
    _on_current_stream(plan)
    _check(load().pwf_state_save(plan, state, buf, n), "pwf_state_save", plan)
    return buf.raw


def pwf_state_load(plan, state, data: bytes):
    buf = ctypes.create_string_buffer(data, len(data))
    _on_current_stream(plan)
    _check(load().pwf_state_load(plan, state, buf, len(data)), "pwf_state_load", plan)


MAX_PASSES = 256


def pwf_plan_launch_count(plan) -> int:
    return int(load().pwf_plan_launch_count(plan))


def pwf_profile_iteration(plan, y, t, psi, iters: int):
    """Returns [(pass name, mean milliseconds)] for one fused iteration."""
    ms = (ctypes.c_float * MAX_PASSES)()
    names = (ctypes.c_char_p * MAX_PASSES)()
    n = ctypes.c_int32()
    _on_current_stream(plan)
    _check(load().pwf_profile_iteration(plan, _ptr(y), _ptr(t), _ptr(psi), int(iters), ms, names,
                                        ctypes.byref(n)), "pwf_profile_iteration", plan)
    return [(names[i].decode(), float(ms[i])) for i in range(n.value)]


def pwf_plan_describe(plan) -> str:
    n = int(load().pwf_plan_describe(plan, None, 0))
    buf = ctypes.create_string_buffer(max(n, 1))
    load().pwf_plan_describe(plan, buf, n)
    return buf.value.decode()


def pwf_plan_column_shapes(plan, pass_index: int) -> int:
    return int(load().pwf_plan_column_shapes(plan, int(pass_index)))


def pwf_plan_set_column_shape(plan, pass_index: int, shape: int):
    _check(load().pwf_plan_set_column_shape(plan, int(pass_index), int(shape)), "pwf_plan_set_column_shape", plan)


def pwf_group_create(plans):
    arr = (_P * len(plans))(*[p.handle if hasattr(p, "handle") else p for p in plans])
    g = ctypes.c_void_p()
    _check(load().pwf_group_create(arr, len(plans), ctypes.byref(g)), "pwf_group_create")
    return g


def pwf_group_destroy(group):
    _check(load().pwf_group_destroy(group), "pwf_group_destroy")


def pwf_group_solve(group, ys, ts, psis, max_iter: int, corr_tol: float = 0.0):
    n = len(ys)
    yp = (_P * n)(*[_ptr(y).value for y in ys])
    tp = (_P * n)(*[_ptr(t).value for t in ts])
    pp = (_P * n)(*[_ptr(p).value for p in psis])
    _check(load().pwf_group_solve(group, _stream_ptr(), yp, tp, pp, int(max_iter), float(corr_tol)),
           "pwf_group_solve")


def pwf_group_read(group, index: int, batch: int):
    import numpy as np
    loss = np.zeros(batch, np.float64)
    iters = np.zeros(batch, np.int32)
    _check(load().pwf_group_read(group, int(index), loss.ctypes.data_as(_P), iters.ctypes.data_as(_P)),
           "pwf_group_read")
    return loss, iters


def pwf_calibrate_coherence(plan, I_ref, max_lag: int):
    """(x_coh, y_coh) in metres from the reference speckle I_ref (float32 [ny][nx])."""
    xc, yc = ctypes.c_double(), ctypes.c_double()
    _on_current_stream(plan)
    _check(load().pwf_calibrate_coherence(plan, _ptr(I_ref), int(max_lag), ctypes.byref(xc), ctypes.byref(yc)),
           "pwf_calibrate_coherence", plan)
    return xc.value, yc.value


def pwf_diffuser_from_reference(plan, I_ref, wiener_eps: float, t_out):
    _on_current_stream(plan)
    _check(load().pwf_diffuser_from_reference(plan, _ptr(I_ref), float(wiener_eps), _ptr(t_out)),
           "pwf_diffuser_from_reference", plan)


def pwf_fbp_workspace_bytes(n_angles: int, ny: int, nx: int) -> int:
    return int(load().pwf_fbp_workspace_bytes(int(n_angles), int(ny), int(nx)))


def pwf_fbp(psi, angles_rad, wavelength_m: float, voxel_m: float, vol=None, workspace=None):
    """beta + i delta [ny][nx][nx] (complex64, device) from psi [n_angles][ny][nx]."""
    import torch
    n_angles, ny, nx = psi.shape
    if vol is None:
        vol = torch.empty((ny, nx, nx), dtype=torch.complex64, device=psi.device)
    need = pwf_fbp_workspace_bytes(n_angles, ny, nx)
    if workspace is None:
        workspace = torch.empty(max(need, 1), dtype=torch.uint8, device=psi.device)
    ang = (ctypes.c_double * n_angles)(*[float(a) for a in angles_rad])
    _check(load().pwf_fbp(_ptr(psi), n_angles, ny, nx, ang, float(wavelength_m), float(voxel_m), _ptr(vol),
                          _ptr(workspace), workspace.numel() * workspace.element_size(), _stream_ptr()),
           "pwf_fbp")
    return vol


def pwf_status_string(status: int) -> str:
    return load().pwf_status_string(int(status)).decode()


def pwf_plan_last_error(plan) -> str:
    return (load().pwf_plan_last_error(plan) or b"").decode()


# ----------------------------------------------------------------------------
# convenience: an owning plan object
# ----------------------------------------------------------------------------
class Plan:
    """Owns a pwf_plan (and lazily a pwf_state); methods call the entry points."""

    def __init__(self, desc: PlanDesc):
        self.desc = desc
        self.handle = pwf_plan_create(desc)
        self._state = None

    def close(self):
        if self._state is not None:
            pwf_state_destroy(self._state)
            self._state = None
        if self.handle is not None and self.handle.value:
            pwf_plan_destroy(self.handle)
        self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    @property
    def state(self):
        if self._state is None:
            self._state = pwf_state_create(self.handle)
        return self._state

    def forward(self, psi, t, f=None):
        import torch
        if f is None:
            f = torch.empty(psi.shape, dtype=torch.float32, device=psi.device)
        pwf_forward(self.handle, psi, t, f)
        return f

    def gradient(self, psi, t, y, g=None, loss=None):
        import torch
        if g is None:
            g = torch.empty_like(psi)
        if loss is None:
            loss = torch.empty(self.desc.batch, dtype=torch.float64, device=psi.device)
        pwf_gradient(self.handle, psi, t, y, g, loss)
        return g, loss

    def vjp(self, psi, t, grad_f, want_psi=True, want_t=True):
        import torch
        gp = torch.empty_like(psi) if want_psi else None
        gt = torch.empty_like(t) if want_t else None
        pwf_forward_vjp(self.handle, psi, t, grad_f, gp, gt)
        return gp, gt

    def solve(self, y, t, psi, max_iter, corr_tol=0.0, read_back=True):
        return pwf_solve(self.handle, y, t, psi, max_iter, corr_tol, self.desc.batch if read_back else None)

    def solve_host(self, y, t, psi, max_iter, corr_tol=0.0, psi_is_input=True, chunk=0):
        return pwf_solve_host(self.handle, self.desc, y, t, psi, max_iter, corr_tol, psi_is_input, chunk)

    def solve_joint(self, y, t, psi, max_iter, eta_t, read_back=True):
        return pwf_solve_joint(self.handle, y, t, psi, max_iter, eta_t, self.desc.batch if read_back else None)

    def step(self, y, t, psi, corr_tol=0.0):
        pwf_step(self.handle, self.state, y, t, psi, corr_tol)

    def reset(self):
        pwf_state_reset(self.handle, self.state)

    def calibrate_coherence(self, I_ref, max_lag=3):
        return pwf_calibrate_coherence(self.handle, I_ref, max_lag)

    def diffuser_from_reference(self, I_ref, wiener_eps, t_out=None):
        import torch
        if t_out is None:
            t_out = torch.empty(I_ref.shape, dtype=torch.complex64, device=I_ref.device)
        pwf_diffuser_from_reference(self.handle, I_ref, wiener_eps, t_out)
        return t_out

    def read(self):
        return pwf_state_read(self.handle, self.state, self.desc.batch)
