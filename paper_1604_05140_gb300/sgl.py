"""Python binding of libsgl (include/sgl.h): argument marshalling only.

Every function named ``sgl_*`` here calls the C function of the same name.
The ``Plan`` class wraps a plan for torch tensors (device memory and streams
come from PyTorch; every step of the transform runs in libsgl's kernels), and
``SGLForward`` / ``SGLInverse`` make the transforms differentiable with the
library's adjoint transforms as backward passes.

The library must have been built (``paper_1604_05140_gb300.build.build()``);
importing the binding without it raises immediately: there is no fallback.
"""
from __future__ import annotations

import ctypes
import os
import re
from typing import Optional, Sequence

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "lib", "libsgl.so")
HEADER = os.path.join(os.path.dirname(_HERE), "include", "sgl.h")

SGL_OK, SGL_ERR_ARG, SGL_ERR_ALLOC, SGL_ERR_CUDA, SGL_ERR_TIMEOUT, SGL_ERR_UNSUPPORTED = range(6)
SGL_FP64, SGL_FP32, SGL_TF32X3, SGL_TF32, SGL_BF16X3, SGL_FP16X3 = 0, 1, 2, 3, 4, 5
SGL_SAMPLES_WEIGHTED, SGL_SAMPLES_PHYSICAL, SGL_SAMPLES_REAL = 0, 1, 2
SGL_GRID_LAGUERRE, SGL_GRID_HALF_RANGE_HERMITE = 0, 1
GRIDS = {"laguerre": SGL_GRID_LAGUERRE, "hermite": SGL_GRID_HALF_RANGE_HERMITE}
SGL_MAX_B = 128

PRECISIONS = {"fp64": SGL_FP64, "fp32": SGL_FP32, "tf32x3": SGL_TF32X3, "tf32": SGL_TF32, "bf16x3": SGL_BF16X3,
              "fp16x3": SGL_FP16X3}
STATUS_NAMES = {0: "SGL_OK", 1: "SGL_ERR_ARG", 2: "SGL_ERR_ALLOC", 3: "SGL_ERR_CUDA",
                4: "SGL_ERR_TIMEOUT", 5: "SGL_ERR_UNSUPPORTED"}


class SGLError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


_lib = None


def load_library():
    """Load libsgl.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(
            f"libsgl.so not found at {LIB_PATH}: build it first with "
            "`python -m paper_1604_05140_gb300.build` (nvcc, sm_103a)")
    lib = ctypes.CDLL(LIB_PATH)
    vp, i32, i64 = ctypes.c_void_p, ctypes.c_int, ctypes.c_int64
    dp = ctypes.POINTER(ctypes.c_double)
    sigs = {
        "sgl_plan": (i32, [ctypes.POINTER(vp), i32, i32, i32, i32]),
        "sgl_plan_grid": (i32, [ctypes.POINTER(vp), i32, i32, i32, i32, i32]),
        "sgl_plan_many": (i32, [ctypes.POINTER(vp), ctypes.POINTER(ctypes.c_int), i32, i32]),
        "sgl_forward": (i32, [vp, vp, vp, vp]),
        "sgl_inverse": (i32, [vp, vp, vp, vp]),
        "sgl_adjoint": (i32, [vp, i32, vp, vp, vp]),
        "sgl_grid": (i32, [vp, i32, dp, dp, dp, dp, dp]),
        "sgl_sample_count": (i64, [vp]),
        "sgl_coeff_count": (i64, [vp]),
        "sgl_sample_offset": (i64, [vp, i32]),
        "sgl_coeff_offset": (i64, [vp, i32]),
        "sgl_num_functions": (i32, [vp]),
        "sgl_bandlimit": (i32, [vp, i32]),
        "sgl_radii": (i32, [vp, i32]),
        "sgl_workspace_bytes": (i64, [vp]),
        "sgl_launches_per_call": (i32, [vp]),
        "sgl_check": (i32, [vp, vp]),
        "sgl_last_error": (ctypes.c_char_p, [vp]),
        "sgl_destroy": (None, [vp]),
        "sgl_version": (ctypes.c_char_p, []),
        "sgl_set_profiling": (i32, [vp, i32]),
        "sgl_stage_times": (i32, [vp, vp, vp]),
        "sgl_stage_name": (ctypes.c_char_p, [i32]),
        "sgl_forward_noalloc": (i32, [i32, i32, vp, vp, vp]),
        "sgl_autotune": (i32, [vp, vp, vp, ctypes.c_char_p, vp]),
        "sgl_tuning": (ctypes.c_char_p, [vp]),
        "sgl_selftest_wait": (i32, [i64, ctypes.POINTER(ctypes.c_int)]),
        "sgl_midpoint": (i32, [i32, i32, ctypes.c_double, i32, i32, vp, vp, vp]),
        "sgl_set_dlt": (i32, [vp, i32]),
        "sgl_set_graphs": (i32, [vp, i32]),
        "sgl_graph_count": (i32, [vp]),
    }
    for name, (res, args) in sigs.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def header_functions(path: str = HEADER):
    """Names of the functions declared in include/sgl.h."""
    with open(path) as fh:
        text = fh.read()
    return sorted(set(re.findall(r"^\s*[A-Za-z_][\w\s\*]*?\b(sgl_\w+)\s*\(", text, re.M)))


def _check(st: int, plan=None):
    if st != SGL_OK:
        lib = load_library()
        msg = lib.sgl_last_error(plan)
        raise SGLError(st, msg.decode() if msg else "")


# ---------------------------------------------------------------------------
# C ABI, same names
# ---------------------------------------------------------------------------

def sgl_plan(B: int, batch: int = 1, prec: int = SGL_FP64, samples: int = SGL_SAMPLES_WEIGHTED):
    lib = load_library()
    h = ctypes.c_void_p()
    _check(lib.sgl_plan(ctypes.byref(h), int(B), int(batch), int(prec), int(samples)))
    return h


def sgl_plan_grid(B: int, batch: int = 1, prec: int = SGL_FP64, samples: int = SGL_SAMPLES_WEIGHTED,
                  grid: int = SGL_GRID_LAGUERRE):
    lib = load_library()
    h = ctypes.c_void_p()
    _check(lib.sgl_plan_grid(ctypes.byref(h), int(B), int(batch), int(prec), int(samples), int(grid)))
    return h


def sgl_plan_many(Bs: Sequence[int], prec: int = SGL_TF32X3):
    lib = load_library()
    arr = (ctypes.c_int * len(Bs))(*[int(b) for b in Bs])
    h = ctypes.c_void_p()
    _check(lib.sgl_plan_many(ctypes.byref(h), arr, len(Bs), int(prec)))
    return h


def sgl_forward(plan, samples_ptr: int, coeffs_ptr: int, stream: int = 0):
    _check(load_library().sgl_forward(plan, samples_ptr, coeffs_ptr, stream), plan)


def sgl_inverse(plan, coeffs_ptr: int, samples_ptr: int, stream: int = 0):
    _check(load_library().sgl_inverse(plan, coeffs_ptr, samples_ptr, stream), plan)


def sgl_adjoint(plan, of_inverse: int, in_ptr: int, out_ptr: int, stream: int = 0):
    _check(load_library().sgl_adjoint(plan, int(of_inverse), in_ptr, out_ptr, stream), plan)


def sgl_grid(plan, fn: int = 0):
    lib = load_library()
    B = lib.sgl_bandlimit(plan, fn)
    if B < 1:
        raise SGLError(SGL_ERR_ARG, "function index out of range")
    R = lib.sgl_radii(plan, fn)
    r, th, ph, wr, wt = (np.zeros(n) for n in (R, 2 * B, 2 * B, R, 2 * B))
    P = ctypes.POINTER(ctypes.c_double)
    _check(lib.sgl_grid(plan, fn, *(a.ctypes.data_as(P) for a in (r, th, ph, wr, wt))), plan)
    return r, th, ph, wr, wt


def sgl_destroy(plan):
    load_library().sgl_destroy(plan)


def sgl_autotune(plan, samples_ptr: int, coeffs_ptr: int, cache_path: Optional[str] = None, stream: int = 0):
    path = cache_path.encode() if cache_path else None
    _check(load_library().sgl_autotune(plan, samples_ptr, coeffs_ptr, path, stream), plan)


def sgl_tuning(plan) -> str:
    return load_library().sgl_tuning(plan).decode()


def sgl_selftest_wait(limit_ns: int = 50_000_000) -> bool:
    """True when a bounded device-side wait that can never be satisfied gave
    up after limit_ns and its kernel ended (sgl_selftest_wait)."""
    flag = ctypes.c_int(0)
    _check(load_library().sgl_selftest_wait(int(limit_ns), ctypes.byref(flag)))
    return bool(flag.value)


def sgl_midpoint(B: int, M: int, L: float, batch: int, prec: int, f_ptr: int, coeffs_ptr: int, stream: int = 0):
    _check(load_library().sgl_midpoint(int(B), int(M), float(L), int(batch), int(prec), f_ptr, coeffs_ptr, stream))


def midpoint(f, B: int, L: float, out=None):
    """Midpoint-rule coefficients (sgl_midpoint) of physical samples f of
    shape (batch, M, M, M) on the cell midpoints of [-L, L]^3: a CUDA
    complex128 (FP64) or complex64 (FP32) tensor."""
    import torch
    if not (isinstance(f, torch.Tensor) and f.is_cuda and f.dim() == 4 and f.is_contiguous()):
        raise TypeError("f must be a contiguous CUDA tensor of shape (batch, M, M, M)")
    if f.dtype not in (torch.complex128, torch.complex64):
        raise TypeError("f must be complex128 or complex64")
    batch, M = f.shape[0], f.shape[1]
    if f.shape[2] != M or f.shape[3] != M:
        raise ValueError("f must have M cells on every axis")
    n = B * (B + 1) * (2 * B + 1) // 6
    if out is None:
        out = torch.empty((batch, n), dtype=f.dtype, device=f.device)
    prec = SGL_FP64 if f.dtype == torch.complex128 else SGL_FP32
    sgl_midpoint(B, M, L, batch, prec, f.data_ptr(), out.data_ptr(), torch.cuda.current_stream(f.device).cuda_stream)
    return out


def sgl_check(plan, stream: int = 0):
    _check(load_library().sgl_check(plan, stream), plan)


def sgl_sample_count(plan) -> int:
    return load_library().sgl_sample_count(plan)


def sgl_coeff_count(plan) -> int:
    return load_library().sgl_coeff_count(plan)


def sgl_sample_offset(plan, fn: int) -> int:
    return load_library().sgl_sample_offset(plan, int(fn))


def sgl_coeff_offset(plan, fn: int) -> int:
    return load_library().sgl_coeff_offset(plan, int(fn))


def sgl_num_functions(plan) -> int:
    return load_library().sgl_num_functions(plan)


def sgl_bandlimit(plan, fn: int) -> int:
    return load_library().sgl_bandlimit(plan, int(fn))


def sgl_radii(plan, fn: int) -> int:
    return load_library().sgl_radii(plan, int(fn))


def sgl_workspace_bytes(plan) -> int:
    return load_library().sgl_workspace_bytes(plan)


def sgl_launches_per_call(plan) -> int:
    return load_library().sgl_launches_per_call(plan)


def sgl_last_error(plan=None) -> str:
    msg = load_library().sgl_last_error(plan)
    return msg.decode() if msg else ""


def sgl_version() -> str:
    return load_library().sgl_version().decode()


SGL_NUM_STAGES = 6


def sgl_set_profiling(plan, enable: bool):
    _check(load_library().sgl_set_profiling(plan, int(bool(enable))), plan)


def sgl_set_graphs(plan, enable: bool):
    _check(load_library().sgl_set_graphs(plan, int(bool(enable))), plan)


def sgl_graph_count(plan) -> int:
    return load_library().sgl_graph_count(plan)


def sgl_stage_times(plan):
    """{stage name: (summed device ms, launches)} since profiling was enabled."""
    lib = load_library()
    ms = (ctypes.c_double * SGL_NUM_STAGES)()
    n = (ctypes.c_int64 * SGL_NUM_STAGES)()
    _check(lib.sgl_stage_times(plan, ms, n), plan)
    return {sgl_stage_name(k): (ms[k], int(n[k])) for k in range(SGL_NUM_STAGES)}


def sgl_stage_name(stage: int) -> str:
    name = load_library().sgl_stage_name(int(stage))
    return name.decode() if name else ""


def sgl_forward_noalloc(B: int, batch: int, samples_ptr: int, coeffs_ptr: int, stream: int = 0):
    _check(load_library().sgl_forward_noalloc(int(B), int(batch), samples_ptr, coeffs_ptr, stream))


def sgl_set_dlt(plan, seminaive: bool):
    _check(load_library().sgl_set_dlt(plan, int(bool(seminaive))), plan)


# ---------------------------------------------------------------------------
# torch-facing plan
# ---------------------------------------------------------------------------

class Plan:
    """A libsgl plan operating on torch tensors.

    Single-bandlimit plans take samples of shape (batch, B, 2B, 2B) and
    coefficients of shape (batch, Omega); plans over uneven bandlimits
    (``Plan.many``) take flat 1-D tensors packed at ``sample_offset(f)`` /
    ``coeff_offset(f)``.  Tensors may live on the GPU (used in place, launch
    on the current torch stream) or in host memory (staged by the library).
    ``samples="real"`` makes a plan of real functions: real sample tensors
    (``sample_dtype``), complex coefficients, and the inverse returns the real
    part (SGL_SAMPLES_REAL in sgl.h).  ``grid="hermite"`` samples on the
    paper's own grid of 2B half-range Gauss-Hermite radii (every precision
    and sample convention): samples of shape (batch, 2B, 2B, 2B).
    """

    def __init__(self, B: Optional[int] = None, batch: int = 1, precision: str = "fp64",
                 samples: str = "weighted", grid: str = "laguerre", _handle=None, _Bs=None):
        import torch  # noqa: F401  (device memory and streams)
        self.lib = load_library()
        self.prec = PRECISIONS[precision]
        self.precision = precision
        self.real = samples == "real"
        self.grid_kind = grid
        if _handle is not None:
            self.handle = _handle
            self.Bs = list(_Bs)
            self.B = None
            self.batch = len(self.Bs)
        else:
            conv = {"weighted": SGL_SAMPLES_WEIGHTED, "physical": SGL_SAMPLES_PHYSICAL,
                    "real": SGL_SAMPLES_REAL}[samples]
            self.handle = sgl_plan_grid(B, batch, self.prec, conv, GRIDS[grid])
            self.B = int(B)
            self.batch = int(batch)
            self.Bs = [self.B] * self.batch
        self.n_samples = self.lib.sgl_sample_count(self.handle)
        self.n_coeffs = self.lib.sgl_coeff_count(self.handle)

    @classmethod
    def many(cls, Bs: Sequence[int], precision: str = "tf32x3") -> "Plan":
        h = sgl_plan_many(Bs, PRECISIONS[precision])
        return cls(precision=precision, _handle=h, _Bs=Bs)

    # shapes and types ----------------------------------------------------
    @property
    def dtype(self):
        import torch
        return torch.complex128 if self.prec == SGL_FP64 else torch.complex64

    @property
    def sample_dtype(self):
        """Element type of the sample tensors: the coefficient type, or its
        real counterpart for plans of real functions (samples="real")."""
        import torch
        if self.real:
            return torch.float64 if self.prec == SGL_FP64 else torch.float32
        return self.dtype

    @property
    def radii(self) -> int:
        """Radial nodes per function: B, or 2B on the paper's grid."""
        return 2 * self.B if self.grid_kind == "hermite" else self.B

    @property
    def sample_shape(self):
        if self.B is None:
            return (self.n_samples,)
        return (self.batch, self.radii, 2 * self.B, 2 * self.B)

    @property
    def coeff_shape(self):
        if self.B is None:
            return (self.n_coeffs,)
        return (self.batch, self.n_coeffs // self.batch)

    def sample_offset(self, f: int) -> int:
        return self.lib.sgl_sample_offset(self.handle, f)

    def coeff_offset(self, f: int) -> int:
        return self.lib.sgl_coeff_offset(self.handle, f)

    @property
    def workspace_bytes(self) -> int:
        return self.lib.sgl_workspace_bytes(self.handle)

    @property
    def launches_per_call(self) -> int:
        return self.lib.sgl_launches_per_call(self.handle)

    def grid(self, fn: int = 0):
        return sgl_grid(self.handle, fn)

    # execution ------------------------------------------------------------
    def _prep(self, t, numel: int, name: str, dtype=None):
        import torch
        dtype = self.dtype if dtype is None else dtype
        if not isinstance(t, torch.Tensor):
            raise TypeError(f"{name} must be a torch tensor")
        if t.dtype != dtype:
            raise TypeError(f"{name} must be {dtype}, got {t.dtype}")
        if t.numel() != numel:
            raise ValueError(f"{name} has {t.numel()} elements, expected {numel}")
        if not t.is_contiguous():
            raise ValueError(f"{name} must be contiguous")
        return t

    def _stream(self, *tensors) -> int:
        import torch
        for t in tensors:
            if t.is_cuda:
                return torch.cuda.current_stream(t.device).cuda_stream
        return 0

    def _out(self, like, shape, out, dtype=None):
        import torch
        if out is None:
            out = torch.empty(shape, dtype=self.dtype if dtype is None else dtype, device=like.device,
                              pin_memory=(not like.is_cuda and torch.cuda.is_available()))
        return out

    def forward(self, samples, out=None):
        """Coefficients of the samples (sgl_forward)."""
        self._prep(samples, self.n_samples, "samples", self.sample_dtype)
        out = self._out(samples, self.coeff_shape, out)
        self._prep(out, self.n_coeffs, "out")
        sgl_forward(self.handle, samples.data_ptr(), out.data_ptr(), self._stream(samples, out))
        return out

    def inverse(self, coeffs, out=None):
        """Samples of the function with these coefficients (sgl_inverse)."""
        self._prep(coeffs, self.n_coeffs, "coeffs")
        out = self._out(coeffs, self.sample_shape, out, self.sample_dtype)
        self._prep(out, self.n_samples, "out", self.sample_dtype)
        sgl_inverse(self.handle, coeffs.data_ptr(), out.data_ptr(), self._stream(coeffs, out))
        return out

    def adjoint(self, x, of_inverse: bool, out=None):
        """Hermitian adjoint of the forward map (of_inverse=False, coefficients
        -> samples) or of the inverse map (of_inverse=True, samples ->
        coefficients), sgl_adjoint."""
        if of_inverse:
            self._prep(x, self.n_samples, "x", self.sample_dtype)
            out = self._out(x, self.coeff_shape, out)
            self._prep(out, self.n_coeffs, "out")
        else:
            self._prep(x, self.n_coeffs, "x")
            out = self._out(x, self.sample_shape, out, self.sample_dtype)
            self._prep(out, self.n_samples, "out", self.sample_dtype)
        sgl_adjoint(self.handle, int(bool(of_inverse)), x.data_ptr(), out.data_ptr(), self._stream(x, out))
        return out

    def set_graphs(self, enable: bool = True) -> "Plan":
        """Replay this plan's device-buffer calls through CUDA graphs of its
        own (sgl_set_graphs); returns the plan."""
        sgl_set_graphs(self.handle, enable)
        return self

    @property
    def graph_count(self) -> int:
        return int(self.lib.sgl_graph_count(self.handle))

    def autotune(self, cache: Optional[str] = None, samples=None, coeffs=None) -> str:
        """Choose the plan's launch configuration by timing it (sgl_autotune).
        samples / coeffs are device scratch tensors of the plan's shapes
        (allocated here when None; their contents are overwritten).  Returns
        the configuration text (sgl_tuning)."""
        import torch
        dev = torch.device("cuda", torch.cuda.current_device())
        if samples is None:
            samples = torch.empty(self.sample_shape, dtype=self.sample_dtype, device=dev)
        if coeffs is None:
            coeffs = torch.empty(self.coeff_shape, dtype=self.dtype, device=dev)
        self._prep(samples, self.n_samples, "samples", self.sample_dtype)
        self._prep(coeffs, self.n_coeffs, "coeffs")
        sgl_autotune(self.handle, samples.data_ptr(), coeffs.data_ptr(), cache, self._stream(samples, coeffs))
        return self.tuning

    def set_dlt(self, seminaive: bool):
        """Forward Legendre sums directly (False) or by the seminaive
        algorithm (True); FP64/FP32 plans (sgl_set_dlt)."""
        _check(self.lib.sgl_set_dlt(self.handle, int(bool(seminaive))), self.handle)

    @property
    def tuning(self) -> str:
        return sgl_tuning(self.handle)

    def check(self):
        import torch
        sgl_check(self.handle, torch.cuda.current_stream().cuda_stream if torch.cuda.is_available() else 0)

    def close(self):
        if getattr(self, "handle", None) is not None:
            sgl_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ---------------------------------------------------------------------------
# autograd
# ---------------------------------------------------------------------------

_AUTOGRAD = None


def _autograd_classes():
    global _AUTOGRAD
    if _AUTOGRAD is not None:
        return _AUTOGRAD
    import torch

    class SGLForward(torch.autograd.Function):
        """coeffs = forward(samples); backward: the adjoint of the forward map.
        PyTorch's complex gradients are conjugate-Wirtinger, so the
        vector-Jacobian product of a linear map is its Hermitian adjoint."""

        @staticmethod
        def forward(ctx, samples, plan):
            ctx.plan = plan
            return plan.forward(samples.contiguous())

        @staticmethod
        def backward(ctx, grad):
            return ctx.plan.adjoint(grad.contiguous(), of_inverse=False), None

    class SGLInverse(torch.autograd.Function):
        """samples = inverse(coeffs); backward: the adjoint of the inverse map."""

        @staticmethod
        def forward(ctx, coeffs, plan):
            ctx.plan = plan
            return plan.inverse(coeffs.contiguous())

        @staticmethod
        def backward(ctx, grad):
            return ctx.plan.adjoint(grad.contiguous(), of_inverse=True), None

    _AUTOGRAD = (SGLForward, SGLInverse)
    return _AUTOGRAD


def sgl_forward_autograd(samples, plan):
    return _autograd_classes()[0].apply(samples, plan)


def sgl_inverse_autograd(coeffs, plan):
    return _autograd_classes()[1].apply(coeffs, plan)
