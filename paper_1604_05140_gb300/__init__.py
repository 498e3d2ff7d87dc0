"""GB300-native spherical Gauss-Laguerre (SGL) Fourier transform.

The transform (forward, inverse, adjoints; batched, uneven bandlimits) runs in
the CUDA library ``lib/libsgl.so`` behind the C ABI of ``include/sgl.h``;
``sgl`` is its Python binding.  Importing this package does not load the
library; the first call that needs it does, and raises if it was not built.
"""
from .sgl import (  # noqa: F401
    Plan, SGLError, load_library, header_functions,
    sgl_plan, sgl_plan_many, sgl_forward, sgl_inverse, sgl_adjoint, sgl_grid,
    sgl_destroy, sgl_check, sgl_autotune, sgl_tuning, sgl_selftest_wait, sgl_forward_autograd, sgl_inverse_autograd,
    SGL_FP64, SGL_FP32, SGL_TF32X3, SGL_TF32, SGL_BF16X3, SGL_SAMPLES_WEIGHTED, SGL_SAMPLES_PHYSICAL,
    SGL_SAMPLES_REAL, SGL_GRID_LAGUERRE, SGL_GRID_HALF_RANGE_HERMITE, sgl_plan_grid,
    sgl_midpoint, midpoint,
)

__version__ = "0.1"
