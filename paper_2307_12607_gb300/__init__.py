"""ExWarp's warping fast path (arXiv 2307.12607) on GB300: CUDA kernels for sm_103a behind a C ABI.

``paper_2307_12607_gb300.binding`` holds the Python face of the C entry points (same names as include/exw.h);
they are re-exported here lazily, so importing ``paper_2307_12607_gb300.scenes`` (the seeded input generator)
does not import torch.  ``paper_2307_12607_gb300.autograd`` wraps stage (b) and its adjoint for training losses.
"""


def __getattr__(name):
    if name.startswith("exw_") or name in ("ExwError", "workspace", "F32", "F16", "FLAG_NO_FILL", "MASK_EMPTY",
                                           "MASK_CRACK", "KEY_EMPTY", "OP_MOTION_BOUNDS", "OP_FILL_HOLES",
                                           "OP_EXTRAPOLATE", "OP_WARP_BACKWARD", "lib"):
        from . import binding
        return getattr(binding, name)
    raise AttributeError(f"module {__name__!r} has no attribute {name!r}")
