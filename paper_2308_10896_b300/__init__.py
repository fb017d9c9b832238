"""Differentiable variance shadow mapping on B300 (sm_103a): CUDA kernels behind
the C ABI of ``include/dsm.h`` and a thin ctypes binding (``dsm``)."""
from .dsm import (Context, DSMFunction, DsmError, Renderer, l2_loss_grad, load_library, render)  # noqa: F401

__all__ = ["Context", "DSMFunction", "DsmError", "Renderer", "l2_loss_grad", "load_library", "render"]
