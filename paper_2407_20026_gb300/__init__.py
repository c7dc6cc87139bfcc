"""GB300-native differentiable structural FEM hot path (arXiv 2407.20026, JAX-SSO).

The compute path is libsso.so (CUDA for sm_103a, C-ABI in include/sso.h); this
package binds it.  Importing the package does not load the library; the first
call does, and fails loudly if the library has not been built.
"""
from ._lib import SSOError  # noqa: F401

__all__ = ["Model", "Batch", "options", "beam_stiffness", "quad_stiffness", "bsr_spmv",
           "SSOError", "SSOFunction", "kernel_launches"]


def __getattr__(name):
    if name in ("Model", "Batch", "options", "beam_stiffness", "quad_stiffness", "bsr_spmv",
                "kernel_launches"):
        from . import model
        return getattr(model, name)
    if name == "SSOFunction":
        from . import autograd
        return autograd.SSOFunction
    raise AttributeError(name)
