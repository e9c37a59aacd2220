"""GB300-native Nystrom-accelerated primal LS-SVM ODE solver (arXiv 2510.04094).

The solver lives in the C-ABI library libnys.so (include/nys.h), built for
sm_103a by ``build.build()``.  ``_abi`` exposes its entry points under their
C names; ``api.Batch`` marshals problem dicts and torch tensors onto them;
``api.NysSolve`` wires the adjoint gradient into torch.autograd.
"""
from . import build  # noqa: F401

__all__ = ["build", "load"]


def load():
    """Load libnys.so and return the binding module (raises if the library is missing)."""
    from . import _abi
    _abi.lib()
    return _abi
