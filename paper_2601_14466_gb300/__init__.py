"""Single-GPU dense SPD solver for GB300 (sm_103a): Cholesky potrf / potrs /
posv with FP64 and mixed-precision (tensor-core + FP64 refinement) paths.

Submodules:
  jmg     -- ctypes binding of libjmg.so (raw C entry points + tensor helpers)
  autograd-- torch.autograd.Function with the hand-written adjoint
  inputs  -- seeded synthetic workloads (no solver arithmetic)

Importing the package does not load the CUDA library; the first call does.
"""

__all__ = ["jmg", "inputs"]


def build(force: bool = False) -> str:
    from . import _build

    return _build.build(force=force)
