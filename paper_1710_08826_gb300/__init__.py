"""GB300-native unbinned maximum-likelihood engine (GooFit 2.0 hot path, arXiv:1710.08826).

Layout:
  csrc/        CUDA C++ (sm_103a) kernels and the C ABI of include/goo.h -> libgoo.so
  buildlib.py  in-tree nvcc build of libgoo.so
  goo.py       ctypes binding (argument marshalling only)
  autograd.py  torch.autograd.Function over goo_nll_grad
"""


def build(verbose=False, force=False):
    from .buildlib import build as _build
    return _build(verbose=verbose, force=force)


def load():
    """Import the binding (raises ImportError if libgoo.so has not been built)."""
    from . import goo
    return goo
