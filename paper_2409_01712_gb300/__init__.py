"""GB300-native mixed-precision kernel ridge regression for multivariate GWAS.

The compute path is libkrr.so (hand-written CUDA for sm_103a, C ABI in
include/krr.h); this package only marshals arguments (``KRR``) and draws
seeded synthetic inputs (``inputs``).
"""
from . import inputs  # noqa: F401
from .autograd import held_out_loss  # noqa: F401
from .krr import KRR, KRRBatch, KRRError, load_library  # noqa: F401

__all__ = ["KRR", "KRRBatch", "KRRError", "held_out_loss", "inputs", "load_library"]
