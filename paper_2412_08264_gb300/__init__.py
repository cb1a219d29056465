"""GB300-native hypergradients for bilevel imaging with recycled Krylov solves.

Implements the data-parallel hot path of Ehrhardt, Gazzola and Scott,
"Efficient gradient-based methods for bilevel learning via recycling Krylov
subspaces": lower-level solve, recycled CG on the Hessian system with Ritz or
Ritz-generalized-singular-vector recycling and the hypergradient-error
stopping rule, and the J w contraction, batched over training pairs on one GPU.

  api.Problem      binding of the C ABI (include/bl.h), one batch of pairs
  strategy.parse   Table 1 acronyms (e.g. "RGen-L(R)-NSC")
  autograd         torch.autograd.Function with the recycled solve as backward
  synth            seeded synthetic inputs (no arithmetic of the method)
"""
from .strategy import Strategy, parse  # noqa: F401

__all__ = ["Strategy", "parse"]
