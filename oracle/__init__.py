"""FP64 CPU checker for the bilevel hypergradient path (test infrastructure).

Plain, slow NumPy/SciPy code written from the paper (Ehrhardt, Gazzola,
Scott, "Efficient gradient-based methods for bilevel learning via recycling
Krylov subspaces"), used only by the tests, by ``__graft_entry__.smoke()``
and by the ``cpu_baseline`` / ``--impl reference`` legs of ``bench.py``.
The product path never imports it, and it imports nothing from the product
except the seeded input generator ``paper_2412_08264_gb300.synth`` (which
holds no arithmetic of the method).

Modules
  operators   blur A, correlation filters K_j, forward differences D (Section 5)
  functional  lower-level Phi, gradient, Hessian action, J w (eqs. (1.1), (2.4)-(2.7), (5.1));
              A is the blur or the inpainting mask diag(m) of Section 5.1
  krylov      CG, recycled CG, MINRES, RMINRES (Section 2.2, Algorithm 3, Appendix A)
  recycle     Ritz, harmonic Ritz, Ritz generalized singular vectors, NSC, and the outer and
              inner refreshes (Sections 3, 4; eqs. (3.3), (3.4); Table 1's sizes and sides)
  lbfgs       lower-level L-BFGS with backtracking (Section 5.1)
  bilevel     hypergradient, gradient descent with Armijo backtracking (Algorithms 1, 2), Adam

Parity status: every function is pinned by a test under tests/ against a
property fixed by the mathematics (adjoint identities, finite differences,
dense assembly, closed forms, textbook special cases) or, for Table 1, by
the golden fixture tests/golden/table1_strategies.tsv.  Iteration counts of
the paper's own experiments are not reproducible (its datasets and figures
are absent): parity unpinned for those counts.
"""
