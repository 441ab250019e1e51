"""FP64 CPU oracle for randomized block-Lanczos PCA (Halko, Martinsson,
Shkolnisky, Tygert, "An algorithm for the principal component analysis of
large data sets").

TEST INFRASTRUCTURE ONLY.  Nothing in the product path (the CUDA library and
its Python binding) imports, calls or links anything in this package; only
the tests, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline leg do.
It shares no code with the CUDA path: the only common module is the seeded
input generator package ``synth``, which holds none of the method's
arithmetic.

Modules
  philox       counter-based RNG (Philox4x32-10) + Box-Muller, used to draw
               the Gaussian test matrix G from a seed (Section 3, Step 1)
  rpca_oracle  the six steps of Section 3 in FP64, streaming A by row blocks
               as in Section 4.2, plus column-mean centering (Section 1)
  estimator    the Appendix power-method estimate p_{j,k}(D) of ||D||_2, the
               error bound of eq. (sort_of_svd) and the largest principal
               angle between two subspaces (the parity metric for U and V)
"""
