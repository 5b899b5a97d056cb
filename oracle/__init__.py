"""Plain FP64 CPU oracle for the MGCNN solver (arXiv 2312.11093).

TEST INFRASTRUCTURE ONLY.  Nothing in the product path may import, call or
execute this package: only `tests/`, `__graft_entry__.smoke()` and the
`cpu_baseline` / `--impl reference` legs of `bench.py` use it.  It shares no
code with the CUDA library (no kernels, headers, helpers or constant tables);
the only common dependency is the seeded input generator module, which holds
none of the method's arithmetic.

Everything is numpy in float64, written for a reader to check against the
paper by eye: no blocking, fusion or reordering beyond the definitions.
Arrays are indexed [j, i] with x = i h, y = j h (y grows with the row index);
multi-channel tensors are [C, n, n] as in PyTorch.

Modules
  grid       level sizes and spacings (Sec. 4.1 level rule)
  operator   5-point discretisations (Sec. 2.5, Eq. convection_diffusion,
             the divergence form of Remark 2.1), coarse operators, dense matrix
  gmg        classical geometric multigrid (Sec. 2.3, Algorithm 1 extended to
             a V-cycle) inside the stationary iteration (Eq. 1)
  convnet    3x3 convolution primitives in PyTorch semantics (Sec. 2.4,
             Eqs. conv / transconv) and their adjoints
  mgcnn      setup phase (Algorithm 2), solve phase (Algorithm 3, Eq.
             heteroresnet), the stationary iteration, and the network weights
             that make the solve phase reproduce GMG exactly
  adjoint    the training loss (Eq. loss) after K unrolled cycles and its
             hand-written FP64 gradient

Parity status: every function is pinned by `tests/test_oracle_*.py` against
closed forms, a dense direct solve, brute-force loops or invariants, except
the learned-network quality, which has no pin (no trained weights exist).
"""
