"""Plain FP64 CPU oracle of the damped real Chebyshev wave-packet method.

TEST INFRASTRUCTURE ONLY. Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU
baseline legs of ``bench.py`` may import anything from this package. The product
path (the CUDA library and its Python binding) never imports, calls or links it,
and this package never imports the product package.

It restates the method of Roncero & del Mazo-Sevillano, "MADWAVE3" (arXiv
2412.10167) from the paper's equations, written for readability rather than speed:
dense matrices where a definition is a matrix, numpy/scipy routines only as plain
library primitives (matmul, eigh, Gauss-Legendre nodes).

Modules
  units        atomic-unit conversions
  pes          Jacobi geometry, Sato LEPS, two-state diabatic extension (Section 4)
  basis        sine DVR / DST-II, Gauss-Legendre, normalised associated Legendre,
               angular FBR matrices (Section 2.1, items 2-3)
  hamiltonian  the grid Hamiltonian of Eq. (hamiltonian) and its coupled grid
               equations, the Coriolis coupling, spectral bounds and H_s (Section 2.2)
  propagate    damping (Eq. imaginary-potential), initial packet (Eqs.
               initial-collision-wvp, initial-gaussian), the modified Chebyshev
               recursion (Eq. wvp-k), energy projection (Eqs. wvf-chebyshev,
               chebyshev-expansion-constants), incoming amplitude
               (Eq. initial-flux-collisions), total flux (Eq. total-flux),
               reactant-channel projections (Eqs. Chebyshev-products-overlaps,
               S-matrix-from-chebyshev)
  jshift       J-shifting interpolation (Eq. J-shifting-interpolation)
  mlp          FP64 reference MLP forward/backward (surrogate gradient checks)

Parity status: every function here is pinned by a ``-m "not gpu"`` test in
``tests/test_oracle_*.py`` except where its docstring says "parity unpinned".
"""
