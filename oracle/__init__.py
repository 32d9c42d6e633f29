"""Plain, slow, FP64 CPU oracle of the divide-and-conquer CheFSI pass (arXiv 2609.13115).

TEST INFRASTRUCTURE ONLY.  Only the test suite, the package's `smoke()` self-check
and the CPU-baseline leg of the benchmark may import or run anything in this
package.  The product path (the CUDA library and its binding) never calls it and
shares no code with it; the two meet only through the seeded inputs of `synth`.

Every function follows a passage of the paper (cited by section / equation) or a
reading of it where the paper is silent; the readings are listed in the design
notes of the repository.  Arithmetic is FP64 throughout; numpy/scipy routines
serve as single steps (a matmul, a Cholesky factor, a symmetric eigensolve, an
FFT) with no blocking, fusion or reordering beyond the definitions.

Modules
  fd        12th-order central finite-difference Laplacian (Sec. 5.B.2, n0 = 6)
  pseudo    pseudocharge electrostatics (Eq. poisson) and KB projectors
  operator  the subdomain Hamiltonian H^alpha (Eq. ks restricted to Omega^alpha)
  chefsi    Chebyshev filter, projection, generalised eigensolve, rotation (Sec. 5.A.3)
  fermi     Fermi level, density, band/entropy energies (Eqs. density, dos; Sec. 5.A.4-5)
  dc        divide-and-conquer partition, restriction, interior weights (Sec. 5.A.2)

Parity status: every function is pinned by the `-m "not gpu"` tests against
closed forms, brute-force dense diagonalisation or invariants; none is
"parity unpinned".
"""
