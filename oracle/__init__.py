"""CPU FP64 oracle for algebraic hybridization and static condensation of H(div).

TEST INFRASTRUCTURE ONLY. This package is a plain, slow, obviously-correct
restatement of the method of Dobrev, Kolev, Lee, Tomov and Vassilevski,
"Algebraic hybridization and static condensation with application to scalable
H(div) preconditioning" (arXiv:1801.08914). Only the test-suite, the smoke
check and the benchmark's CPU-baseline leg may import it; the product path
(the CUDA library and its binding) never does, and it shares no code with it.

Modules
  quadrature  Gauss-Legendre / Gauss-Lobatto rules by Newton's method on Legendre polynomials
  basis       1-D Lagrange polynomials and the reference RT_k basis (nodal, tensor product)
  mesh        structured hex-mesh topology: faces, multipliers, conforming dofs
  element     element matrices A_T, unit mass M_T and loads through the Piola map
  hybrid      hybridization (Thm 2.1, eq. 2.4), static condensation (Sec. 3.1),
              conforming assembly (eq. 2.2), dense saddle-point solve, diagonal PCG

Every function cites the passage of the paper it follows. Readings of points
the paper leaves open are stated where they are used.
"""
