"""FP64 CPU oracle for the deflated/recycled BDDC-PCG path (test infrastructure).

This package is test infrastructure, not part of the product. Only `tests/`,
`__graft_entry__.smoke()` and `bench.py`'s CPU-baseline / reference arm may
import it. It shares no code with the CUDA path: the only common input is the
seeded generator in `workload/`.

Contents (each function cites the part of the paper it restates):
  q1        Q1 element matrices by Gauss quadrature, global assembly (Sect. 2, eq. 5)
  cholesky  nested-dissection multifrontal sparse Cholesky of K (direct solve of eq. 5)
  dd        substructuring, Schur complement, globs, BDDC two-/three-level, adaptive
            face constraints (Sect. 3.1-3.3)
  pcg       deflated PCG (Algorithm 1), recycling B1-B4, harmonic Ritz (eq. 15),
            freezing criterion (eq. 16), stopping criteria (Sect. 5)
  adjoint   adjoint solve and coefficient gradient of a quadratic loss
  lobpcg    block LOBPCG for the largest eigenpairs of a symmetric pencil (the paper's face
            eigensolver, Sect. 3.3), used by dd.adaptive_face_constraints(method="lobpcg")

Parity status: every function is pinned by a `-m "not gpu"` test except the
adaptive face constraints (`dd.adaptive_face_constraints`), which are
"parity unpinned" against the paper: the paper obtains them by LOBPCG with
iteration limits, so only invariants (lambda_min >= 1, lambda_max not above the
non-adaptive one, the solution unchanged) pin them.
"""
