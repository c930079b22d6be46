"""Plain FP64 CPU oracle for the SIPG multigrid hot path (Cui & Kanschat,
"Multilevel Interior Penalty Methods on GPUs", arXiv 2405.18982).

TEST INFRASTRUCTURE ONLY.  Nothing in the library imports this package; only
``tests/``, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` / reference
legs of ``bench.py`` may call it.  It shares no code with the CUDA path.

Everything here is written to be read against the paper, not to be fast:
generic d-dimensional quadrature assembly of the SIPG matrix (Sec. 2, Eq.
bilinear_form), explicit sparse prolongation / restriction (Sec. 3), dense
patch matrices inverted by Cholesky (Eqs. residual and local-solver,
Algorithm 1), the V-cycle of Sec. 3, flexible CG, and an independent global
fast-diagonalisation direct solver (Sec. 3.2, Eqs. inverse2d / inverse3d
applied to the whole Cartesian mesh).

Module map
  basis     Gauss-Lobatto nodes, Gauss rules, Lagrange basis (Appendix A)
  assembly  SIPG matrix, mass matrix, right-hand side, element blocks (Sec. 2)
  mg        hierarchy, transfer, vertex patches, smoother, V-cycle, FCG (Sec. 3)
  direct    Kronecker form and global fast-diagonalisation solve (Sec. 2.2, 3.2)
  adjoint   gradients of a least-squares loss through the solve
  layout    cell-wise lexicographic indexing helpers (Sec. 4.1)

Parity status of each function is stated in its docstring; every function is
pinned by a ``-m "not gpu"`` test in ``tests/test_oracle_*.py`` except the
ones marked "parity unpinned".
"""
