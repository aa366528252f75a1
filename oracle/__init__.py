"""Plain, slow FP64 CPU oracle for the MGCG / interior-point / OC topology-optimisation path.

TEST INFRASTRUCTURE ONLY.  Nothing in the product package imports, links or runs this
package; only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py`` (its CPU-baseline
and reference legs) may use it.  It shares no code with the CUDA path: it assembles
sparse matrices, solves them exactly with banded Cholesky (LAPACK), and runs the
paper's algorithms step by step in the paper's order.

Paper: M. Kocvara, S. Mohammed, "Primal-dual interior-point multigrid method for
topology optimization" (arXiv 1606.06201).  Each function cites the section, equation
or algorithm it restates.

Modules
-------
fe        grid numbering, element stiffness K0 (2D Q1 plane stress, 3D trilinear hex),
          assembly of K(x) = sum_i x_i K_i  (Eq. (to), Sec. 7)
linsolve  exact SPD solves: banded Cholesky, bordering for the arrow matrix Z
mg        explicit prolongation, Galerkin coarse operators, Algorithm MG, Algorithm PCG
ip        primal-dual interior-point method (Sec. 2-3, Eq. (nwt), (nwtr), (nwtr2))
simp      SIMP model with the density filter and its IP method (Sec. 9)
oc        OC / damped OC / averaged OC (Sec. 4)
grad      adjoint gradient of a linear functional of u
runs      whole IP / AOC runs with per-step records, and a process pool to run them beside a GPU

Functions without an independent pin say so in their docstring ("parity unpinned").
"""
