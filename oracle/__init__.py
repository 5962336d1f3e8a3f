"""Plain FP64 CPU oracle for the twisted-mass DD-alpha-AMG solve (arXiv:1710.06198).

TEST INFRASTRUCTURE ONLY.  Nothing in the product path (the CUDA library and its Python binding)
imports, links or executes this package; only ``tests/``, ``__graft_entry__.smoke()`` and the CPU
baseline legs of ``bench.py`` use it.  It shares no code, tables or helpers with the CUDA path.

Every routine is written for readability over speed: whole-lattice numpy operations (``np.roll``
for neighbour hops, ``np.einsum`` for colour and spin algebra) in complex128, following the
definitions of the paper in the order the paper states them:

* ``dirac``  -- clover-improved Wilson operator D (Sec. 1.1), twisted mass D(+-mu) = D +- i mu G5
  (Sec. 1.1), the non-degenerate doublet D_ND (Eq. 2) and their Hermitian forms (Eqs. 3, 4).
* ``mg``     -- the two-level error propagation of Eq. 1: SAP smoother M, aggregation-based
  prolongation P (Gamma5-compatible), coarse operator D_c = P^dag D P, cycle and adaptive setup.
* ``krylov`` -- CG on the normal equations, MR, GMRES and flexible GMRES (Sec. 1.1, 1.2).
* ``force``  -- link derivative of the pseudofermion action phi^dag (D D^dag)^-1 phi (Sec. 1).

Parity status of each function is stated in its docstring ("pinned by ..." or "parity unpinned").
"""
