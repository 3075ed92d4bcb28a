"""FP64 CPU oracle for the symmetry-reduced Poisson solve (arXiv 2407.05930).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and
the ``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import or
run anything in this package.  The CUDA library never calls it and shares no
code with it; the two sides meet only through the seeded inputs of ``synth``.

What the oracle computes is the plain definition: assemble the full,
unreduced operator ``A`` in natural lexicographic order and solve
``A x = b`` (dense Cholesky for small ``n``, unpreconditioned CG otherwise,
and an exact sine-transform solve on uniform constant-coefficient grids).
The symmetry machinery of Sec. 2 (mirrored ordering, the change of basis
``P_s`` of eq. "P_s", the decoupled blocks of eqs. "hL_s"/"hL_splitting") is
written out here only so that the tests can pin it on small inputs; the
oracle's own solves never use it.

Modules
-------
grid      cell nodes: uniform or the tanh stretching of eq. "tanh" (Sec. 2.2)
fv        cell-centred finite-volume assembly of -div(k grad u) = f, Dirichlet
symmetry  mirrored ordering map ``perm`` and block extraction (Sec. 2, Fig. 1)
transform dense ``P_s`` (eq. "P_s") and the decoupled blocks (eq. "hL_s")
solvers   dense Cholesky, plain CG, closed-form spectra and the DST-II solve
adjoint   loss/gradient definitions for the differentiable solve

Parity status: every function here is pinned by ``tests/test_oracle_*.py``
(closed forms, brute force, invariants).  The AMG iteration counts of the
paper's Table "lrcamg" are context only ("parity unpinned": the paper gives
no tolerance for them).
"""
