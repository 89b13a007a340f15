"""FP64 CPU oracle for the kernel-compensated MFD Maxwell eigenproblem (test infrastructure only).

This package is the checker, not the product. Only ``tests/``, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` /
``--impl reference`` legs of ``bench.py`` may import it. It shares no code with the CUDA path: it builds every operator
as an explicit scipy sparse matrix straight from the paper's Kronecker/circulant definitions, and uses library
primitives (sparse matvec, numpy FFT, LAPACK eigh, ARPACK) for the individual steps, in the paper's order.

Modules and what each one follows:

* ``mfd``       -- Table 1 stencils, circulants D1/D0 (eq. circ_def, stencils), D_i = K_i + iL_i (eq. discre, blocks),
                   grad/curl/div block matrices (eq. discrete_2nd_block), the compensated operator (eq. Ker_comp), the
                   penalty gamma (eq. pnt_number), the preconditioner matrix (eq. penalised_marix).
* ``spectrum``  -- the exact discrete spectrum for a homogeneous permittivity, derived from the circulant symbols
                   (Section 5.2, eq. diag_of_circ) together with Proposition 3.1.
* ``geometry``  -- M0 from a sphere structure: inverse permittivity at edge midpoints with the interface rule
                   (Section 4.4); the BCC gyroid and the FCC diamond of Section 6.3.
* ``precond``   -- the FFT preconditioner solve (Algorithm 5.1 with the 3x3 symbol of eq. penalised_marix).
* ``eigs``      -- dense / shift-invert reference eigenpairs, an independent block LOBPCG (Section 5.1), the
                   recompute check (Algorithm 4.1) and the k = 0 treatment (Remark after eq. penalised_marix).
* general lattices -- ``mfd``, ``spectrum``, ``precond`` and ``geometry`` take an optional ``lattice`` A (Section 2's
                   coordinate change, Section 4.2.2: K_hat_i = sum_j b_ji K_j with b = A^{-1}).
* ``warmstart`` -- the learned warm start's network (no counterpart in the paper, whose LOBPCG starts from a random
                   block): forward and hand-derived backward of each layer, the subspace loss, Adam.
* ``rng``       -- the counter-based generator that seeds initial blocks (splitmix64 finaliser + Box-Muller).

Every function states the passage it follows. Pins for each function live in ``tests/test_oracle_*.py``.
"""
