"""Oracle: a plain, slow, complex128 CPU restatement of QR-based TEBD.

This package is TEST INFRASTRUCTURE. Only ``tests/``, ``__graft_entry__.smoke()``
and the ``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import it.
The CUDA library never calls it, and it never calls the CUDA library: the two
share no code. Inputs reach both sides from ``paper_2212_09782_b300.workloads``,
which draws seeded random numbers and does none of the method's arithmetic.

Modules
-------
clock       clock-model operators, bond Hamiltonians and Trotter gates (Sec. IV, Eqs. 2-3)
bond        the QR bond update (Sec. II, Fig. 2), controlled bond expansion
            (Sec. III, Fig. 3) and the SVD-truncated update used as a comparison
householder a textbook Householder QR used to cross-check the LAPACK QR on tiny inputs
mps         finite and uniform MPS in right-isometric form (Eq. 1, Fig. 1) and the
            Strang-split TEBD driver (Fig. 2a)
exact       state-vector references: Trotterised state vector and Krylov evolution
symmetric   CBE with Z_d charge sectors (Sec. III, closing paragraphs): the clock model in
            the charge (Fourier) basis, per-block expansion, one cut over all blocks that
            sets each block's dimension, and a finite-chain driver

Every function runs in complex128 / float64. Library primitives (matmul, LAPACK
QR, eigh, SVD, expm) serve as single steps; nothing is blocked, fused or reordered
beyond what the paper's steps state.

Parity status: every function here is pinned by ``tests/test_oracle_*.py`` against
closed forms, invariants, brute force or exact references. The tie rule of the CBE cut
(``bond.cbe_cut``: never cut inside a multiplet) is a reading of a point the paper leaves
open. It is pinned by the property it exists for: with it, the kept subspace does not
depend on the initial guess Y0; without it, it does.
"""
