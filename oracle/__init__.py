"""CPU FP64 oracle for the solve phase of the block-preconditioned Jacobian.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and
the ``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import,
call or execute anything in this package.  The product path (the CUDA library
and its Python binding) never touches it and shares no code with it.

Contents (each function cites the passage of Franceschini, Gazzola and
Ferronato, arXiv 2112.12397, that it follows):

* ``sparse``   scalar CSR views of the generator's blocks and the full
               Jacobian of Eq. JacSys.
* ``rng``      SplitMix64 counter generator (Steele, Lea and Flood 2014),
               written from its published definition; the AMG draws its
               aggregation priorities and power-iteration start from it.
* ``schur``    H~ = Bdiag(H,3), T~ = diag(T), S1, S~ (Alg. 1, Alg. 3,
               Eq. appSchur_1, Eq. Schur1_2) and the algebraic fixed-stress
               S_K / S~2 (Eq. FS_algebraic, Eq. app_Schur2_2).
* ``amg``      smoothed-aggregation AMG (Vanek et al., the aggregation family
               the paper uses through GAMG, Sec. 3.1) and its V-cycle with a
               Chebyshev smoother.
* ``precond``  app_tpu (Alg. 2) and app_tup (Alg. 4) with AMG, V-cycle or
               exact inner solves.
* ``fgmres``   right-preconditioned flexible GMRES with classical
               Gram-Schmidt applied twice (Sec. 4, zero initial guess,
               relative residual stop).
* ``dense``    plain dense definitions used as pins on tiny cases:
               x = J^-1 b (Eq. ex_Jac_appl), exact Schur complements,
               the preconditioned operators of Eq. P1 / Eq. P2.
"""
