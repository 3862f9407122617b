"""Plain, slow FP64 CPU oracle of the exact spin spherical harmonic transform
(McEwen, "Fast, exact (but unstable) spin spherical harmonic transforms",
arXiv:0807.4494).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline / reference leg of ``bench.py`` may import, call, link or execute
anything in this package.  The CUDA library never imports it and shares no code
with it.

Modules:
  ``transforms``  the method's steps in the paper's order (Risbo recursion and
                  the O(L^3) sums in C, the DFTs through numpy.fft);
  ``brute``       plain definitions used to pin the oracle: the explicit Wigner
                  sum at beta = pi/2 in exact rational arithmetic, eqn wignerd_b
                  through Jacobi polynomials, spin harmonics by eqn ssh_wigner
                  and eqn ssh_goldberg, direct synthesis and Gauss-Legendre
                  quadrature.

Parity status: every function is pinned by a ``-m "not gpu"`` test (see
``tests/test_oracle_*.py``); the paper's triangular forward
(``transforms.forward_triangular``) is pinned only qualitatively (machine
precision at small L, growth with L), because the paper gives its instability as
figures without numbers.
"""
