"""Plain FP64 CPU oracle for the matrix-free kernel products and the HMC step.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import this
package.  The library (``paper_2412_20884_gb300``) never imports it, and this
package imports nothing from the library: the two share no code.

Everything is written from the paper's definitions, in float64, with no
blocking, fusion or reordering beyond what a definition states (row blocks
are used only to bound memory; every block evaluates the same formula):

  * ``se_kernel``  - A(theta) = K(theta) + sigma^2 I (Eq. kerdef, Eq. kernmat)
                     with the squared-exponential kernel of Sec. 1, its
                     products A V and the adjoint of L = sum G o (A V).
  * ``hmc``        - the potential U (Eq. U), the force by its direct
                     expression (Sec. 3.2.1), the leapfrog map (Sec. 3.2.2),
                     the Hamiltonian and the Metropolis test (Algorithm 1), the
                     exact marginal posterior P(theta) (Eq. P) and the exact
                     Gibbs draw phi = A^{-1/2} xi (Sec. 3.1).
  * ``poles``      - the pole expansion of A^{-1/2} (Eq. pex, App. A, Eq. msqdisc).
  * ``diagnostics``- moving-window means (Sec. 4.1) and the integrated
                     autocorrelation time (App. C).
  * ``cheb_kernel``- the Chebyshev log-amplitude kernel family of Sec. 4, its
                     dense A and derivatives.
  * ``nystrom``    - the randomized Nystrom approximation and preconditioner
                     (Frangella, Tropp and Udell) the paper uses for its
                     solves, and preconditioned CG.
  * ``implicit``   - the implicit midpoint step (Sec. 3.2.3, Eq. Phi) solved
                     by Anderson acceleration (App. B).

Pins (tests/test_oracle_*.py) tie each function to values fixed by the paper
or by mathematics rather than to itself.  Parity status per function is listed
in each module's header.
"""
