"""CPU FP64 oracle for the mixed-precision multilevel Monte Carlo (MPML) hot path.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import this
package.  The GPU library (``paper_2503_05533_gb300``) never imports it and
shares no code with it: the two meet only through the seeded input generators
in ``tests/inputs.py`` and through the public C ABI.

Everything here is plain, slow and written to be checked against the paper by
eye.  Floating point is IEEE FP64 throughout.  Each module names the passage of
arXiv 2503.05533 ("Exploiting Inexact Computations in Multilevel Monte Carlo
and Other Sampling Methods") that it follows:

* ``rng``      -- the random inputs omega_j ~ N(0, 1) of the log-coefficient
                  (Sec. 5.1, Eq. (5.2)); generator definition: Philox4x32-10
                  (Salmon et al., SC'11) and Wichura's AS241 inverse normal.
* ``kl``       -- truncated Karhunen-Loeve bases: the paper's field
                  (Sec. 5.1, Eq. (5.2)) and a separable exponential covariance.
* ``fem``      -- P1 finite elements for Problem 3.1 (Sec. 3.1), element by
                  element; banded Cholesky / dense LU solves; the QoI of
                  Problem 4.5 (Sec. 4.3, Sec. 5.1).
* ``mlmc``     -- MLMC estimator (Eq. (4.1)), sample variance (Eq. (4.2)),
                  accuracy rule (Eqs. (4.7), (4.12)), adaptive MPML
                  (Algorithm 4.1), cost model (Sec. 4.2, Cor. 4.4).
* ``adjoint``  -- dQ/domega by the discrete adjoint of the P1 system.

The refinement of Algorithm 2.1 has no separate oracle: its result is the
solution of the P1 system, which ``fem`` computes directly, and every GPU
solve is checked through the FP64 residual of its returned solution against
``fem``'s own assembly.
"""
