"""CPU oracle for the collision-resolution hot path (test infrastructure).

This package is a plain, slow, FP64 restatement of what the GPU library
computes, written independently from the paper.  It exists only to check the
CUDA path: only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline
leg of ``bench.py`` may import it.  The product library never calls it and
shares no code, tables or constants with it.

Contents (each function cites the passage it follows):

* ``quadrature``  sphere node/weight template (product Gauss-Legendre x uniform)
* ``contacts``    collisional set and the contact matrix D (Sec. 3, Eq. collisional-set)
* ``bie``         dense boundary-integral mobility: stresslet matrix, rigid
                  projector, Stokeslet/rotlet right-hand side, LU solve (Sec. 2, Fig. 1)
* ``rpy``         Rotne-Prager-Yamakawa pair mobility (low-fidelity operator)
* ``lcp``         LCP/QP definitions, KKT errors, projected Gauss-Seidel and
                  brute-force active-set enumeration (Sec. 3.1)
* ``pqn``         Mono-PQN (Algorithm 1), step size (Algorithm 2), weighted
                  prox by semi-smooth Newton (Prop. 1, Appendix A), Bi-PQN
                  (Algorithm 4, Appendix D)
* ``mf``          matrix-free FP64 GMRES mobility in plain C for sizes where the
                  dense matrix does not fit

Parity status: every function here is pinned by ``tests/test_oracle_*.py``
against closed forms, invariants or brute force.  The physical accuracy of the
discretised boundary-integral operator for interacting spheres is pinned
against exact two-sphere Stokes flow (moving together and approaching each
other along the line of centres) at centre distances of 2.5 radii and more;
closer than that, at gaps below about 0.2 radii, the plain quadrature misses
the lubrication resistance and that regime stays outside the workloads.
"""
