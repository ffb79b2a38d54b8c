"""Plain FP64 CPU oracle for the truncated-solver-method (TSM) loop path.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import anything from this package.  The
product path (the CUDA library and its Python binding) never imports it and
shares no code, table or constant with it.

Everything here is written from the definitions of Alexandrou et al.,
"Evaluation of disconnected contributions using GPUs" (LATTICE 2012):

* noise sources with the Z2/Z4 moments of Sec. 2.1, Eq. (2.1);
* the stochastic inverse and its loops, Sec. 2.1 Eq. (2.2) and Sec. 2.3;
* the TSM estimator, Sec. 2.2 Eq. (2.4).

The paper leaves the Dirac operator, the gamma basis, the even/odd scheme and
the solver unstated; the twisted-mass operator D_tm = 1 - kappa*H +
2i*kappa*mu*gamma5 with the (1 -/+ gamma_mu) Wilson hopping term, the chiral
gamma basis and CG on the normal equations of the even/odd Schur complement are
the readings this oracle fixes.  Each module states which passage (or which
reading) it follows.

Modules
-------
gamma   gamma matrices (chiral basis) and the 16-element Gamma list
philox  Philox4x32-10 counter-based generator and the Z4/Z2 noise map
dirac   hopping term, D_tm, twist, even/odd Schur complement, dense assembly
solver  CGNR on the Schur complement normal equations
loops   local loop contraction, exact loops from a dense inverse, TSM combine

Pins: every function is checked in ``tests/test_oracle_*.py`` against things
other than itself (closed forms, algebraic identities, dense inversion,
exact variance formulas, statistics).  The Philox bit stream, whose exact
bits the paper does not fix, is pinned by the generator's published
known-answer vectors (Salmon et al., SC'11, Random123 distribution) and by
the distribution properties of Eq. (2.1).
"""
