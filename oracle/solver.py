"""CG on the normal equations of the even/odd Schur complement (oracle; test infrastructure).

The paper truncates the low-precision (LP) inversions either at a loose
residual or after a fixed number of iterations, treating the two as the same
rule (Sec. 2.2), and runs a few high-precision (HP) ones, but never names the
solver.  Reading used here:
conjugate gradient on  Dhat^dagger Dhat x = Dhat^dagger bhat  (CGNR), zero
initial guess, stopped when the iterated normal residual satisfies
||r_k|| / ||Dhat^dagger bhat|| < rel_tol (not squared), or after max_iter
iterations, whichever comes first.  rel_tol = 0 means "fixed iteration count".

Iteration (textbook CG, Hestenes-Stiefel) with Dhat from oracle.dirac:
    r = p = Dhat^dag bhat,  rr = <r, r>
    repeat: q = Dhat p;  alpha = rr / <q, q>;  x += alpha p;
            r -= alpha Dhat^dag q;  rr' = <r, r>;  beta = rr' / rr;  p = r + beta p
The convergence test runs after every update.
"""
import numpy as np

from . import dirac


def _dot(a, b):
    return np.vdot(a.ravel(), b.ravel())


def cgnr(U, bhat, dims, kappa, mu, rel_tol, max_iter, antiperiodic_t=True):
    """Solve Dhat x = bhat on even sites.  Returns (x, iterations, final rel. residual)."""
    e = dirac.even_mask(dims)
    x = np.zeros_like(bhat)
    r = dirac.schur_dag(U, e * bhat, dims, kappa, mu, antiperiodic_t)
    p = r.copy()
    rr = _dot(r, r).real
    rhs_norm = np.sqrt(rr)
    if rhs_norm == 0.0:
        return x, 0, 0.0
    k = 0
    while k < max_iter and np.sqrt(rr) >= rel_tol * rhs_norm:
        q = dirac.schur(U, p, dims, kappa, mu, antiperiodic_t)
        alpha = rr / _dot(q, q).real
        x = x + alpha * p
        r = r - alpha * dirac.schur_dag(U, q, dims, kappa, mu, antiperiodic_t)
        rr_new = _dot(r, r).real
        beta = rr_new / rr
        p = r + beta * p
        rr = rr_new
        k += 1
    return x, k, float(np.sqrt(rr) / rhs_norm)


def solve_full(U, b, dims, kappa, mu, rel_tol, max_iter, antiperiodic_t=True):
    """D_tm s = b by even/odd reduction + CGNR + odd reconstruction.

    Returns (s, iterations, rel. normal residual, true residual ||b - D s|| / ||b||).
    """
    bhat = dirac.schur_source(U, b, dims, kappa, mu, antiperiodic_t)
    xe, iters, res = cgnr(U, bhat, dims, kappa, mu, rel_tol, max_iter, antiperiodic_t)
    s = dirac.schur_reconstruct(U, xe, b, dims, kappa, mu, antiperiodic_t)
    true_res = np.linalg.norm(b - dirac.dtm(U, s, dims, kappa, mu, antiperiodic_t)) / np.linalg.norm(b)
    return s, iters, res, float(true_res)
