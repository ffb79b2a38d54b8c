"""Pins for the one-end trick (Sec. 2.3, Eq. 2.5) in oracle.loops.

* The identity behind it, on dense matrices assembled from the operator at
  +mu and at -mu separately: D_u^-1 - D_d^-1 = -4 i kappa mu D_u^-1 D_u^-dag gamma5.
* Summed over a complete orthonormal basis of sources (E[eta eta^dag] = 1
  exactly), the per-source values add up to the exact isovector loop
  Tr[P Gamma (D_u^-1 - D_d^-1)] of the two dense inverses.
* With Z4 noise the sample mean approaches that loop within its error.
* The TSM estimate with the one-end values reaches it too (both solves of
  the correction use the same quadratic form).
"""
import numpy as np

from oracle import dirac, loops, philox
from paper_1211_0126_gb300 import synthetic as S

KAPPA, MU = 0.124, 0.03
GAM = list(range(16))
MOMS = [(0, 0, 0), (1, 0, 0)]


def _gamma5_full(vol):
    return np.kron(np.eye(vol), np.kron(np.diag([1.0, 1.0, -1.0, -1.0]), np.eye(3)))


def test_isovector_identity_dense():
    dims = (2, 2, 2, 2)
    U = S.gauge_field(dims, 0.5, 1)
    Du = dirac.dense_dtm(U, dims, KAPPA, MU)
    Dd = dirac.dense_dtm(U, dims, KAPPA, -MU)
    iu, idd = np.linalg.inv(Du), np.linalg.inv(Dd)
    rhs = -4j * KAPPA * MU * iu @ iu.conj().T @ _gamma5_full(16)
    assert np.abs((iu - idd) - rhs).max() < 1e-12 * np.abs(iu).max()


def test_complete_basis_reproduces_exact_isovector_loop():
    dims = (2, 2, 2, 2)
    U = S.gauge_field(dims, 0.5, 2)
    iu = np.linalg.inv(dirac.dense_dtm(U, dims, KAPPA, MU))
    idd = np.linalg.inv(dirac.dense_dtm(U, dims, KAPPA, -MU))
    exact = loops.exact_loops(iu - idd, dims, GAM, MOMS)
    vol = 16
    total = np.zeros_like(exact)
    for k in range(12 * vol):
        s = iu[:, k].reshape(dims[3], dims[2], dims[1], dims[0], 4, 3)
        total += loops.one_end_loops(s, dims, KAPPA, MU, GAM, MOMS)
    assert np.abs(total - exact).max() < 1e-11 * max(np.abs(exact).max(), 1.0)
    # and it differs from the plain u loop (the d part matters)
    assert np.abs(exact - loops.exact_loops(iu, dims, GAM, MOMS)).max() > 1e-3


def test_z4_average_converges():
    dims = (2, 2, 2, 2)
    U = S.gauge_field(dims, 0.5, 3)
    iu = np.linalg.inv(dirac.dense_dtm(U, dims, KAPPA, MU))
    idd = np.linalg.inv(dirac.dense_dtm(U, dims, KAPPA, -MU))
    exact = loops.exact_loops(iu - idd, dims, GAM, MOMS)
    vals = []
    for j in range(600):
        eta = philox.noise(7, j, dims, 4)
        s = (iu @ eta.ravel()).reshape(eta.shape)
        vals.append(loops.one_end_loops(s, dims, KAPPA, MU, GAM, MOMS))
    vals = np.array(vals)
    mean = vals.mean(0)
    err = vals.std(0) / np.sqrt(len(vals)) + 1e-14
    z = np.abs(mean - exact) / err
    assert np.median(z) < 1.5 and z.max() < 6.0


def test_tsm_one_end_against_dense():
    dims = (2, 2, 2, 2)
    U = S.gauge_field(dims, 0.5, 4)
    iu = np.linalg.inv(dirac.dense_dtm(U, dims, KAPPA, MU))
    idd = np.linalg.inv(dirac.dense_dtm(U, dims, KAPPA, -MU))
    exact = loops.exact_loops(iu - idd, dims, GAM, MOMS)
    got = loops.tsm_loops(U, dims, KAPPA, MU, 11, 4, 8, 200, (1e-12, 2000), (0.0, 1), GAM, MOMS,
                          estimator='one_end')
    z = np.abs(got['loops'] - exact) / (got['err'] + 1e-14)
    assert np.median(z) < 1.5 and z.max() < 6.0
    # the truncated (1-iteration) LP-only mean alone is biased, far outside its own
    # statistical error; the correction removes that bias
    lp = got['lp']
    sig_lp = np.sqrt((np.abs(lp - lp.mean(0)) ** 2).sum(0) / (len(lp) - 1) / len(lp)) + 1e-14
    zl = np.abs(got['lp_mean'] - exact) / sig_lp
    assert zl.max() > 10.0


# ---- generalised one-end trick (Eq. 2.6), isoscalar u + d

def test_isoscalar_identity_dense():
    dims = (2, 2, 2, 2)
    U = S.gauge_field(dims, 0.5, 5)
    Du = dirac.dense_dtm(U, dims, KAPPA, MU)
    Dd = dirac.dense_dtm(U, dims, KAPPA, -MU)
    Dw = dirac.dense_dtm(U, dims, KAPPA, 0.0)          # 1 - kappa H, assembled on its own
    iu, idd = np.linalg.inv(Du), np.linalg.inv(Dd)
    g5 = _gamma5_full(16)
    rhs = 2.0 * g5 @ iu.conj().T @ g5 @ Dw @ iu
    assert np.abs((iu + idd) - rhs).max() < 1e-12 * np.abs(iu).max()
    # the property the stochastic form rests on
    assert np.abs(Du @ Du.conj().T - g5 @ Du.conj().T @ Du @ g5).max() < 1e-12


def test_gen_complete_basis_reproduces_exact_isoscalar_loop():
    dims = (2, 2, 2, 2)
    U = S.gauge_field(dims, 0.5, 6)
    iu = np.linalg.inv(dirac.dense_dtm(U, dims, KAPPA, MU))
    idd = np.linalg.inv(dirac.dense_dtm(U, dims, KAPPA, -MU))
    exact = loops.exact_loops(iu + idd, dims, GAM, MOMS)
    total = np.zeros_like(exact)
    for k in range(12 * 16):
        s = iu[:, k].reshape(dims[3], dims[2], dims[1], dims[0], 4, 3)
        total += loops.gen_one_end_loops(U, s, dims, KAPPA, GAM, MOMS)
    assert np.abs(total - exact).max() < 1e-11 * max(np.abs(exact).max(), 1.0)


def test_gen_tsm_against_dense():
    dims = (2, 2, 2, 2)
    U = S.gauge_field(dims, 0.5, 7)
    iu = np.linalg.inv(dirac.dense_dtm(U, dims, KAPPA, MU))
    idd = np.linalg.inv(dirac.dense_dtm(U, dims, KAPPA, -MU))
    exact = loops.exact_loops(iu + idd, dims, GAM, MOMS)
    got = loops.tsm_loops(U, dims, KAPPA, MU, 13, 4, 8, 300, (1e-12, 2000), (0.0, 2), GAM, MOMS,
                          estimator='gen_one_end')
    z = np.abs(got['loops'] - exact) / (got['err'] + 1e-14)
    assert np.median(z) < 1.5 and z.max() < 6.0
