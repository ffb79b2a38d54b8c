"""Pins for the one-derivative insertions in oracle.loops.

* A complete orthonormal basis of sources reproduces, through the per-source
  estimator, the loop computed term by term from the operator's site-pair
  blocks and a dense inverse (two independent codings of the operator).
* Gauge invariance of the exact derivative loops (U -> G U G^dag).
* Free field, q = 0: the loop of gamma_mu D_mu equals the closed form
  obtained in momentum space, 12 V_s (1/V) sum_p (-i sin p_mu) tr-part,
  here checked against a direct momentum sum of the free propagator.
* Z4 noise average approaches the exact loop.
"""
import numpy as np

from oracle import dirac, loops, philox
from paper_1211_0126_gb300 import synthetic as S

KAPPA, MU = 0.124, 0.02
GAM = list(range(16))
MUS = [0, 3]
MOMS = [(0, 0, 0), (1, 0, 0)]
DIMS = (2, 2, 2, 4)


def test_complete_basis_matches_blockwise_definition():
    U = S.gauge_field(DIMS, 0.5, 1)
    iu = np.linalg.inv(dirac.dense_dtm(U, DIMS, KAPPA, MU))
    exact = loops.exact_deriv_loops(U, iu, DIMS, GAM, MUS, MOMS)
    vol = int(np.prod(DIMS))
    total = np.zeros_like(exact)
    for k in range(12 * vol):
        e = np.zeros(12 * vol, dtype=np.complex128)
        e[k] = 1.0
        eta = e.reshape(DIMS[3], DIMS[2], DIMS[1], DIMS[0], 4, 3)
        s = iu[:, k].reshape(eta.shape)
        total += loops.deriv_loops(U, eta, s, DIMS, GAM, MUS, MOMS)
    assert np.abs(total - exact).max() < 1e-11 * max(np.abs(exact).max(), 1.0)
    assert np.abs(exact).max() > 1e-3


def test_exact_deriv_loops_gauge_invariant():
    U = S.gauge_field(DIMS, 0.5, 2)
    G = S.gauge_transform(DIMS, 3)
    Ug = S.transform_links(U, G)
    a = loops.exact_deriv_loops(U, np.linalg.inv(dirac.dense_dtm(U, DIMS, KAPPA, MU)), DIMS, GAM, MUS, MOMS)
    b = loops.exact_deriv_loops(Ug, np.linalg.inv(dirac.dense_dtm(Ug, DIMS, KAPPA, MU)), DIMS, GAM, MUS, MOMS)
    assert np.abs(a - b).max() < 1e-11 * np.abs(a).max()


def test_free_field_momentum_sum():
    dims = (2, 2, 2, 4)
    U = S.gauge_field(dims, 0.0, 0)
    iu = np.linalg.inv(dirac.dense_dtm(U, dims, KAPPA, MU))
    got = loops.exact_deriv_loops(U, iu, dims, GAM, [0, 3], [(0, 0, 0)])
    # momentum space: for a plane-wave propagator S(p), the q = 0 loop of
    # Gamma D<->_mu summed over a timeslice is (V_s / V) sum_p i sin(p_mu) tr[Gamma S(p)]
    # (the forward and backward hops give e^{+-ip_mu}; the four terms add to i sin p_mu)
    from oracle.gamma import gamma_matrices
    g, g5 = gamma_matrices()
    lx, ly, lz, lt = dims
    vol = lx * ly * lz * lt
    want = np.zeros((16, 2), dtype=np.complex128)
    Glist = __import__('oracle.gamma', fromlist=['gamma_list']).gamma_list()
    for nx in range(lx):
        for ny in range(ly):
            for nz in range(lz):
                for nt in range(lt):
                    p = [2 * np.pi * nx / lx, 2 * np.pi * ny / ly, 2 * np.pi * nz / lz,
                         2 * np.pi * (nt + 0.5) / lt]
                    A = 1 - 2 * KAPPA * sum(np.cos(pp) for pp in p)
                    Dp = A * np.eye(4) + 1j * (sum(2 * KAPPA * np.sin(p[m]) * g[m] for m in range(4))
                                               + 2 * KAPPA * MU * g5)
                    Sp = np.linalg.inv(Dp)
                    for gi in range(16):
                        for k, mu in enumerate([0, 3]):
                            want[gi, k] += 3 * 1j * np.sin(p[mu]) * np.trace(Glist[gi] @ Sp) / vol
    want *= lx * ly * lz   # per timeslice sum over V_s sites
    assert np.allclose(got[:, :, 0, :], want[:, :, None], atol=1e-12)
    assert np.abs(want).max() > 1e-3


def test_z4_average_converges():
    U = S.gauge_field(DIMS, 0.5, 4)
    iu = np.linalg.inv(dirac.dense_dtm(U, DIMS, KAPPA, MU))
    exact = loops.exact_deriv_loops(U, iu, DIMS, GAM, MUS, MOMS)
    vals = []
    for j in range(400):
        eta = philox.noise(9, j, DIMS, 4)
        s = (iu @ eta.ravel()).reshape(eta.shape)
        vals.append(loops.deriv_loops(U, eta, s, DIMS, GAM, MUS, MOMS))
    vals = np.array(vals)
    err = vals.std(0) / np.sqrt(len(vals)) + 1e-14
    z = np.abs(vals.mean(0) - exact) / err
    assert np.median(z) < 1.5 and z.max() < 6.0
