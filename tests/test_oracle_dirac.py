"""Pins for oracle.dirac and oracle.solver.

What fixes the operator independently of the oracle's own code:
* free field (U = 1): a plane wave exp(i p.x) u is an eigenvector with the
  momentum-space matrix  A + i (sum_mu gamma_mu B_mu + C gamma_5),
  A = 1 - 2 kappa sum cos p_mu, B_mu = 2 kappa sin p_mu, C = 2 kappa mu,
  p_4 = 2 pi (n + 1/2) / T for antiperiodic time (pins projector signs,
  hopping directions, axis mapping and the boundary sign);
* gamma_5-hermiticity gamma_5 D(mu) gamma_5 = D(-mu)^dagger (pins the adjoint);
* gauge covariance D[U^G] G psi = G D[U] psi (pins link placement, U vs U^T
  and U vs U^dagger on backward hops);
* dense linear algebra: the Schur complement solve and CGNR reproduce
  numpy.linalg.solve of the dense D_tm (pins the even/odd algebra and the
  solver);
* a 2^4 lattice, where the forward and backward neighbours coincide.
"""
import numpy as np
import pytest

from oracle import dirac, solver
from oracle.gamma import gamma_matrices
from paper_1211_0126_gb300 import synthetic as S

KAPPA, MU = 0.124, 0.01


def _dot(a, b):
    return np.vdot(a.ravel(), b.ravel())


def _plane_wave(dims, n, u, antiperiodic):
    lx, ly, lz, lt = dims
    t, z, y, x = np.meshgrid(np.arange(lt), np.arange(lz), np.arange(ly), np.arange(lx),
                             indexing='ij')
    shift = 0.5 if antiperiodic else 0.0
    p = (2 * np.pi * n[0] / lx, 2 * np.pi * n[1] / ly, 2 * np.pi * n[2] / lz,
         2 * np.pi * (n[3] + shift) / lt)
    ph = np.exp(1j * (p[0] * x + p[1] * y + p[2] * z + p[3] * t))
    return ph[..., None, None] * u[None, None, None, None], p


@pytest.mark.parametrize("dims", [(4, 4, 4, 4), (2, 2, 2, 2), (4, 2, 6, 4)])
@pytest.mark.parametrize("antiperiodic", [True, False])
def test_free_field_plane_wave(dims, antiperiodic):
    rng = np.random.default_rng(3)
    g, g5 = gamma_matrices()
    U = S.gauge_field(dims, 0.0, 0)
    for _ in range(4):
        n = [int(rng.integers(0, d)) for d in dims]
        u = rng.standard_normal((4, 3)) + 1j * rng.standard_normal((4, 3))
        psi, p = _plane_wave(dims, n, u, antiperiodic)
        A = 1 - 2 * KAPPA * sum(np.cos(p))
        M = A * np.eye(4) + 1j * (sum(g[m] * 2 * KAPPA * np.sin(p[m]) for m in range(4))
                                  + 2 * KAPPA * MU * g5)
        want, _ = _plane_wave(dims, n, M @ u, antiperiodic)
        got = dirac.dtm(U, psi, dims, KAPPA, MU, antiperiodic)
        assert np.allclose(got, want, atol=1e-13)


@pytest.mark.parametrize("dims", [(4, 4, 4, 4), (2, 2, 2, 2)])
def test_gamma5_hermiticity(dims):
    U = S.gauge_field(dims, 0.3, 11)
    phi = S.random_spinor(dims, 1)
    psi = S.random_spinor(dims, 2)
    lhs = _dot(phi, dirac.gamma5(dirac.dtm(U, dirac.gamma5(psi), dims, KAPPA, MU)))
    rhs = _dot(dirac.dtm(U, phi, dims, KAPPA, -MU), psi)
    assert abs(lhs - rhs) < 1e-12 * abs(lhs)
    # the literal adjoint (projectors swapped) equals the gamma_5 sandwich at -mu
    a = dirac.dtm(U, psi, dims, KAPPA, MU, adjoint=True)
    b = dirac.gamma5(dirac.dtm(U, dirac.gamma5(psi), dims, KAPPA, -MU))
    assert np.allclose(a, b, atol=1e-13)


def test_adjoint_is_dense_conjugate_transpose():
    dims = (2, 2, 2, 2)
    U = S.gauge_field(dims, 0.3, 5)
    D = dirac.dense_dtm(U, dims, KAPPA, MU)
    psi = S.random_spinor(dims, 4)
    got = dirac.dtm(U, psi, dims, KAPPA, MU, adjoint=True).reshape(-1)
    assert np.allclose(got, D.conj().T @ psi.reshape(-1), atol=1e-13)


@pytest.mark.parametrize("dims", [(4, 4, 4, 4), (2, 2, 2, 2), (4, 2, 2, 6)])
def test_gauge_covariance(dims):
    U = S.gauge_field(dims, 0.3, 21)
    G = S.gauge_transform(dims, 22)
    UG = S.transform_links(U, G)
    psi = S.random_spinor(dims, 23)
    lhs = dirac.dtm(UG, S.transform_spinor(psi, G), dims, KAPPA, MU)
    rhs = S.transform_spinor(dirac.dtm(U, psi, dims, KAPPA, MU), G)
    assert np.abs(lhs - rhs).max() < 1e-13 * np.abs(rhs).max()
    # the gauge transform is not trivial: without it the result differs
    assert np.abs(dirac.dtm(U, S.transform_spinor(psi, G), dims, KAPPA, MU)
                  - rhs).max() > 1e-3


def test_hop_at_site_matches_full_stencil():
    dims = (4, 2, 6, 4)
    U = S.gauge_field(dims, 0.3, 31)
    psi = S.random_spinor(dims, 32)
    full = dirac.hop(U, psi, dims)
    for site in [(0, 0, 0, 0), (3, 1, 5, 3), (1, 0, 2, 0), (2, 1, 0, 3)]:
        x, y, z, t = site
        assert np.allclose(dirac.hop_at_site(U, psi, dims, site), full[t, z, y, x], atol=1e-13)


def test_hop_only_couples_opposite_parity():
    dims = (4, 4, 4, 4)
    U = S.gauge_field(dims, 0.3, 41)
    psi = S.random_spinor(dims, 42) * dirac.even_mask(dims)
    h = dirac.hop(U, psi, dims)
    assert np.abs(h * dirac.even_mask(dims)).max() == 0.0


@pytest.mark.parametrize("dims", [(2, 2, 2, 2), (4, 2, 2, 2)])
def test_schur_complement_against_dense_solve(dims):
    U = S.gauge_field(dims, 0.3, 51)
    b = S.random_spinor(dims, 52)
    D = dirac.dense_dtm(U, dims, KAPPA, MU)
    x_exact = np.linalg.solve(D, b.reshape(-1)).reshape(b.shape)
    # Dhat x_e = bhat_e holds for the exact solution, and reconstruction returns it
    e = dirac.even_mask(dims)
    bhat = dirac.schur_source(U, b, dims, KAPPA, MU)
    assert np.allclose(dirac.schur(U, e * x_exact, dims, KAPPA, MU), bhat, atol=1e-12)
    rec = dirac.schur_reconstruct(U, e * x_exact, b, dims, KAPPA, MU)
    assert np.allclose(rec, x_exact, atol=1e-12)


def test_schur_dag_is_adjoint():
    dims = (4, 2, 2, 2)
    U = S.gauge_field(dims, 0.3, 61)
    e = dirac.even_mask(dims)
    a = S.random_spinor(dims, 62) * e
    c = S.random_spinor(dims, 63) * e
    lhs = _dot(a, dirac.schur(U, c, dims, KAPPA, MU))
    rhs = _dot(dirac.schur_dag(U, a, dims, KAPPA, MU), c)
    assert abs(lhs - rhs) < 1e-13 * abs(lhs)


@pytest.mark.parametrize("dims", [(4, 4, 4, 4), (2, 2, 2, 2)])
def test_cgnr_converges_to_dense_solution(dims):
    U = S.gauge_field(dims, 0.3, 71)
    b = S.random_spinor(dims, 72)
    D = dirac.dense_dtm(U, dims, KAPPA, MU)
    x_exact = np.linalg.solve(D, b.reshape(-1)).reshape(b.shape)
    s, iters, res, true_res = solver.solve_full(U, b, dims, KAPPA, MU, 1e-12, 5000)
    assert res < 1e-12 and iters > 5
    assert true_res < 1e-9
    assert np.linalg.norm(s - x_exact) / np.linalg.norm(x_exact) < 1e-9
    # fixed-iteration truncation stops exactly at max_iter
    _, it5, res5, _ = solver.solve_full(U, b, dims, KAPPA, MU, 0.0, 5)
    assert it5 == 5 and res5 > res


def test_cgnr_zero_source():
    dims = (2, 2, 2, 2)
    U = S.gauge_field(dims, 0.3, 81)
    s, iters, res = solver.cgnr(U, np.zeros((2, 2, 2, 2, 4, 3), complex), dims, KAPPA, MU,
                               1e-10, 100)
    assert iters == 0 and np.all(s == 0)
