"""Pins for oracle.loops: contraction, exact loops and the TSM combine.

* Free field: closed forms from the momentum-space inverse
  Dtilde^-1(p) = (A - i sum gamma_mu B_mu - i C gamma_5) / (A^2 + sum B_mu^2 + C^2):
  L_1(t, 0) = 12 V_s <A/den>_p, L_gamma5(t, 0) = -12 i C V_s <1/den>_p,
  every other Gamma and every q != 0 vanish (<.>_p = mean over momenta).
* Exact per-source variance of eta^dag B eta (B = P Gamma D^-1):
  Z4: sum_{a != b} |B_ab|^2 ; Z2: sum_{a != b} (|B_ab|^2 + B_ab conj(B_ba)).
  A transposed or mis-conjugated contraction gives another mean and variance.
* Sec. 2.1 / Eq. 2.3: the stochastic estimate converges to the exact loop as
  1/sqrt(N).
* Sec. 2.2 / Eq. 2.4: a strongly truncated LP solve biases the LP-only mean;
  the HP - LP correction removes the bias, and the stated error matches the
  scatter of independent TSM runs.
* Gauge covariance: per-source loops are unchanged when links and noise are
  gauge transformed together.
"""
import numpy as np
import pytest

from oracle import dirac, loops, philox, solver
from paper_1211_0126_gb300 import synthetic as S

KAPPA, MU = 0.124, 0.01
ALL_G = list(range(16))
MOMS4 = [(0, 0, 0), (1, 0, 0), (0, 1, 0), (0, 0, 1)]


def _free_closed_form(dims, kappa, mu):
    lx, ly, lz, lt = dims
    ps = np.meshgrid(2 * np.pi * np.arange(lx) / lx, 2 * np.pi * np.arange(ly) / ly,
                     2 * np.pi * np.arange(lz) / lz, 2 * np.pi * (np.arange(lt) + 0.5) / lt,
                     indexing='ij')
    A = 1 - 2 * kappa * sum(np.cos(p) for p in ps)
    den = A ** 2 + sum((2 * kappa * np.sin(p)) ** 2 for p in ps) + (2 * kappa * mu) ** 2
    C = 2 * kappa * mu
    vs = lx * ly * lz
    return 12 * vs * np.mean(A / den), -12j * C * vs * np.mean(1.0 / den)


@pytest.mark.parametrize("dims", [(4, 4, 4, 4), (2, 2, 2, 4), (4, 2, 2, 2)])
def test_free_field_exact_loops_closed_form(dims):
    U = S.gauge_field(dims, 0.0, 0)
    Dinv = np.linalg.inv(dirac.dense_dtm(U, dims, KAPPA, MU))
    L = loops.exact_loops(Dinv, dims, ALL_G, MOMS4)
    l1, l5 = _free_closed_form(dims, KAPPA, MU)
    assert np.allclose(L[0, 0], l1, atol=1e-12)
    assert np.allclose(L[5, 0], l5, atol=1e-12)
    mask = np.ones(L.shape, bool)
    mask[0, 0] = mask[5, 0] = False
    assert np.abs(L[mask]).max() < 1e-12


def _dense_setup(dims, eps, seed):
    U = S.gauge_field(dims, eps, seed)
    Dinv = np.linalg.inv(dirac.dense_dtm(U, dims, KAPPA, MU))
    return U, Dinv


def _B(Dinv, dims, g, q, t):
    """Matrix of the bilinear L(g, t, q) = eta^dag B eta  with s = Dinv eta."""
    from oracle.gamma import gamma_list
    ph = loops.phases(dims, [MOMS4[q]])[0]
    sel = np.zeros_like(ph)
    sel[t] = ph[t]
    P = np.kron(np.diag(sel.reshape(-1)), np.kron(gamma_list()[g], np.eye(3)))
    return P @ Dinv


@pytest.mark.parametrize("kind", [4, 2])
def test_per_source_mean_and_exact_variance(kind):
    dims = (2, 2, 2, 2)
    U, Dinv = _dense_setup(dims, 0.3, 101)
    n = 4096
    vals = []
    for j in range(n):
        eta = philox.noise(777, j, dims, kind)
        s = (Dinv @ eta.reshape(-1)).reshape(eta.shape)
        vals.append(loops.local_loops(eta, s, dims, ALL_G, MOMS4))
    vals = np.array(vals)
    exact = loops.exact_loops(Dinv, dims, ALL_G, MOMS4)
    for (g, q, t) in [(0, 0, 0), (5, 1, 1), (3, 2, 0), (8, 3, 1), (13, 0, 1), (4, 0, 0)]:
        B = _B(Dinv, dims, g, q, t)
        assert np.isclose(np.trace(B), exact[g, q, t], atol=1e-12)
        off = ~np.eye(B.shape[0], dtype=bool)
        if kind == 4:
            var = np.sum(np.abs(B[off]) ** 2)
        else:
            var = np.sum(np.abs(B[off]) ** 2 + (B * B.T.conj())[off]).real
        v = vals[:, g, q, t]
        sample_var = np.mean(np.abs(v - v.mean()) ** 2) * n / (n - 1)
        assert abs(sample_var / var - 1.0) < 0.12
        assert abs(v.mean() - exact[g, q, t]) < 4.5 * np.sqrt(var / n)


def test_one_over_sqrt_n_convergence():
    dims = (2, 2, 2, 2)
    U, Dinv = _dense_setup(dims, 0.3, 111)
    exact = loops.exact_loops(Dinv, dims, [0], [(0, 0, 0)])[0, 0].sum()
    ns = [16, 64, 256, 1024]
    rms = []
    for n in ns:
        errs = []
        for seed in range(32):
            acc = 0.0
            for j in range(n):
                eta = philox.noise(5000 + seed, j, dims, 4)
                s = (Dinv @ eta.reshape(-1)).reshape(eta.shape)
                acc += loops.local_loops(eta, s, dims, [0], [(0, 0, 0)])[0, 0].sum()
            errs.append(abs(acc / n - exact))
        rms.append(np.sqrt(np.mean(np.square(errs))))
    slope = np.polyfit(np.log(ns), np.log(rms), 1)[0]
    assert abs(slope + 0.5) < 0.1


def test_local_loops_gauge_invariant():
    dims = (4, 2, 2, 4)
    U = S.gauge_field(dims, 0.3, 121)
    G = S.gauge_transform(dims, 122)
    UG = S.transform_links(U, G)
    eta = philox.noise(9, 0, dims, 4)
    s, _, _, _ = solver.solve_full(U, eta, dims, KAPPA, MU, 1e-12, 3000)
    etag = S.transform_spinor(eta, G)
    sg, _, _, _ = solver.solve_full(UG, etag, dims, KAPPA, MU, 1e-12, 3000)
    a = loops.local_loops(eta, s, dims, ALL_G, MOMS4)
    b = loops.local_loops(etag, sg, dims, ALL_G, MOMS4)
    assert np.abs(a - b).max() < 1e-9 * np.abs(a).max()


def test_tsm_combine_definition_cases():
    rng = np.random.default_rng(0)
    corr = rng.standard_normal((5, 3)) + 1j * rng.standard_normal((5, 3))
    lp = rng.standard_normal((40, 3)) + 1j * rng.standard_normal((40, 3))
    est, err = loops.tsm_combine(corr, lp)
    assert np.allclose(est, corr.mean(0) + lp.mean(0))
    # zero correction (LP exact) leaves the plain stochastic mean
    est0, err0 = loops.tsm_combine(np.zeros((5, 3)), lp)
    assert np.allclose(est0, lp.mean(0))
    # complex variance = variance of the real part + variance of the imaginary part
    v_lp = np.var(lp.real, axis=0, ddof=1) + np.var(lp.imag, axis=0, ddof=1)
    v_c = np.var(corr.real, axis=0, ddof=1) + np.var(corr.imag, axis=0, ddof=1)
    assert np.allclose(err0, np.sqrt(v_lp / 40))
    assert np.allclose(err, np.sqrt(v_c / 5 + v_lp / 40))
    # a constant per-source value has zero error
    _, errc = loops.tsm_combine(np.ones((5, 3)), np.ones((40, 3)))
    assert np.all(errc == 0)


@pytest.mark.slow
def test_tsm_removes_truncation_bias_and_error_is_honest():
    dims = (2, 2, 2, 2)
    U, Dinv = _dense_setup(dims, 0.3, 131)
    exact = loops.exact_loops(Dinv, dims, [0, 5], [(0, 0, 0)])
    n_hp, n_lp, runs = 8, 32, 40
    est, errs, lp_means = [], [], []
    for r in range(runs):
        out = loops.tsm_loops(U, dims, KAPPA, MU, 9000 + r, 4, n_hp, n_lp,
                              (1e-12, 4000), (0.0, 2), [0, 5], [(0, 0, 0)])
        est.append(out['loops'])
        errs.append(out['err'])
        lp_means.append(out['lp_mean'])
    est, errs, lp_means = np.array(est), np.array(errs), np.array(lp_means)
    # LP-only mean (2 CG iterations) is biased: its scatter cannot explain its offset
    lp_off = np.abs(lp_means.mean(0) - exact)
    lp_sd = lp_means.std(0) / np.sqrt(runs)
    assert np.any(lp_off > 8 * lp_sd)
    # TSM mean over runs agrees with the exact loop
    off = np.abs(est.mean(0) - exact)
    sd = np.sqrt(np.mean(errs ** 2, axis=0) / runs)
    assert np.all(off < 4 * sd)
    # the stated error matches the actual scatter of independent runs
    scatter = np.sqrt(np.mean(np.abs(est - exact) ** 2, axis=0))
    ratio = scatter / np.sqrt(np.mean(errs ** 2, axis=0))
    assert np.all((ratio > 0.6) & (ratio < 1.5))


@pytest.mark.slow
def test_config0_tsm_against_dense_inverse_4x4x4x4():
    """4^4 lattice (V = 256), eps = 0.3, kappa = 0.124, mu = 0.01, Z4 noise,
    N_HP = 4 at 1e-12, N_LP = 64 at 1e-2, 16 Gammas x 4 momenta: the TSM
    estimate agrees with Tr[Gamma D^-1] within its stated error."""
    dims = (4, 4, 4, 4)
    U, Dinv = _dense_setup(dims, 0.3, 1)
    exact = loops.exact_loops(Dinv, dims, ALL_G, MOMS4)
    out = loops.tsm_loops(U, dims, KAPPA, MU, 2024, 4, 4, 64, (1e-12, 5000), (1e-2, 5000),
                          ALL_G, MOMS4)
    z = np.abs(out['loops'] - exact) / out['err']
    assert np.isfinite(z).all()
    assert np.median(z) < 1.5 and np.max(z) < 6.0
    # HP solves reached the requested residual, LP solves were truncated early
    assert max(out['lp_iters']) < min(out['hp_iters'])


def test_fft_loops_equal_direct_phase_sums():
    """Every momentum at once (FFT) against the direct phase sums of
    local_loops, including negative momenta (index L - n)."""
    dims = (4, 2, 6, 4)
    rng = np.random.default_rng(31)
    eta = philox.noise(5, 2, dims, 4)
    s = rng.standard_normal(eta.shape) + 1j * rng.standard_normal(eta.shape)
    gam = [0, 3, 5, 12]
    allq = loops.fft_loops(eta, s, dims, gam)
    moms = [(0, 0, 0), (1, 0, 0), (-1, 1, 2), (3, 1, -5), (2, 0, 3)]
    direct = loops.local_loops(eta, s, dims, gam, moms)
    for k, (nx, ny, nz) in enumerate(moms):
        got = allq[:, :, nz % dims[2], ny % dims[1], nx % dims[0]]
        assert np.abs(got - direct[:, k, :]).max() < 1e-12 * np.abs(direct).max()
