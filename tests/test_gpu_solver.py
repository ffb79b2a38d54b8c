"""GPU solves against the oracle: CG iterates (fixed iteration count), HP
solves against dense inversion, the precision tiers, the stopping rule."""
import numpy as np
import pytest

from oracle import dirac, solver
from paper_1211_0126_gb300 import synthetic as S
from paper_1211_0126_gb300 import tsm

pytestmark = pytest.mark.gpu

KAPPA, MU = 0.124, 0.01


def _rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


@pytest.mark.parametrize("dims", [(4, 4, 4, 4), (6, 4, 4, 6), (2, 2, 2, 2)])
def test_fixed_iteration_cg_matches_oracle_fp64(ctx, dims):
    U = S.gauge_field(dims, 0.3, 31)
    ctx.load_gauge(U, dims, KAPPA, MU)
    b = S.random_spinor(dims, 32)
    for n in (1, 7, 25):
        s, iters, tres, st = ctx.solve(b, tsm.stop(0.0, n, tsm.TSM_F64))
        want, it_o, _, tr_o = solver.solve_full(U, b, dims, KAPPA, MU, 0.0, n)
        assert iters[0] == it_o == n
        assert _rel(s, want) < 1e-11
        assert abs(tres[0] - tr_o) < 1e-9 * max(tr_o, 1e-3)


def test_hp_solve_against_dense_inverse(ctx):
    dims = (4, 4, 4, 4)
    U = S.gauge_field(dims, 0.3, 41)
    ctx.load_gauge(U, dims, KAPPA, MU)
    b = S.random_spinor(dims, 42)
    D = dirac.dense_dtm(U, dims, KAPPA, MU)
    x = np.linalg.solve(D, b.reshape(-1)).reshape(b.shape)
    s, iters, tres, st = ctx.solve(b, tsm.stop(1e-12, 5000, tsm.TSM_F64))
    _, it_o, _, _ = solver.solve_full(U, b, dims, KAPPA, MU, 1e-12, 5000)
    assert st == 0 and abs(int(iters[0]) - it_o) <= 1
    assert tres[0] < 1e-10 and _rel(s, x) < 1e-9
    # FP32 iterations with FP64 reliable updates reach 1e-10
    s32, it32, tr32, st32 = ctx.solve(b, tsm.stop(1e-10, 5000, tsm.TSM_F32, reliable=True))
    assert st32 == 0 and tr32[0] < 1e-8 and _rel(s32, x) < 1e-7


@pytest.mark.parametrize("prec,tol", [(tsm.TSM_F32, 1e-4), (tsm.TSM_F16, 5e-3), (tsm.TSM_BF16, 5e-3)])
def test_low_precision_tiers_truncated(ctx, prec, tol):
    dims = (6, 4, 4, 6)
    U = S.gauge_field(dims, 0.3, 51)
    ctx.load_gauge(U, dims, KAPPA, MU)
    b = S.random_spinor(dims, 52)
    s, iters, tres, st = ctx.solve(b, tsm.stop(tol, 500, prec))
    assert st == 0, "solve did not reach its truncation residual"
    want, it_o, _, _ = solver.solve_full(U, b, dims, KAPPA, MU, tol, 500)
    # same stopping rule on the same system: iteration counts agree closely,
    # the solutions agree to the truncation level
    assert abs(int(iters[0]) - it_o) <= max(2, it_o // 5)
    x = solver.solve_full(U, b, dims, KAPPA, MU, 1e-13, 5000)[0]
    assert _rel(s, x) < 20 * tol
    assert tres[0] < 20 * tol


def test_batch_of_sources_and_zero_source(ctx):
    dims = (4, 4, 4, 4)
    U = S.gauge_field(dims, 0.3, 61)
    ctx.load_gauge(U, dims, KAPPA, MU)
    b = S.random_spinor(dims, 62, batch=(3,))
    b[1] = 0.0
    s, iters, tres, st = ctx.solve(b, tsm.stop(1e-10, 2000, tsm.TSM_F64))
    assert iters[1] == 0 and np.all(s[1] == 0)
    for r in (0, 2):
        want = solver.solve_full(U, b[r], dims, KAPPA, MU, 1e-10, 2000)[0]
        assert _rel(s[r], want) < 1e-8


def test_not_converged_status(ctx):
    dims = (4, 4, 4, 4)
    ctx.load_gauge(S.gauge_field(dims, 0.3, 71), dims, KAPPA, MU)
    b = S.random_spinor(dims, 72)
    s, iters, tres, st = ctx.solve(b, tsm.stop(1e-12, 3, tsm.TSM_F64))
    assert st == tsm.TSM_ERR_NOT_CONVERGED and iters[0] == 3


def test_production_lattice_solve(ctx):
    """24^3 x 48 with the benchmark's physics (eps = 0.25, kappa = 0.1245,
    mu = 0.005): one LP solve (FP16, 5e-3 / 60 iterations) and the oracle's
    full-lattice operator checks its true residual."""
    dims = (24, 24, 24, 48)
    U = S.gauge_field(dims, 0.25, 3)
    ctx.load_gauge(U, dims, 0.1245, 0.005)
    from oracle import philox
    b = philox.noise(1000, 0, dims, 4)
    s, iters, tres, st = ctx.solve(b, tsm.stop(5e-3, 60, tsm.TSM_F16))
    r = b - dirac.dtm(U, s, dims, 0.1245, 0.005)
    true_res = np.linalg.norm(r) / np.linalg.norm(b)
    assert abs(true_res - tres[0]) < 1e-6 * max(true_res, 1e-3)
    assert 0 < iters[0] <= 60 and true_res < 1.0


@pytest.mark.parametrize("prec,reliable", [(tsm.TSM_F64, False), (tsm.TSM_F32, True), (tsm.TSM_F16, False),
                                           (tsm.TSM_BF16, False), (tsm.TSM_F32, False)])
def test_batched_solve_bit_identical_to_single(ctx, prec, reliable):
    """Multi-RHS kernels (one launch over every right-hand side still iterating,
    converged ones dropped) give exactly the single-source results."""
    dims = (6, 4, 4, 6)
    U = S.gauge_field(dims, 0.3, 91)
    ctx.load_gauge(U, dims, KAPPA, MU)
    b = S.random_spinor(dims, 92, batch=(5,))
    b[2] *= 1e-3                     # different scales -> different iteration counts
    b[3] = 0.0                       # converged before the first iteration
    stp = tsm.stop(1e-9 if prec in (tsm.TSM_F64,) or reliable else 5e-3, 400, prec, reliable=reliable)
    s_b, it_b, tr_b, _ = ctx.solve(b, stp)
    for r in range(5):
        s_1, it_1, tr_1, _ = ctx.solve(b[r], stp)
        assert it_b[r] == it_1[0]
        assert np.array_equal(s_b[r], s_1), r
    assert it_b[3] == 0
