"""One-end-trick loops (Sec. 2.3, Eq. 2.5) on the GPU against the oracle.

* The per-source contraction on random fields (single and difference form)
  equals oracle.loops.one_end_loops to 1e-12 relative in FP64 and 1e-5 in FP32.
* tsm_loops with estimator = 1 on the FP64 path reproduces the oracle's TSM
  estimate, error and per-source values to 1e-9 relative (LP truncated at a
  fixed iteration count).
* The estimate agrees with the exact isovector loop Tr[P Gamma (D_u^-1 - D_d^-1)]
  from two dense inverses within its error, and the mixed-precision path
  (FP32 + FP64 reliable HP, FP16 LP) agrees with the FP64 path within the
  stochastic error.
"""
import numpy as np
import pytest

from oracle import dirac, loops as oloops
from paper_1211_0126_gb300 import synthetic as S
from paper_1211_0126_gb300 import tsm

pytestmark = pytest.mark.gpu

DIMS = (4, 4, 4, 4)
KAPPA, MU = 0.124, 0.03
GAM = list(range(16))
MOMS = S.default_momenta(4)


def _rel(a, b):
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


@pytest.fixture(scope="module")
def field():
    return S.gauge_field(DIMS, 0.3, 5)


@pytest.mark.parametrize("prec,tol", [(tsm.TSM_F64, 1e-12), (tsm.TSM_F32, 1e-5)])
def test_contract_one_end_matches_oracle(ctx, field, prec, tol):
    ctx.load_gauge(field, DIMS, KAPPA, MU)
    a = S.random_spinor(DIMS, 1)
    b = a + 0.01 * S.random_spinor(DIMS, 2)
    got = ctx.contract_one_end(a, GAM, MOMS, prec=prec)
    want = oloops.one_end_loops(a, DIMS, KAPPA, MU, GAM, MOMS)
    assert _rel(got, want) < tol
    got = ctx.contract_one_end(a, GAM, MOMS, s_b=b, prec=prec)
    want = want - oloops.one_end_loops(b, DIMS, KAPPA, MU, GAM, MOMS)
    assert _rel(got, want) < tol * 10


def test_fp64_one_end_tsm_matches_oracle(ctx, field):
    ctx.load_gauge(field, DIMS, KAPPA, MU)
    hp, lp = (1e-12, 5000), (0.0, 5)
    got = ctx.loops(41, 4, 4, 16, tsm.stop(*hp, tsm.TSM_F64), tsm.stop(*lp, tsm.TSM_F64), GAM, MOMS,
                    per_source=True, estimator=1)
    want = oloops.tsm_loops(field, DIMS, KAPPA, MU, 41, 4, 4, 16, hp, lp, GAM, MOMS, estimator='one_end')
    assert _rel(got["per_lp"], want["lp"]) < 1e-9
    assert _rel(got["per_corr"], want["corr"]) < 1e-8
    assert _rel(got["loops"], want["loops"]) < 1e-9
    assert _rel(got["err"], want["err"]) < 1e-8


def test_one_end_tsm_against_dense_and_mixed(ctx, field):
    ctx.load_gauge(field, DIMS, KAPPA, MU)
    iu = np.linalg.inv(dirac.dense_dtm(field, DIMS, KAPPA, MU))
    idd = np.linalg.inv(dirac.dense_dtm(field, DIMS, KAPPA, -MU))
    exact = oloops.exact_loops(iu - idd, DIMS, GAM, MOMS)
    ref = ctx.loops(77, 4, 8, 96, tsm.stop(1e-12, 5000, tsm.TSM_F64), tsm.stop(1e-2, 5000, tsm.TSM_F64),
                    GAM, MOMS, estimator=1)
    z = np.abs(ref["loops"] - exact) / (ref["err"] + 1e-300)
    assert np.median(z) < 1.5 and z.max() < 6.0
    mixed = ctx.loops(77, 4, 8, 96, tsm.stop(1e-10, 5000, tsm.TSM_F32, reliable=True),
                      tsm.stop(1e-2, 60, tsm.TSM_F16), GAM, MOMS, batch=8, estimator=1)
    # same noise on both sides: every entry within 0.1 of the FP64 path's error
    zm = np.abs(mixed["loops"] - ref["loops"]) / ref["err"]
    print("one-end mixed: |L_mixed - L_FP64| / sigma_FP64: max %.3g, median %.3g" % (zm.max(), np.median(zm)))
    assert zm.max() <= 0.1


# ---- generalised one-end trick (Eq. 2.6): isoscalar u + d

@pytest.mark.parametrize("prec,tol", [(tsm.TSM_F64, 1e-12), (tsm.TSM_F32, 1e-5)])
def test_contract_gen_one_end_matches_oracle(ctx, field, prec, tol):
    ctx.load_gauge(field, DIMS, KAPPA, MU)
    a = S.random_spinor(DIMS, 3)
    b = a + 0.01 * S.random_spinor(DIMS, 4)
    want = oloops.gen_one_end_loops(field, a, DIMS, KAPPA, GAM, MOMS)
    assert _rel(ctx.contract_gen_one_end(a, GAM, MOMS, prec=prec), want) < tol
    want = want - oloops.gen_one_end_loops(field, b, DIMS, KAPPA, GAM, MOMS)
    assert _rel(ctx.contract_gen_one_end(a, GAM, MOMS, s_b=b, prec=prec), want) < tol * 100


def test_fp64_gen_one_end_tsm_matches_oracle_and_dense(ctx, field):
    ctx.load_gauge(field, DIMS, KAPPA, MU)
    hp, lp = (1e-12, 5000), (0.0, 5)
    got = ctx.loops(43, 4, 4, 12, tsm.stop(*hp, tsm.TSM_F64), tsm.stop(*lp, tsm.TSM_F64), GAM, MOMS,
                    per_source=True, estimator=2)
    want = oloops.tsm_loops(field, DIMS, KAPPA, MU, 43, 4, 4, 12, hp, lp, GAM, MOMS, estimator='gen_one_end')
    assert _rel(got["per_lp"], want["lp"]) < 1e-9
    assert _rel(got["per_corr"], want["corr"]) < 1e-8
    assert _rel(got["loops"], want["loops"]) < 1e-9
    iu = np.linalg.inv(dirac.dense_dtm(field, DIMS, KAPPA, MU))
    idd = np.linalg.inv(dirac.dense_dtm(field, DIMS, KAPPA, -MU))
    exact = oloops.exact_loops(iu + idd, DIMS, GAM, MOMS)
    est = ctx.loops(79, 4, 8, 160, tsm.stop(1e-12, 5000, tsm.TSM_F64), tsm.stop(1e-2, 5000, tsm.TSM_F64),
                    GAM, MOMS, estimator=2)
    z = np.abs(est["loops"] - exact) / (est["err"] + 1e-300)
    assert np.median(z) < 1.5 and z.max() < 6.0
