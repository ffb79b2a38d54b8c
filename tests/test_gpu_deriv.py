"""One-derivative insertions on the GPU against the oracle.

* Per-source contraction on random fields (and the difference form) against
  oracle.loops.deriv_loops: 1e-12 relative in FP64, 1e-5 in FP32.
* tsm_loops with local + derivative blocks on the FP64 path against the
  oracle's TSM to 1e-9 (LP truncated at a fixed iteration count); the local
  block is unchanged by asking for derivatives.
* The estimate agrees with the loop built term by term from the operator's
  blocks and a dense inverse, within its error.
"""
import numpy as np
import pytest

from oracle import dirac, loops as oloops, philox
from paper_1211_0126_gb300 import synthetic as S
from paper_1211_0126_gb300 import tsm

pytestmark = pytest.mark.gpu

DIMS = (4, 4, 2, 4)
KAPPA, MU = 0.124, 0.02
GAM = list(range(16))
MOMS = S.default_momenta(4)


def _rel(a, b):
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


@pytest.fixture(scope="module")
def field():
    return S.gauge_field(DIMS, 0.3, 8)


@pytest.mark.parametrize("prec,tol", [(tsm.TSM_F64, 1e-12), (tsm.TSM_F32, 1e-5)])
@pytest.mark.parametrize("mask,mus", [(0b1111, [0, 1, 2, 3]), (0b1010, [1, 3])])
def test_contract_deriv_matches_oracle(ctx, field, prec, tol, mask, mus):
    ctx.load_gauge(field, DIMS, KAPPA, MU)
    s = S.random_spinor(DIMS, 5)
    b = S.random_spinor(DIMS, 6)
    eta = philox.noise(17, 3, DIMS, 4)
    got = ctx.contract_deriv(17, 3, s, GAM, mask, MOMS, prec=prec)
    want = np.transpose(oloops.deriv_loops(field, eta, s, DIMS, GAM, mus, MOMS), (1, 0, 2, 3))
    assert _rel(got, want) < tol
    got = ctx.contract_deriv(17, 3, s, GAM, mask, MOMS, s_b=b, prec=prec)
    want = np.transpose(oloops.deriv_loops(field, eta, s - b, DIMS, GAM, mus, MOMS), (1, 0, 2, 3))
    assert _rel(got, want) < tol


def test_fp64_tsm_with_derivatives_matches_oracle(ctx, field):
    ctx.load_gauge(field, DIMS, KAPPA, MU)
    hp, lp = (1e-12, 5000), (0.0, 5)
    got = ctx.loops(23, 4, 3, 10, tsm.stop(*hp, tsm.TSM_F64), tsm.stop(*lp, tsm.TSM_F64), GAM, MOMS,
                    per_source=True, deriv_mask=0b1001)
    want = oloops.tsm_loops(field, DIMS, KAPPA, MU, 23, 4, 3, 10, hp, lp, GAM, MOMS, deriv_mus=(0, 3))
    assert got["loops"].shape == (3, 16, 4, DIMS[3])
    assert _rel(got["per_lp"], want["lp"]) < 1e-9
    assert _rel(got["per_corr"], want["corr"]) < 1e-8
    assert _rel(got["loops"], want["loops"]) < 1e-9
    assert _rel(got["err"], want["err"]) < 1e-8
    plain = ctx.loops(23, 4, 3, 10, tsm.stop(*hp, tsm.TSM_F64), tsm.stop(*lp, tsm.TSM_F64), GAM, MOMS)
    assert np.array_equal(plain["loops"], got["loops"][0])


def test_deriv_tsm_against_dense(ctx, field):
    ctx.load_gauge(field, DIMS, KAPPA, MU)
    iu = np.linalg.inv(dirac.dense_dtm(field, DIMS, KAPPA, MU))
    exact = oloops.exact_deriv_loops(field, iu, DIMS, GAM, [2, 3], MOMS)
    got = ctx.loops(91, 4, 8, 128, tsm.stop(1e-12, 5000, tsm.TSM_F64), tsm.stop(1e-2, 5000, tsm.TSM_F64),
                    GAM, MOMS, deriv_mask=0b1100)
    est = np.transpose(got["loops"][1:], (1, 0, 2, 3))
    err = np.transpose(got["err"][1:], (1, 0, 2, 3))
    # entries whose stochastic error vanishes (err ~ 1e-16) are compared at the
    # FP64 rounding level of the whole array
    z = np.abs(est - exact) / (err + 1e-10 * np.abs(exact).max())
    assert np.median(z) < 1.5 and z.max() < 6.0
