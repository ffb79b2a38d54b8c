"""Loops at every spatial momentum (batched 3-D FFT per source) on the GPU.

* One source: against oracle.loops.fft_loops, 1e-12 relative in FP64 and
  1e-5 in FP32, also in the difference form (a - b).
* The whole TSM with all momenta (running means and variances in source
  order) equals, at sampled momenta, the TSM with those momenta projected
  by direct phase sums: estimate to 1e-10, error to 1e-8 (two-pass versus
  running variance).
"""
import numpy as np
import pytest

from oracle import loops as oloops, philox
from paper_1211_0126_gb300 import synthetic as S
from paper_1211_0126_gb300 import tsm

pytestmark = pytest.mark.gpu

DIMS = (4, 6, 2, 4)
KAPPA, MU = 0.124, 0.01
GAM = [0, 1, 5, 9, 15]


def _rel(a, b):
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


@pytest.mark.parametrize("prec,tol", [(tsm.TSM_F64, 1e-12), (tsm.TSM_F32, 1e-5)])
def test_contract_fft_matches_oracle(ctx, prec, tol):
    ctx.load_gauge(S.gauge_field(DIMS, 0.3, 2), DIMS, KAPPA, MU)
    s = S.random_spinor(DIMS, 3)
    b = S.random_spinor(DIMS, 4)
    eta = philox.noise(11, 6, DIMS, 4)
    got = ctx.contract_fft(11, 6, s, GAM, prec=prec)
    assert _rel(got, oloops.fft_loops(eta, s, DIMS, GAM)) < tol
    got = ctx.contract_fft(11, 6, s, GAM, s_b=b, prec=prec)
    assert _rel(got, oloops.fft_loops(eta, s - b, DIMS, GAM)) < tol


@pytest.mark.parametrize("tier", ["fp64", "mixed"])
def test_all_momenta_tsm_matches_direct_projection(ctx, tier):
    U = S.gauge_field(DIMS, 0.3, 5)
    ctx.load_gauge(U, DIMS, KAPPA, MU)
    if tier == "fp64":
        hp, lp = tsm.stop(1e-12, 5000, tsm.TSM_F64), tsm.stop(0.0, 4, tsm.TSM_F64)
    else:
        hp, lp = tsm.stop(1e-10, 5000, tsm.TSM_F32, reliable=True), tsm.stop(5e-3, 60, tsm.TSM_F16)
    moms = [(0, 0, 0), (1, 0, 0), (-1, 2, 1), (3, -1, 0)]
    direct = ctx.loops(13, 4, 3, 7, hp, lp, GAM, moms, batch=4)
    allq = ctx.loops(13, 4, 3, 7, hp, lp, GAM, None, batch=4, all_momenta=True)
    tol_est, tol_err = (1e-10, 1e-8) if tier == "fp64" else (1e-5, 1e-4)
    for k, (nx, ny, nz) in enumerate(moms):
        i = (slice(None), slice(None), nz % DIMS[2], ny % DIMS[1], nx % DIMS[0])
        assert _rel(allq["loops"][i], direct["loops"][:, k, :]) < tol_est
        assert _rel(allq["err"][i], direct["err"][:, k, :]) < tol_err
