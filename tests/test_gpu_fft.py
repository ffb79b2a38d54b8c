"""Loops at every spatial momentum (batched 3-D FFT per source) on the GPU.

* One source: against oracle.loops.fft_loops, 1e-12 relative in FP64 and
  1e-5 in FP32, also in the difference form (a - b), on extents whose
  factorisations take every butterfly of the library's FFT (radix 4, 2, 3
  and the direct DFT of another prime: 10 = 2 * 5, 14 = 2 * 7) and on a
  24^3 spatial volume (the production extent, 4 * 2 * 3).
* A plane too large for shared memory, or an extent with a prime factor
  above 13, is refused with TSM_ERR_TOO_LARGE before any launch.
* The whole TSM with all momenta (running means and variances in source
  order) equals, at sampled momenta, the TSM with those momenta projected
  by direct phase sums: estimate to 1e-10, error to 1e-8 in FP64 (two-pass
  versus running variance); 1e-5 and 1e-4 in the mixed tier, whose FP32
  batch sums over 32 sources (of each value minus the batch's first one)
  are merged into FP64 moments.
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


@pytest.mark.parametrize("dims", [DIMS, (10, 12, 14, 2), (24, 24, 24, 2)])
@pytest.mark.parametrize("prec,tol", [(tsm.TSM_F64, 1e-12), (tsm.TSM_F32, 1e-5)])
def test_contract_fft_matches_oracle(ctx, prec, tol, dims):
    ctx.load_gauge(S.gauge_field(dims, 0.3, 2), dims, KAPPA, MU)
    s = S.random_spinor(dims, 3)
    b = S.random_spinor(dims, 4)
    eta = philox.noise(11, 6, dims, 4)
    gam = GAM if dims == DIMS else list(range(16))
    got = ctx.contract_fft(11, 6, s, gam, prec=prec)
    assert _rel(got, oloops.fft_loops(eta, s, dims, gam)) < tol
    got = ctx.contract_fft(11, 6, s, gam, s_b=b, prec=prec)
    assert _rel(got, oloops.fft_loops(eta, s - b, dims, gam)) < tol


def test_contract_fft_plane_too_large(ctx):
    dims = (128, 128, 2, 2)    # an FP64 128 x 128 plane needs 256 KB of shared memory
    ctx.load_gauge(S.gauge_field(dims, 0.0, 0), dims, KAPPA, MU)
    s = S.random_spinor(dims, 1)
    with pytest.raises(tsm.TsmError) as e:
        ctx.contract_fft(1, 0, s, [0], prec=tsm.TSM_F64)
    assert e.value.status == -9   # TSM_ERR_TOO_LARGE
    dims = (34, 2, 2, 2)       # 34 = 2 * 17: a prime factor above the largest butterfly (13)
    ctx.load_gauge(S.gauge_field(dims, 0.0, 0), dims, KAPPA, MU)
    with pytest.raises(tsm.TsmError) as e:
        ctx.contract_fft(1, 0, S.random_spinor(dims, 1), [0], prec=tsm.TSM_F32)
    assert e.value.status == -9


@pytest.mark.parametrize("tier", ["fp64", "mixed"])
def test_all_momenta_tsm_matches_direct_projection(ctx, tier):
    U = S.gauge_field(DIMS, 0.3, 5)
    ctx.load_gauge(U, DIMS, KAPPA, MU)
    if tier == "fp64":
        hp, lp = tsm.stop(1e-12, 5000, tsm.TSM_F64), tsm.stop(0.0, 4, tsm.TSM_F64)
    else:
        hp, lp = tsm.stop(1e-10, 5000, tsm.TSM_F32, reliable=True), tsm.stop(5e-3, 60, tsm.TSM_F16)
    moms = [(0, 0, 0), (1, 0, 0), (-1, 2, 1), (3, -1, 0)]
    # mixed tier: 70 LP-set sources, so the FP32 batch sums of the projection
    # are merged into the FP64 moments twice mid-run (after 32 and 64) and once
    # at the end
    n_lp = 7 if tier == "fp64" else 70
    direct = ctx.loops(13, 4, 3, n_lp, hp, lp, GAM, moms, batch=4)
    allq = ctx.loops(13, 4, 3, n_lp, hp, lp, GAM, None, batch=4, all_momenta=True)
    tol_est, tol_err = (1e-10, 1e-8) if tier == "fp64" else (1e-5, 1e-4)
    for k, (nx, ny, nz) in enumerate(moms):
        i = (slice(None), slice(None), nz % DIMS[2], ny % DIMS[1], nx % DIMS[0])
        assert _rel(allq["loops"][i], direct["loops"][:, k, :]) < tol_est
        assert _rel(allq["err"][i], direct["err"][:, k, :]) < tol_err
