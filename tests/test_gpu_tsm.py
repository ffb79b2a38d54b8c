"""The whole TSM path on the GPU against the oracle.

4^4 lattice as in the plain FP64 workload: eps = 0.3, kappa = 0.124, mu = 0.01,
antiperiodic t, Z4 noise, all 16 insertions at 4 momenta.  The FP64 GPU path
reproduces the oracle's estimate, error, LP-only mean, correction mean and
per-source loops to 1e-9 relative (LP truncation by a fixed iteration count,
so both sides run exactly the same iterations; and by the 1e-2 residual rule,
where the iteration counts must agree).  Splitting the source ranges over
several calls and combining gives bit-identical results.  The estimate agrees
with Tr[Gamma D^-1] from dense inversion within its error.
"""
import numpy as np
import pytest

from oracle import dirac, loops as oloops
from paper_1211_0126_gb300 import synthetic as S
from paper_1211_0126_gb300 import tsm

pytestmark = pytest.mark.gpu

DIMS = (4, 4, 4, 4)
KAPPA, MU = 0.124, 0.01
GAM = list(range(16))
MOMS = S.default_momenta(4)


@pytest.fixture(scope="module")
def field():
    return S.gauge_field(DIMS, 0.3, 1)


def _close(a, b, rel=1e-9):
    scale = max(np.abs(b).max(), 1e-300)
    return np.abs(a - b).max() <= rel * scale


@pytest.mark.parametrize("lp_rule", ["fixed", "residual"])
def test_fp64_tsm_matches_oracle(ctx, field, lp_rule):
    n_hp, n_lp = 4, 64 if lp_rule == "residual" else 24
    lp = (0.0, 6) if lp_rule == "fixed" else (1e-2, 5000)
    hp = (1e-12, 5000)
    ctx.load_gauge(field, DIMS, KAPPA, MU)
    got = ctx.loops(2024, 4, n_hp, n_lp, tsm.stop(*hp, tsm.TSM_F64), tsm.stop(*lp, tsm.TSM_F64), GAM, MOMS,
                    per_source=True)
    want = oloops.tsm_loops(field, DIMS, KAPPA, MU, 2024, 4, n_hp, n_lp, hp, lp, GAM, MOMS)
    assert got["stats"]["lp_iters"] == sum(want["lp_iters"])
    assert abs(got["stats"]["hp_iters"] - sum(want["hp_iters"])) <= n_hp
    assert _close(got["per_lp"], want["lp"])
    assert _close(got["per_corr"], want["corr"], 1e-8)
    assert _close(got["loops"], want["loops"])
    assert _close(got["lp_mean"], want["lp_mean"])
    assert _close(got["corr_mean"], want["corr_mean"], 1e-8)
    assert _close(got["err"], want["err"], 1e-8)
    assert got["stats"]["hp_max_true_res"] < 1e-10


def test_tsm_against_dense_inverse(ctx, field):
    ctx.load_gauge(field, DIMS, KAPPA, MU)
    exact = oloops.exact_loops(np.linalg.inv(dirac.dense_dtm(field, DIMS, KAPPA, MU)), DIMS, GAM, MOMS)
    got = ctx.loops(77, 4, 4, 64, tsm.stop(1e-12, 5000, tsm.TSM_F64), tsm.stop(1e-2, 5000, tsm.TSM_F64),
                    GAM, MOMS)
    z = np.abs(got["loops"] - exact) / got["err"]
    assert np.median(z) < 1.5 and z.max() < 6.0


def test_split_source_ranges_bit_identical(ctx, field):
    ctx.load_gauge(field, DIMS, KAPPA, MU)
    hp, lp = tsm.stop(1e-10, 5000, tsm.TSM_F64), tsm.stop(1e-2, 5000, tsm.TSM_F64)
    full = ctx.loops(5, 4, 4, 12, hp, lp, GAM, MOMS, per_source=True)
    parts = [ctx.loops(5, 4, 0, 0, hp, lp, GAM, MOMS, hp_range=h, lp_range=l, per_source=True)
             for h, l in [((0, 1), (4, 9)), ((1, 4), (9, 16))]]
    pc = np.concatenate([p["per_corr"] for p in parts])
    pl = np.concatenate([p["per_lp"] for p in parts])
    assert np.array_equal(pc, full["per_corr"]) and np.array_equal(pl, full["per_lp"])
    comb = ctx.combine(pc, pl)
    for k in ("loops", "err", "lp_mean", "corr_mean"):
        assert np.array_equal(comb[k], full[k]), k


@pytest.mark.parametrize("tiers", ["mixed16", "mixedbf16", "fp32"])
def test_mixed_precision_tsm_within_tenth_sigma(ctx, field, tiers):
    """HP: FP32 + FP64 reliable updates to 1e-10; LP: 16-bit (or FP32)
    storage at 5e-3.  Against the FP64 path with the same seed and the same
    stopping rules:
    * every entry of the estimate within 0.1 of the FP64 path's stochastic
      error (the bar the precision tiers must meet): both runs use the same
      noise, so the difference is the precision effect alone,
      mean_LP(dL) - mean_HP(dL) for the per-source LP differences dL;
    * every source's HP loop L(s_HP) = corr + L(s_LP) equal to the FP64 one
      to the HP tolerance (the LP loops of the HP-set sources come from a call
      whose LP set is those sources: the LP map does not depend on the set)."""
    ctx.load_gauge(field, DIMS, KAPPA, MU)
    lp_prec = {"mixed16": tsm.TSM_F16, "mixedbf16": tsm.TSM_BF16, "fp32": tsm.TSM_F32}[tiers]
    hp = tsm.stop(1e-10, 5000, tsm.TSM_F32, reliable=True)
    lp = tsm.stop(5e-3, 60, lp_prec)
    hp64, lp64 = tsm.stop(1e-12, 5000, tsm.TSM_F64), tsm.stop(5e-3, 60, tsm.TSM_F64)
    got = ctx.loops(11, 4, 8, 64, hp, lp, GAM, MOMS, per_source=True)
    ref = ctx.loops(11, 4, 8, 64, hp64, lp64, GAM, MOMS, per_source=True)
    assert got["stats"]["hp_not_converged"] == 0
    assert got["stats"]["hp_max_true_res"] < 1e-8
    dz = np.abs(got["loops"] - ref["loops"]) / ref["err"]
    print("%s: |L_mixed - L_FP64| / sigma_FP64: max %.3g, median %.3g" % (tiers, dz.max(), np.median(dz)))
    assert dz.max() <= 0.1
    # HP loops per source
    lp_of_hp = ctx.loops(11, 4, 0, 0, hp, lp, GAM, MOMS, hp_range=(0, 0), lp_range=(0, 8), per_source=True)
    lp_of_hp64 = ctx.loops(11, 4, 0, 0, hp64, lp64, GAM, MOMS, hp_range=(0, 0), lp_range=(0, 8), per_source=True)
    l_hp = got["per_corr"] + lp_of_hp["per_lp"]
    l_hp64 = ref["per_corr"] + lp_of_hp64["per_lp"]
    assert np.abs(l_hp - l_hp64).max() <= 1e-5 * np.abs(l_hp64).max()
    # and the per-source LP loops of the LP set agree to the LP precision
    assert np.abs(got["per_lp"] - ref["per_lp"]).max() <= 0.05 * np.abs(ref["per_lp"]).max()


@pytest.mark.parametrize("batch", [3, 8])
def test_batched_tsm_bit_identical(ctx, field, batch):
    """tsm_loops with multi-RHS batches equals the single-source run bit for bit
    (the LP map does not depend on which sources share a batch)."""
    ctx.load_gauge(field, DIMS, KAPPA, MU)
    hp = tsm.stop(1e-10, 5000, tsm.TSM_F32, reliable=True)
    lp = tsm.stop(5e-3, 60, tsm.TSM_F16)
    one = ctx.loops(31, 4, 4, 13, hp, lp, GAM, MOMS, per_source=True, batch=1)
    many = ctx.loops(31, 4, 4, 13, hp, lp, GAM, MOMS, per_source=True, batch=batch)
    for k in ("loops", "err", "per_corr", "per_lp"):
        assert np.array_equal(one[k], many[k]), k
    assert one["stats"]["lp_iters"] == many["stats"]["lp_iters"]


def test_hp_warm_start(ctx):
    """HP solves started from the LP solutions: the LP map and the LP-set loops
    are bit-identical to the zero-start run, every HP solution still meets the
    FP64 true-residual bar, each source's HP loop L(s_HP) = corr + L(s_LP)
    agrees with the zero-start one to the HP tolerance, and fewer HP iterations
    are needed.  6^3x8 so that the HP solves take enough iterations to show it."""
    dims = (6, 6, 6, 8)
    u = S.gauge_field(dims, 0.25, 3)
    ctx.load_gauge(u, dims, 0.1245, 0.005)
    moms = S.default_momenta(7)
    hp = tsm.stop(1e-10, 5000, tsm.TSM_F32, reliable=True, reliable_delta=1e-5)
    lp = tsm.stop(5e-3, 60, tsm.TSM_F16)
    cold = ctx.loops(41, 4, 6, 10, hp, lp, GAM, moms, per_source=True, batch=6)
    warm = ctx.loops(41, 4, 6, 10, hp, lp, GAM, moms, per_source=True, batch=6, hp_warm_start=True)
    assert np.array_equal(cold["per_lp"], warm["per_lp"])
    assert cold["stats"]["lp_iters"] == warm["stats"]["lp_iters"]
    assert warm["stats"]["hp_not_converged"] == 0
    assert warm["stats"]["hp_max_true_res"] < 1e-9
    # same LP solutions on both sides, so the difference of the corrections is
    # L(s_HP, zero start) - L(s_HP, LP start): the HP tolerance plus the FP32
    # rounding of the site sums of the contraction (216 sites per timeslice)
    diff = cold["per_corr"] - warm["per_corr"]
    assert np.abs(diff).max() <= 2e-6 * max(np.abs(cold["per_corr"]).max(), 1.0)
    assert warm["stats"]["hp_iters"] <= 0.95 * cold["stats"]["hp_iters"]
    assert np.isfinite(warm["loops"]).all()
