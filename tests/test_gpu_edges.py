"""Edge cases of the TSM path on the GPU against the oracle.

* Z2 noise (real sign sources) through the whole FP64 path.
* More momenta than one contraction pass holds (20 > 16: two chunks) and a
  non-contiguous, unordered insertion list.
* Degenerate index sets: no HP sources (the LP-only estimate) and no LP
  sources (the correction alone), against oracle.loops.tsm_combine.
* A batch wider than the number of sources equals single-source solves bit
  for bit.
* Lattices with an odd or too small extent are rejected on the host.
* Faults injected on the host: a NaN in a host source makes tm_solve_batch
  return TSM_ERR_NONFINITE in every tier; twist and hopping parameters whose
  operator overflows (finite kappa = 1e200) make tsm_loops return
  TSM_ERR_NONFINITE; in both cases the next call on the same context, with
  clean inputs, succeeds.
"""
import numpy as np
import pytest

from oracle import loops as oloops
from paper_1211_0126_gb300 import synthetic as S
from paper_1211_0126_gb300 import tsm

pytestmark = pytest.mark.gpu

DIMS = (4, 4, 4, 4)
KAPPA, MU = 0.124, 0.01
HP, LP = (1e-12, 5000), (0.0, 4)


def _rel(a, b):
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


@pytest.fixture(scope="module")
def field():
    return S.gauge_field(DIMS, 0.3, 21)


def _stops():
    return tsm.stop(*HP, tsm.TSM_F64), tsm.stop(*LP, tsm.TSM_F64)


def test_z2_noise_tsm(ctx, field):
    ctx.load_gauge(field, DIMS, KAPPA, MU)
    gam, moms = list(range(16)), S.default_momenta(4)
    got = ctx.loops(3, 2, 3, 9, *_stops(), gam, moms, per_source=True)
    want = oloops.tsm_loops(field, DIMS, KAPPA, MU, 3, 2, 3, 9, HP, LP, gam, moms)
    assert _rel(got["per_lp"], want["lp"]) < 1e-9
    assert _rel(got["loops"], want["loops"]) < 1e-9


def test_many_momenta_and_unordered_gammas(ctx, field):
    ctx.load_gauge(field, DIMS, KAPPA, MU)
    gam = [15, 0, 7]
    moms = [(a, b, c) for a in (-1, 0, 1) for b in (0, 1) for c in (-1, 0, 1)][:20]
    moms += [(2, 1, -2)] * (20 - len(moms))
    got = ctx.loops(5, 4, 2, 5, *_stops(), gam, moms, per_source=True)
    want = oloops.tsm_loops(field, DIMS, KAPPA, MU, 5, 4, 2, 5, HP, LP, gam, moms)
    assert got["loops"].shape == (3, 20, DIMS[3])
    assert _rel(got["per_lp"], want["lp"]) < 1e-9
    assert _rel(got["per_corr"], want["corr"]) < 1e-8


@pytest.mark.parametrize("n_hp,n_lp", [(0, 6), (4, 0)])
def test_empty_hp_or_lp_set(ctx, field, n_hp, n_lp):
    ctx.load_gauge(field, DIMS, KAPPA, MU)
    gam, moms = list(range(16)), S.default_momenta(4)
    got = ctx.loops(7, 4, n_hp, n_lp, *_stops(), gam, moms, per_source=True)
    want = oloops.tsm_loops(field, DIMS, KAPPA, MU, 7, 4, n_hp, n_lp, HP, LP, gam, moms)
    assert _rel(got["loops"], want["loops"]) < 1e-8
    assert _rel(got["err"], want["err"]) < 1e-8


def test_batch_wider_than_sources(ctx, field):
    ctx.load_gauge(field, DIMS, KAPPA, MU)
    gam, moms = list(range(16)), S.default_momenta(4)
    hp = tsm.stop(1e-10, 5000, tsm.TSM_F32, reliable=True)
    lp = tsm.stop(5e-3, 60, tsm.TSM_F16)
    one = ctx.loops(9, 4, 2, 3, hp, lp, gam, moms, per_source=True, batch=1)
    wide = ctx.loops(9, 4, 2, 3, hp, lp, gam, moms, per_source=True, batch=64)
    for k in ("loops", "err", "per_corr", "per_lp"):
        assert np.array_equal(one[k], wide[k]), k


@pytest.mark.parametrize("dims", [(3, 4, 4, 4), (4, 4, 4, 1), (4, 0, 4, 4)])
def test_bad_lattices_rejected(ctx, dims):
    U = np.zeros((max(dims[3], 1), max(dims[2], 1), max(dims[1], 1), max(dims[0], 1), 4, 3, 3), dtype=np.complex128)
    with pytest.raises(tsm.TsmError):
        ctx.load_gauge(U, dims, KAPPA, MU)


@pytest.mark.parametrize("prec", [tsm.TSM_F64, tsm.TSM_F32, tsm.TSM_F16, tsm.TSM_BF16])
def test_nan_in_host_source_reports_nonfinite(ctx, field, prec):
    ctx.load_gauge(field, DIMS, KAPPA, MU)
    b = S.random_spinor(DIMS, 5)
    b[1, 2, 3, 0, 2, 1] = complex(float("nan"), 0.0)
    s = np.zeros_like(b)
    stop = tsm.stop(1e-8, 200, prec, reliable=(prec == tsm.TSM_F32))
    with pytest.raises(tsm.TsmError) as e:
        tsm.tm_solve_batch(ctx.h, b, s, stop)
    assert e.value.status == -5   # TSM_ERR_NONFINITE
    # the context stays usable
    clean = S.random_spinor(DIMS, 6)
    sol, iters, tres, st = ctx.solve(clean, tsm.stop(1e-8, 2000, tsm.TSM_F64))
    assert st == 0 and tres[0] < 1e-7


def test_overflowing_operator_reports_nonfinite_in_tsm_loops(ctx, field):
    ctx.load_gauge(field, DIMS, 1e200, MU)   # finite, so accepted; kappa^2 overflows
    hp, lp = _stops()
    with pytest.raises(tsm.TsmError) as e:
        ctx.loops(3, 4, 2, 4, hp, lp, list(range(16)), S.default_momenta(4))
    assert e.value.status == -5   # TSM_ERR_NONFINITE
    ctx.load_gauge(field, DIMS, KAPPA, MU)
    got = ctx.loops(3, 4, 2, 4, hp, lp, list(range(16)), S.default_momenta(4))
    assert np.isfinite(got["loops"]).all()
