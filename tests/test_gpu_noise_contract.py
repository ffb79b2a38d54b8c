"""GPU parity of noise generation (bit-exact) and loop contraction."""
import numpy as np
import pytest

from oracle import loops as oloops
from oracle import philox
from paper_1211_0126_gb300 import synthetic as S
from paper_1211_0126_gb300 import tsm

pytestmark = pytest.mark.gpu

MOMS13 = S.default_momenta(13)


@pytest.mark.parametrize("dims", [(4, 4, 4, 4), (6, 4, 2, 8), (2, 2, 2, 2)])
@pytest.mark.parametrize("kind", [4, 2])
def test_noise_bit_exact(ctx, dims, kind):
    ctx.load_gauge(S.gauge_field(dims, 0.0, 0), dims, 0.124, 0.01)
    for seed in (1, 2024, (7 << 40) + 12345):
        for src in (0, 1, 77, 2 ** 31 + 5):
            got = ctx.noise(seed, src, kind)
            want = philox.noise(seed, src, dims, kind)
            assert np.array_equal(got.view(np.float64), want.view(np.float64)), (seed, src)


@pytest.mark.parametrize("dims", [(4, 4, 4, 4), (6, 4, 4, 6), (4, 6, 2, 4)])
def test_contraction_fp64_and_fp32(ctx, dims):
    ctx.load_gauge(S.gauge_field(dims, 0.0, 0), dims, 0.124, 0.01)
    s_a = S.random_spinor(dims, 11)
    s_b = S.random_spinor(dims, 12)
    gam = list(range(16))
    moms = MOMS13 + [(2, 1, 0), (-1, 2, 1), (1, -1, -1), (0, 0, 2)]   # 17 momenta: two chunks
    eta = philox.noise(99, 5, dims, 4)
    want = oloops.local_loops(eta, s_a - s_b, dims, gam, moms)
    got = ctx.contract(99, 5, s_a, gam, moms, s_b=s_b, prec=tsm.TSM_F64)
    assert np.abs(got - want).max() < 1e-12 * np.abs(want).max()
    got32 = ctx.contract(99, 5, s_a, gam, moms, s_b=s_b, prec=tsm.TSM_F32)
    assert np.abs(got32 - want).max() < 1e-5 * np.abs(want).max()
    # subset of insertions in a different order, Z2 noise, no s_b
    sub = [15, 5, 0, 9]
    eta2 = philox.noise(3, 0, dims, 2)
    want2 = oloops.local_loops(eta2, s_a, dims, sub, moms[:4])
    got2 = ctx.contract(3, 0, s_a, sub, moms[:4], kind=2, prec=tsm.TSM_F64)
    assert np.abs(got2 - want2).max() < 1e-12 * np.abs(want2).max()


def test_contraction_production_lattice(ctx):
    """24^3 x 48, 16 insertions x 7 momenta: the FP32 contraction of the
    benchmark against the oracle on the full lattice."""
    dims = (24, 24, 24, 48)
    ctx.load_gauge(S.gauge_field(dims, 0.0, 0), dims, 0.1245, 0.005)
    s = S.random_spinor(dims, 21)
    gam, moms = list(range(16)), S.default_momenta(7)
    eta = philox.noise(5, 3, dims, 4)
    want = oloops.local_loops(eta, s, dims, gam, moms)
    got = ctx.contract(5, 3, s, gam, moms, prec=tsm.TSM_F32)
    scale = np.abs(want).max()
    assert np.abs(got - want).max() < 1e-5 * scale
    got64 = ctx.contract(5, 3, s, gam, moms, prec=tsm.TSM_F64)
    assert np.abs(got64 - want).max() < 1e-11 * scale


def test_contraction_momentum_classes(ctx):
    """Momenta that pair up as q and -q, repeat, coincide mod L, are zero mod L
    or are their own negative mod L: the kernel forms each from one cosine and
    one sine sum per class, and every entry still equals the oracle's direct
    phase sum; FP64 and FP32, all 16 insertions and a subset."""
    dims = (4, 6, 4, 4)
    ctx.load_gauge(S.gauge_field(dims, 0.0, 0), dims, 0.124, 0.01)
    s_a = S.random_spinor(dims, 31)
    moms = [(1, 0, 0), (0, 0, 0), (-1, 0, 0), (2, 0, 0), (1, 0, 0), (3, 0, 0), (0, -1, 1), (0, 1, -1),
            (4, 0, 0), (0, 3, 0), (1, 2, -1), (-1, -2, 1), (0, 0, -2)]
    eta = philox.noise(8, 2, dims, 4)
    for gam in (list(range(16)), [7, 3, 12]):
        want = oloops.local_loops(eta, s_a, dims, gam, moms)
        got = ctx.contract(8, 2, s_a, gam, moms, prec=tsm.TSM_F64)
        assert np.abs(got - want).max() < 1e-12 * np.abs(want).max()
        got32 = ctx.contract(8, 2, s_a, gam, moms, prec=tsm.TSM_F32)
        assert np.abs(got32 - want).max() < 1e-5 * np.abs(want).max()
