"""Oracle spot checks at the largest workload size, 32^3 x 64 (V = 2.1 M).

Two sources are solved on the GPU at the HP tier (FP32 + FP64 reliable
updates to 1e-10); the oracle's own FP64 operator gives their true residual,
and the oracle contracts the same solutions (16 local insertions and the
derivative insertion along t at 13 momenta) for an element-by-element
comparison with the GPU contraction of the same fields.  Sizes as in the
at-scale workload (kappa = 0.1248, mu = 0.003; links eps = 0.2 without the
APE steps, which only shape the field and cost minutes in numpy).
"""
import numpy as np
import pytest

from oracle import dirac, loops as oloops, philox
from paper_1211_0126_gb300 import synthetic as S
from paper_1211_0126_gb300 import tsm

pytestmark = pytest.mark.gpu

DIMS = (32, 32, 32, 64)
KAPPA, MU = 0.1248, 0.003


def test_spot_checks_at_32x32x32x64(ctx):
    U = S.gauge_field(DIMS, 0.2, 301)
    ctx.load_gauge(U, DIMS, KAPPA, MU)
    gam, moms = list(range(16)), S.default_momenta(13)
    hp = tsm.stop(1e-10, 20000, tsm.TSM_F32, reliable=True, reliable_delta=1e-5)
    for j in range(2):
        eta = philox.noise(6, j, DIMS, 4)
        s, it, tres, st = ctx.solve(eta, hp)
        assert st == 0 and tres[0] < 1e-9
        r = eta - dirac.dtm(U, s, DIMS, KAPPA, MU)
        assert np.linalg.norm(r) / np.linalg.norm(eta) < 1e-9
        want = oloops.local_loops(eta, s, DIMS, gam, moms)
        got = ctx.contract(6, j, s, gam, moms)
        assert np.abs(got - want).max() < 1e-12 * np.abs(want).max()
        want_d = np.transpose(oloops.deriv_loops(U, eta, s, DIMS, gam, [3], moms), (1, 0, 2, 3))
        got_d = ctx.contract_deriv(6, j, s, gam, 0b1000, moms)
        assert np.abs(got_d - want_d).max() < 1e-12 * np.abs(want_d).max()
