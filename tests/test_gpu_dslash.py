"""GPU parity of the Dslash kernels against the oracle (through the C ABI).

Tolerances (relative, norm-wise over the lattice): FP64 1e-12, FP32 1e-5,
FP16/BF16 5e-3 -- the per-tier bounds for the operator.  Lattices span several
thread blocks with a ragged tail (6x4x4x6: V/2 = 288 = 2 x 128 + 32), the 2^4
lattice where forward and backward neighbours coincide, a non-cubic lattice,
and the 24^3 x 48 production lattice on sampled sites.
"""
import numpy as np
import pytest

from oracle import dirac
from paper_1211_0126_gb300 import synthetic as S
from paper_1211_0126_gb300 import tsm

pytestmark = pytest.mark.gpu

KAPPA, MU = 0.124, 0.01
TOL = {tsm.TSM_F64: 1e-12, tsm.TSM_F32: 1e-5, tsm.TSM_F16: 5e-3, tsm.TSM_BF16: 5e-3}
LATTICES = [(4, 4, 4, 4), (2, 2, 2, 2), (6, 4, 4, 6), (4, 2, 6, 4)]


def _rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def _oracle(op, dagger, U, psi, dims, apbc=True):
    e, o = dirac.even_mask(dims), dirac.odd_mask(dims)
    if op == tsm.TM_OP_FULL:
        return dirac.dtm(U, psi, dims, KAPPA, MU, apbc, adjoint=dagger)
    if op == tsm.TM_OP_HOP_EO:
        return dirac.hop_to(U, psi, dims, 0, apbc, adjoint=dagger)
    if op == tsm.TM_OP_HOP_OE:
        return dirac.hop_to(U, psi, dims, 1, apbc, adjoint=dagger)
    if op == tsm.TM_OP_SCHUR:
        f = dirac.schur_dag if dagger else dirac.schur
        return f(U, e * psi, dims, KAPPA, MU, apbc)
    if op == tsm.TM_OP_NORMAL:
        q = dirac.schur(U, e * psi, dims, KAPPA, MU, apbc)
        return dirac.schur_dag(U, q, dims, KAPPA, MU, apbc)
    raise ValueError(op)


@pytest.mark.parametrize("dims", LATTICES)
@pytest.mark.parametrize("apbc", [True, False])
def test_operators_all_tiers(ctx, dims, apbc):
    U = S.gauge_field(dims, 0.3, 7)
    ctx.load_gauge(U, dims, KAPPA, MU, apbc)
    psi = S.random_spinor(dims, 8)
    for op in (tsm.TM_OP_FULL, tsm.TM_OP_HOP_EO, tsm.TM_OP_HOP_OE, tsm.TM_OP_SCHUR, tsm.TM_OP_NORMAL):
        for dagger in (False, True):
            want = _oracle(op, dagger, U, psi, dims, apbc)
            for prec, tol in TOL.items():
                got = ctx.dslash(psi, op, dagger, prec)
                err = _rel(got, want)
                assert err < tol, (op, dagger, prec, err)
                if op in (tsm.TM_OP_HOP_EO, tsm.TM_OP_SCHUR, tsm.TM_OP_NORMAL):
                    assert np.all(got * dirac.odd_mask(dims) == 0)
                if op == tsm.TM_OP_HOP_OE:
                    assert np.all(got * dirac.even_mask(dims) == 0)


def test_free_field_and_gauge_covariance(ctx):
    dims = (4, 4, 4, 8)
    U = S.gauge_field(dims, 0.3, 17)
    G = S.gauge_transform(dims, 18)
    psi = S.random_spinor(dims, 19)
    ctx.load_gauge(S.transform_links(U, G), dims, KAPPA, MU)
    lhs = ctx.dslash(S.transform_spinor(psi, G))
    ctx.load_gauge(U, dims, KAPPA, MU)
    rhs = S.transform_spinor(ctx.dslash(psi), G)
    assert _rel(lhs, rhs) < 1e-13


def test_non_unitary_links_rejected(ctx):
    dims = (4, 4, 4, 4)
    U = S.gauge_field(dims, 0.3, 27)
    U[1, 2, 3, 0, 2] *= 1.001
    with pytest.raises(tsm.TsmError) as ei:
        ctx.load_gauge(U, dims, KAPPA, MU)
    assert ei.value.status == -7
    with pytest.raises(tsm.TsmError):
        ctx.load_gauge(S.gauge_field((3, 4, 4, 4), 0.3, 1), (3, 4, 4, 4), KAPPA, MU)


@pytest.mark.parametrize("prec", [tsm.TSM_F32, tsm.TSM_F16, tsm.TSM_BF16, tsm.TSM_F64])
def test_production_lattice_sampled_sites(ctx, prec):
    """24^3 x 48 (the benchmark lattice): H_eo on sampled even sites against the
    oracle's site-by-site stencil."""
    dims = (24, 24, 24, 48)
    U = getattr(test_production_lattice_sampled_sites, "_U", None)
    if U is None:
        U = S.gauge_field(dims, 0.25, 3)
        test_production_lattice_sampled_sites._U = U
    ctx.load_gauge(U, dims, 0.1245, 0.005)
    psi = S.random_spinor(dims, 4) * dirac.odd_mask(dims)
    got = ctx.dslash(psi, tsm.TM_OP_HOP_EO, False, prec)
    rng = np.random.default_rng(5)
    sites = [(0, 0, 0, 0), (23, 23, 22, 47), (1, 0, 0, 47), (0, 23, 0, 0)]
    for _ in range(60):
        s = [int(rng.integers(0, d)) for d in dims]
        if sum(s) % 2:
            s[0] = (s[0] + 1) % dims[0]
        sites.append(tuple(s))
    num = den = 0.0
    for (x, y, z, t) in sites:
        if (x + y + z + t) % 2:
            continue
        want = dirac.hop_at_site(U, psi, dims, (x, y, z, t))
        num += np.sum(np.abs(got[t, z, y, x] - want) ** 2)
        den += np.sum(np.abs(want) ** 2)
    assert np.sqrt(num / den) < TOL[prec]
