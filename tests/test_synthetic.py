"""The seeded input generators (paper_1211_0126_gb300/synthetic.py) that feed
both the CUDA path and the oracle: every link exactly SU(3), the same field
for the same seed, a distance from the identity set by eps, APE smearing and
gauge transformations that stay in SU(3), transformed links and spinors that
obey U'(x) = G(x) U(x) G(x+mu)^dag and psi' = G psi, and the momentum lists
used by the workloads."""
import numpy as np
import pytest

from paper_1211_0126_gb300 import synthetic as S

DIMS = (4, 4, 2, 6)


def _su3_deviation(U):
    m = U.reshape(-1, 3, 3)
    unit = np.abs(m @ np.conj(np.swapaxes(m, -1, -2)) - np.eye(3)).max()
    det = np.abs(np.linalg.det(m) - 1.0).max()
    return max(unit, det)


@pytest.mark.parametrize("eps", [0.05, 0.3, 1.0])
def test_links_are_su3(eps):
    U = S.gauge_field(DIMS, eps, 7)
    assert U.shape == (DIMS[3], DIMS[2], DIMS[1], DIMS[0], 4, 3, 3)
    assert _su3_deviation(U) < 1e-13


def test_seeded_and_eps_controls_distance_from_identity():
    a = S.gauge_field(DIMS, 0.25, 11)
    b = S.gauge_field(DIMS, 0.25, 11)
    c = S.gauge_field(DIMS, 0.25, 12)
    assert np.array_equal(a, b) and not np.allclose(a, c)
    dist = [np.abs(S.gauge_field(DIMS, e, 3) - np.eye(3)).mean() for e in (0.05, 0.2, 0.8)]
    assert dist[0] < dist[1] < dist[2]


def _plaquette(U):
    """Mean of Re tr[U_mu(x) U_nu(x+mu) U_mu(x+nu)^dag U_nu(x)^dag] / 3 (gauge invariant)."""
    axis = {0: 3, 1: 2, 2: 1, 3: 0}   # array axis of direction mu in [T, Z, Y, X]
    dag = lambda m: np.conj(np.swapaxes(m, -1, -2))
    tot, n = 0.0, 0
    for mu in range(4):
        for nu in range(mu + 1, 4):
            um, un = U[..., mu, :, :], U[..., nu, :, :]
            un_xm = np.roll(un, -1, axis=axis[mu])
            um_xn = np.roll(um, -1, axis=axis[nu])
            p = um @ un_xm @ dag(um_xn) @ dag(un)
            tot += np.trace(p, axis1=-2, axis2=-1).real.mean() / 3.0
            n += 1
    return tot / n


def test_ape_smearing_stays_su3_and_smooths():
    rough = S.gauge_field(DIMS, 0.8, 5)
    smooth = S.gauge_field(DIMS, 0.8, 5, ape_steps=2, ape_alpha=0.5)
    assert _su3_deviation(smooth) < 1e-12
    # smearing averages links with their staples: the gauge-invariant
    # plaquette moves towards 1
    assert _plaquette(rough) < _plaquette(smooth) < 1.0
    # and the plaquette is invariant under a gauge transformation
    G = S.gauge_transform(DIMS, 8)
    assert abs(_plaquette(S.transform_links(rough, G)) - _plaquette(rough)) < 1e-12


def test_gauge_transformation_of_links_and_spinors():
    U = S.gauge_field(DIMS, 0.3, 2)
    G = S.gauge_transform(DIMS, 9)
    assert _su3_deviation(G) < 1e-13
    Ut = S.transform_links(U, G)
    assert _su3_deviation(Ut) < 1e-12
    # U'_mu(x) = G(x) U_mu(x) G(x + mu)^dag at one interior and one wrapped site
    for (t, z, y, x) in [(1, 0, 1, 2), (DIMS[3] - 1, DIMS[2] - 1, DIMS[1] - 1, DIMS[0] - 1)]:
        for mu in range(4):
            c = [x, y, z, t]
            c[mu] = (c[mu] + 1) % DIMS[mu]
            want = G[t, z, y, x] @ U[t, z, y, x, mu] @ np.conj(G[c[3], c[2], c[1], c[0]]).T
            assert np.abs(Ut[t, z, y, x, mu] - want).max() < 1e-13
    psi = S.random_spinor(DIMS, 4)
    pt = S.transform_spinor(psi, G)
    assert np.abs(pt[1, 0, 1, 2] - np.einsum("ab,sb->sa", G[1, 0, 1, 2], psi[1, 0, 1, 2])).max() < 1e-13


def test_random_spinor_shape_and_seed():
    a = S.random_spinor(DIMS, 3, batch=(2,))
    assert a.shape == (2, DIMS[3], DIMS[2], DIMS[1], DIMS[0], 4, 3)
    assert np.array_equal(a, S.random_spinor(DIMS, 3, batch=(2,)))
    assert not np.allclose(a[0], a[1])


def test_default_momenta():
    assert [tuple(m) for m in S.default_momenta(1)] == [(0, 0, 0)]
    four = {tuple(m) for m in S.default_momenta(4)}
    assert four == {(0, 0, 0), (1, 0, 0), (0, 1, 0), (0, 0, 1)}
    seven = {tuple(m) for m in S.default_momenta(7)}
    assert seven == {(0, 0, 0)} | {tuple(s * e) for s in (1, -1) for e in np.eye(3, dtype=int)}
    thirteen = [tuple(m) for m in S.default_momenta(13)]
    assert len(thirteen) == len(set(thirteen)) == 13 and seven <= set(thirteen)
    pairs = set(thirteen) - seven
    assert all(sum(abs(v) for v in m) == 2 and m.count(0) == 1 for m in pairs)
    assert all(tuple(-v for v in m) in pairs for m in pairs)
