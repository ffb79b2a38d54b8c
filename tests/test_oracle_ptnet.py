"""Pins for oracle.ptnet (the parallel-transport layers of the learned preconditioner).

* T_p^dagger is the adjoint of T_p: <h, T_p psi> = <T_p^dagger h, psi>.
* Gauge covariance: layer(U^G, G psi) = G layer(U, psi).
* Free field with a spatially constant input: every transport is the
  identity (up to the time-boundary sign, absent for periodic time), so the
  layer is the plain matrix product (sum_p W_p) u.
* Central finite differences of a real loss reproduce the analytic weight and
  input gradients (G = dL/dRe + i dL/dIm) through a two-layer stack.
"""
import numpy as np
import pytest

from oracle import ptnet
from paper_1211_0126_gb300 import synthetic as S

DIMS = (4, 2, 2, 4)


def _field(c, seed, dims=DIMS):
    return S.random_spinor(dims, seed, batch=(c,))


def _W(cout, cin, seed):
    rng = np.random.default_rng(seed)
    return (rng.standard_normal((4 * cout, 36 * cin)) + 1j * rng.standard_normal((4 * cout, 36 * cin))) / 10


@pytest.mark.parametrize("apbc", [True, False])
def test_transport_adjoint(apbc):
    U = S.gauge_field(DIMS, 0.4, 1)
    psi, h = _field(2, 2), _field(2, 3)
    for p in range(9):
        lhs = np.vdot(h, ptnet.transport(U, psi, DIMS, p, apbc))
        rhs = np.vdot(ptnet.transport_adjoint(U, h, DIMS, p, apbc), psi)
        assert abs(lhs - rhs) < 1e-12 * abs(lhs)


def test_layer_gauge_covariant():
    U = S.gauge_field(DIMS, 0.4, 4)
    G = S.gauge_transform(DIMS, 5)
    psi = _field(3, 6)
    W = _W(2, 3, 7)
    lhs = ptnet.layer_forward(S.transform_links(U, G), W, S.transform_spinor(psi, G), DIMS)
    rhs = S.transform_spinor(ptnet.layer_forward(U, W, psi, DIMS), G)
    assert np.abs(lhs - rhs).max() < 1e-12 * np.abs(rhs).max()


def test_free_field_constant_input_is_matrix_product():
    U = S.gauge_field(DIMS, 0.0, 0)
    rng = np.random.default_rng(8)
    cin, cout = 2, 3
    u = rng.standard_normal((cin, 4, 3)) + 1j * rng.standard_normal((cin, 4, 3))
    psi = np.broadcast_to(u[:, None, None, None, None], (cin,) + (DIMS[3], DIMS[2], DIMS[1], DIMS[0], 4, 3)).copy()
    W = _W(cout, cin, 9)
    y = ptnet.layer_forward(U, W, psi, DIMS, antiperiodic_t=False)
    Wsum = W.reshape(4 * cout, 9, 4 * cin).sum(axis=1)            # sum over paths
    want = np.einsum('nk,ka->na', Wsum, u.reshape(4 * cin, 3)).reshape(cout, 4, 3)
    assert np.allclose(y, want[:, None, None, None, None], atol=1e-12)


def test_finite_differences_two_layers():
    U = S.gauge_field(DIMS, 0.4, 10)
    x = _field(1, 11)
    t = _field(1, 12)[0]
    mask = np.ones((DIMS[3], DIMS[2], DIMS[1], DIMS[0], 1, 1))
    Ws = [_W(3, 1, 13), _W(1, 3, 14)]

    def loss(Ws_, x_=x):
        y = ptnet.net_forward(U, Ws_, x_, DIMS)[-1]
        return ptnet.relative_loss(y, t, mask)[0]

    acts = ptnet.net_forward(U, Ws, x, DIMS)
    L, gy = ptnet.relative_loss(acts[-1], t, mask)
    grads = ptnet.net_backward(U, Ws, acts, gy, DIMS)
    h = 1e-6
    rng = np.random.default_rng(15)
    for l in range(2):
        for _ in range(4):
            n, k = rng.integers(0, Ws[l].shape[0]), rng.integers(0, Ws[l].shape[1])
            for unit in (1.0, 1j):
                Wp = [w.copy() for w in Ws]
                Wm = [w.copy() for w in Ws]
                Wp[l][n, k] += h * unit
                Wm[l][n, k] -= h * unit
                fd = (loss(Wp) - loss(Wm)) / (2 * h)
                an = grads[l][n, k].real if unit == 1.0 else grads[l][n, k].imag
                assert abs(fd - an) < 1e-6 * max(1.0, abs(an)), (l, n, k, unit, fd, an)
    # input gradient of the first layer stack
    g_in = ptnet.layer_backward(U, Ws[0], x, ptnet.layer_backward(U, Ws[1], acts[1], gy, DIMS)[0], DIMS)[0]
    idx = (0, 1, 0, 1, 2, 3, 1)
    for unit in (1.0, 1j):
        xp, xm = x.copy(), x.copy()
        xp[idx] += h * unit
        xm[idx] -= h * unit
        fd = (loss(Ws, xp) - loss(Ws, xm)) / (2 * h)
        an = g_in[idx].real if unit == 1.0 else g_in[idx].imag
        assert abs(fd - an) < 1e-6 * max(1.0, abs(an))
