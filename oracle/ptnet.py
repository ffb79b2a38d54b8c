"""Parallel-transport network layers of the learned preconditioner (oracle; test infrastructure).

The paper has no network; the learned LP preconditioner is this project's
extension of the LP solves of Sec. 2.2 (it may change only the variance per
unit cost, never the expectation of Eq. 2.4).  This module fixes, in plain
FP64 numpy, what one layer computes and its exact gradient.

Layer (C_in -> C_out complex channels, each channel a spinor field):

    y_{c'}(x)_{s'a} = sum_{p = 0..8} sum_{c, s} W[(c', s'), (p, c, s)] (T_p psi_c)(x)_{s a}

with the gauge-covariant transports (colour index a)
    T_0 psi(x)        = psi(x)
    T_{2mu+1} psi(x)  = U_mu(x) psi(x + mu)              (mu = 0..3)
    T_{2mu+2} psi(x)  = U_mu(x - mu)^dagger psi(x - mu)
and the fermion boundary sign on hops across t = T-1 <-> 0 when the lattice
is antiperiodic in time (the same convention as the Dirac operator).  W acts
on channel and spin indices only, so the layer commutes with gauge
transformations.  Column index of W: k = (p * C_in + c) * 4 + s; row index
n = c' * 4 + s'.

Gradients follow G = dL/dRe + i dL/dIm of a real loss L: for y = W z,
G_W = sum G_y conj(z) and G_z = W^dagger G_y; the transport's adjoint is
T_p^dagger.  Pinned in tests by gauge covariance, a reduction to a plain
matrix product at U = 1 on a 1-site-per-direction check, and central finite
differences of the loss.

Arrays: U [T, Z, Y, X, 4, 3, 3]; fields [C, T, Z, Y, X, 4, 3] complex128.
"""
import numpy as np

_AX = {0: -3, 1: -4, 2: -5, 3: -6}     # axis of direction mu in a [..., T, Z, Y, X, 4, 3] field
_UAX = {0: 3, 1: 2, 2: 1, 3: 0}        # axis of direction mu in U


def _sign(dims, forward):
    lt = dims[3]
    s = np.ones(lt)
    s[lt - 1 if forward else 0] = -1.0
    return s.reshape(lt, 1, 1, 1, 1, 1)


def transport(U, psi, dims, p, antiperiodic_t=True):
    """T_p psi for a field with leading channel axis."""
    if p == 0:
        return psi.copy()
    mu, fwd = (p - 1) // 2, (p - 1) % 2 == 0
    if fwd:
        q = np.roll(psi, -1, axis=_AX[mu])
        if mu == 3 and antiperiodic_t:
            q = q * _sign(dims, True)
        return np.einsum('tzyxab,...tzyxsb->...tzyxsa', U[..., mu, :, :], q)
    ub = np.roll(U[..., mu, :, :], 1, axis=_UAX[mu])
    q = np.roll(psi, 1, axis=_AX[mu])
    if mu == 3 and antiperiodic_t:
        q = q * _sign(dims, False)
    return np.einsum('tzyxba,...tzyxsb->...tzyxsa', np.conj(ub), q)


def transport_adjoint(U, g, dims, p, antiperiodic_t=True):
    """T_p^dagger g: adjoint of transport() under sum_x conj(a) . b."""
    if p == 0:
        return g.copy()
    mu, fwd = (p - 1) // 2, (p - 1) % 2 == 0
    if fwd:
        # (T g)(x) = U(x) g(x+mu)  ->  (T^dag h)(y) = U(y-mu)^dag h(y-mu) * sign(y-mu)
        ub = np.roll(U[..., mu, :, :], 1, axis=_UAX[mu])
        q = np.roll(g, 1, axis=_AX[mu])
        if mu == 3 and antiperiodic_t:
            q = q * _sign(dims, False)
        return np.einsum('tzyxba,...tzyxsb->...tzyxsa', np.conj(ub), q)
    # (T g)(x) = U(x-mu)^dag g(x-mu)  ->  (T^dag h)(y) = U(y) h(y+mu) * sign
    q = np.roll(g, -1, axis=_AX[mu])
    if mu == 3 and antiperiodic_t:
        q = q * _sign(dims, True)
    return np.einsum('tzyxab,...tzyxsb->...tzyxsa', U[..., mu, :, :], q)


def gathered(U, psi, dims, antiperiodic_t=True):
    """z[(p, c, s)] per site/colour: [9, C, T, Z, Y, X, 4, 3]."""
    return np.array([transport(U, psi, dims, p, antiperiodic_t) for p in range(9)])


def layer_forward(U, W, psi, dims, antiperiodic_t=True):
    """y = layer(psi); W complex [4 C_out, 36 C_in]; psi [C_in, ...] -> [C_out, ...]."""
    cin = psi.shape[0]
    cout = W.shape[0] // 4
    z = gathered(U, psi, dims, antiperiodic_t)               # [9, Cin, T, Z, Y, X, 4, 3]
    Wr = W.reshape(cout, 4, 9, cin, 4)                       # [c', s', p, c, s]
    return np.einsum('ospcr,pctzyxra->otzyxsa', Wr, z)


def layer_backward(U, W, psi, gy, dims, antiperiodic_t=True):
    """Gradients (G_psi, G_W) of a real loss given G_y (same convention)."""
    cin = psi.shape[0]
    cout = W.shape[0] // 4
    z = gathered(U, psi, dims, antiperiodic_t)
    Wr = W.reshape(cout, 4, 9, cin, 4)
    gW = np.einsum('otzyxsa,pctzyxra->ospcr', gy, np.conj(z)).reshape(W.shape)
    gz = np.einsum('ospcr,otzyxsa->pctzyxra', np.conj(Wr), gy)   # W^dagger G_y per path
    gpsi = np.zeros_like(psi)
    for p in range(9):
        gpsi += transport_adjoint(U, gz[p], dims, p, antiperiodic_t)
    return gpsi, gW


def net_forward(U, Ws, x, dims, antiperiodic_t=True):
    """Stack of layers (linear, no activation); x [C0, ...]."""
    acts = [x]
    for W in Ws:
        acts.append(layer_forward(U, W, acts[-1], dims, antiperiodic_t))
    return acts


def net_backward(U, Ws, acts, gy, dims, antiperiodic_t=True):
    """Gradients of all weights given G of the output."""
    grads = [None] * len(Ws)
    g = gy
    for l in range(len(Ws) - 1, -1, -1):
        g, grads[l] = layer_backward(U, Ws[l], acts[l], g, dims, antiperiodic_t)
    return grads


def relative_loss(y, t, mask):
    """L = sum_mask |y - t|^2 / sum_mask |t|^2 and its G_y (output channel 0)."""
    d = (y[0] - t) * mask
    den = np.sum(np.abs(t * mask) ** 2)
    L = np.sum(np.abs(d) ** 2) / den
    gy = np.zeros_like(y)
    gy[0] = 2.0 * d / den
    return L, gy
