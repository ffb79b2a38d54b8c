"""Twisted-mass Wilson-Dirac operator, written literally (oracle; test infrastructure).

The paper (Sec. 2.2, Sec. 2.3) relies on twisted-mass fermions but never writes
the operator.  Reading used here:

    D_tm = 1 - kappa * H + 2 i kappa mu gamma_5,
    (H psi)(x) = sum_mu [ (1 - gamma_mu) U_mu(x) psi(x + mu)
                        + (1 + gamma_mu) U_mu(x - mu)^dagger psi(x - mu) ],

with full 4x4 gamma matrices (oracle.gamma), full 3x3 links (no
reconstruction) and periodic wrap, times -1 on hops that cross the time
boundary when the lattice is antiperiodic in t.  The u flavour is +mu and the
d flavour -mu, as in Sec. 2.3 (M_u - M_d = 2 i mu a gamma_5).

Array conventions (canonical layout):
    dims = (Lx, Ly, Lz, T); lexicographic site index x + Lx*(y + Ly*(z + Lz*t))
    U   complex128 [T, Z, Y, X, 4, 3, 3]    (mu = 0:x, 1:y, 2:z, 3:t)
    psi complex128 [..., T, Z, Y, X, 4, 3]  (spin, colour); leading batch axes allowed

Even/odd scheme (not in the paper; standard block elimination).  With parity
p(x) = (x+y+z+t) mod 2, A = 1 + 2 i kappa mu gamma_5 and
A^-1 = (1 - 2 i kappa mu gamma_5) / (1 + 4 kappa^2 mu^2):

    D = [[A_ee, -kappa H_eo], [-kappa H_oe, A_oo]]
    Dhat   = 1 - kappa^2 A_ee^-1 H_eo A_oo^-1 H_oe         (acts on even sites)
    bhat_e = A_ee^-1 (b_e + kappa H_eo A_oo^-1 b_o)
    x_o    = A_oo^-1 (b_o + kappa H_oe x_e)

Everything here works on full-lattice arrays with the other parity zeroed by a
mask, so it shares nothing with a half-lattice implementation.
"""
import numpy as np

from .gamma import gamma_matrices

# axis of each direction inside the trailing [T, Z, Y, X, 4, 3] block of psi
_PSI_AXIS = {0: -3, 1: -4, 2: -5, 3: -6}
# axis of each direction inside the leading [T, Z, Y, X] block of U
_U_AXIS = {0: 3, 1: 2, 2: 1, 3: 0}


def _time_sign(dims, forward):
    """-1 on the timeslice whose hop crosses the t boundary, else +1.

    forward: the hop reads psi(x + t), which wraps for t = T-1.
    backward: the hop reads psi(x - t), which wraps for t = 0.
    Returned with shape [T, 1, 1, 1, 1, 1] to broadcast against psi.
    """
    lt = dims[3]
    s = np.ones(lt)
    s[lt - 1 if forward else 0] = -1.0
    return s.reshape(lt, 1, 1, 1, 1, 1)


def hop(U, psi, dims, antiperiodic_t=True, adjoint=False):
    """H psi, or H^dagger psi when adjoint=True.

    The adjoint of the hopping term is the same stencil with the projectors
    exchanged, (1 - gamma_mu) <-> (1 + gamma_mu): H^dagger(x, x+mu) =
    (1 + gamma_mu) U_mu(x), H^dagger(x, x-mu) = (1 - gamma_mu) U_mu(x-mu)^dagger.
    """
    g, _ = gamma_matrices()
    one = np.eye(4, dtype=np.complex128)
    sgn = -1.0 if adjoint else 1.0
    out = np.zeros(np.broadcast_shapes(psi.shape), dtype=np.complex128)
    for mu in range(4):
        ax = _PSI_AXIS[mu]
        proj_fwd = one - sgn * g[mu]
        proj_bwd = one + sgn * g[mu]
        u_here = U[..., mu, :, :]                                 # U_mu(x)
        u_back = np.roll(U[..., mu, :, :], 1, axis=_U_AXIS[mu])   # U_mu(x - mu)
        psi_fwd = np.roll(psi, -1, axis=ax)                       # psi(x + mu)
        psi_bwd = np.roll(psi, 1, axis=ax)                        # psi(x - mu)
        if mu == 3 and antiperiodic_t:
            psi_fwd = psi_fwd * _time_sign(dims, True)
            psi_bwd = psi_bwd * _time_sign(dims, False)
        # colour: (U psi)_a = sum_b U_ab psi_b ;  (U^dag psi)_a = sum_b conj(U_ba) psi_b
        cf = np.einsum('tzyxab,...tzyxsb->...tzyxsa', u_here, psi_fwd)
        cb = np.einsum('tzyxba,...tzyxsb->...tzyxsa', np.conj(u_back), psi_bwd)
        out += np.einsum('rs,...sa->...ra', proj_fwd, cf)
        out += np.einsum('rs,...sa->...ra', proj_bwd, cb)
    return out


def gamma5(psi):
    _, g5 = gamma_matrices()
    return np.einsum('rs,...sa->...ra', g5, psi)


def dtm(U, psi, dims, kappa, mu, antiperiodic_t=True, adjoint=False):
    """D_tm psi (adjoint=False) or D_tm^dagger psi (adjoint=True).

    D_tm^dagger = 1 - kappa H^dagger - 2 i kappa mu gamma_5.
    """
    tw = 2j * kappa * mu * (-1.0 if adjoint else 1.0)
    return (psi - kappa * hop(U, psi, dims, antiperiodic_t, adjoint)
            + tw * gamma5(psi))


def parity_mask(dims):
    """[T, Z, Y, X, 1, 1] array: 1 on odd sites, 0 on even sites."""
    lx, ly, lz, lt = dims
    t, z, y, x = np.meshgrid(np.arange(lt), np.arange(lz), np.arange(ly),
                             np.arange(lx), indexing='ij')
    return ((x + y + z + t) % 2).astype(np.float64).reshape(lt, lz, ly, lx, 1, 1)


def even_mask(dims):
    return 1.0 - parity_mask(dims)


def odd_mask(dims):
    return parity_mask(dims)


def twist(psi, kappa, mu):
    """A psi = (1 + 2 i kappa mu gamma_5) psi."""
    return psi + 2j * kappa * mu * gamma5(psi)


def twist_inv(psi, kappa, mu):
    """A^-1 psi = (1 - 2 i kappa mu gamma_5) psi / (1 + 4 kappa^2 mu^2)."""
    return (psi - 2j * kappa * mu * gamma5(psi)) / (1.0 + 4.0 * kappa * kappa * mu * mu)


def hop_to(U, psi, dims, target, antiperiodic_t=True, adjoint=False):
    """Parity block of H (or H^dagger): target 0 gives H_eo (odd -> even), 1 H_oe."""
    m_out = even_mask(dims) if target == 0 else odd_mask(dims)
    m_in = odd_mask(dims) if target == 0 else even_mask(dims)
    return m_out * hop(U, m_in * psi, dims, antiperiodic_t, adjoint)


def schur(U, psi_e, dims, kappa, mu, antiperiodic_t=True):
    """Dhat psi_e = psi_e - kappa^2 A_ee^-1 H_eo A_oo^-1 H_oe psi_e (even sites)."""
    pe = even_mask(dims) * psi_e
    t = twist_inv(hop_to(U, pe, dims, 1, antiperiodic_t), kappa, mu)
    t = twist_inv(hop_to(U, t, dims, 0, antiperiodic_t), kappa, mu)
    return pe - kappa * kappa * t


def schur_dag(U, psi_e, dims, kappa, mu, antiperiodic_t=True):
    """Dhat^dagger psi_e, as the literal adjoint of each factor of Dhat:

    Dhat^dagger = 1 - kappa^2 (H_oe)^dag (A_oo^-1)^dag (H_eo)^dag (A_ee^-1)^dag,
    (H_oe)^dag = (H^dagger)_eo, (H_eo)^dag = (H^dagger)_oe, (A^-1)^dag = A^-1 at -mu.
    """
    pe = even_mask(dims) * psi_e
    t = twist_inv(pe, kappa, -mu)
    t = twist_inv(hop_to(U, t, dims, 1, antiperiodic_t, adjoint=True), kappa, -mu)
    t = hop_to(U, t, dims, 0, antiperiodic_t, adjoint=True)
    return pe - kappa * kappa * t


def schur_source(U, b, dims, kappa, mu, antiperiodic_t=True):
    """bhat_e = A_ee^-1 (b_e + kappa H_eo A_oo^-1 b_o)."""
    bo = twist_inv(odd_mask(dims) * b, kappa, mu)
    return twist_inv(even_mask(dims) * b + kappa * hop_to(U, bo, dims, 0, antiperiodic_t),
                     kappa, mu)


def schur_reconstruct(U, x_e, b, dims, kappa, mu, antiperiodic_t=True):
    """Full solution: x_e on even sites, x_o = A_oo^-1 (b_o + kappa H_oe x_e) on odd."""
    xe = even_mask(dims) * x_e
    xo = twist_inv(odd_mask(dims) * b + kappa * hop_to(U, xe, dims, 1, antiperiodic_t),
                   kappa, mu)
    return xe + xo


def hop_at_site(U, psi, dims, site, antiperiodic_t=True):
    """(H psi) at one site (x, y, z, t), summed term by term (for sampled checks
    on lattices too large for the full-array form)."""
    g, _ = gamma_matrices()
    one = np.eye(4, dtype=np.complex128)
    lx, ly, lz, lt = dims
    L = (lx, ly, lz, lt)
    x = list(site)
    out = np.zeros((4, 3), dtype=np.complex128)
    for mu in range(4):
        xf = list(x)
        xf[mu] = (x[mu] + 1) % L[mu]
        xb = list(x)
        xb[mu] = (x[mu] - 1) % L[mu]
        sf = -1.0 if (mu == 3 and antiperiodic_t and x[3] == lt - 1) else 1.0
        sb = -1.0 if (mu == 3 and antiperiodic_t and x[3] == 0) else 1.0
        u_here = U[x[3], x[2], x[1], x[0], mu]
        u_back = U[xb[3], xb[2], xb[1], xb[0], mu]
        pf = sf * psi[xf[3], xf[2], xf[1], xf[0]]
        pb = sb * psi[xb[3], xb[2], xb[1], xb[0]]
        out += (one - g[mu]) @ (pf @ u_here.T)
        out += (one + g[mu]) @ (pb @ np.conj(u_back))
    return out


def dense_dtm(U, dims, kappa, mu, antiperiodic_t=True):
    """D_tm as a dense (12V x 12V) matrix, column j = D_tm applied to unit vector j.

    Row/column index = 12 * site + 3 * spin + colour with the lexicographic site.
    """
    lx, ly, lz, lt = dims
    n = 12 * lx * ly * lz * lt
    out = np.empty((n, n), dtype=np.complex128)
    chunk = 384
    for j0 in range(0, n, chunk):
        j1 = min(n, j0 + chunk)
        e = np.zeros((j1 - j0, n), dtype=np.complex128)
        e[np.arange(j1 - j0), np.arange(j0, j1)] = 1.0
        e = e.reshape(j1 - j0, lt, lz, ly, lx, 4, 3)
        out[:, j0:j1] = dtm(U, e, dims, kappa, mu, antiperiodic_t).reshape(j1 - j0, n).T
    return out
