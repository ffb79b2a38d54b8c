"""Seeded synthetic inputs: gauge links, gauge transformations, random spinors.

This module holds input generators only -- none of the method's arithmetic --
so that the CUDA path and the CPU oracle can be fed identical fields.  The
ensemble the paper measures on (ETMC B55, 32^3 x 64, Sec. 3) is not
available; near-unit random SU(3) links stand in for it:

    U_mu(x) = exp(i eps H),  H = (A + A^dagger)/2 - tr(.)/3,  A_ij ~ complex N(0, 1),

computed by scaling and squaring of a Taylor series, then re-unitarised
(Gram-Schmidt on rows 1 and 2, row 3 = conj(row1 x row2)) so that every link
is exactly SU(3) to rounding.  Optional APE smearing (staple weight alpha,
followed by projection back to SU(3)) shapes the field further.

Layouts match the library's canonical host format:
    U   complex128 [T, Z, Y, X, 4, 3, 3]  (mu = 0:x, 1:y, 2:z, 3:t)
    psi complex128 [T, Z, Y, X, 4, 3]
"""
import numpy as np


def _expm_i_herm(h, eps):
    """exp(i eps h) for a stack of 3x3 hermitian matrices (scaling and squaring)."""
    x = 1j * eps * h
    squarings = 4
    x = x / float(2 ** squarings)
    out = np.broadcast_to(np.eye(3, dtype=np.complex128), x.shape).copy()
    term = out.copy()
    for k in range(1, 11):
        term = term @ x / k
        out = out + term
    for _ in range(squarings):
        out = out @ out
    return out


def reunitarise(m):
    """Project a stack of 3x3 matrices onto SU(3) by Gram-Schmidt of rows 1-2."""
    r1 = m[..., 0, :]
    r1 = r1 / np.linalg.norm(r1, axis=-1, keepdims=True)
    r2 = m[..., 1, :]
    r2 = r2 - np.sum(np.conj(r1) * r2, axis=-1, keepdims=True) * r1
    r2 = r2 / np.linalg.norm(r2, axis=-1, keepdims=True)
    r3 = np.conj(np.cross(r1, r2))
    return np.stack([r1, r2, r3], axis=-2)


def random_hermitian_traceless(rng, shape):
    a = rng.standard_normal(shape + (3, 3)) + 1j * rng.standard_normal(shape + (3, 3))
    h = 0.5 * (a + np.conj(np.swapaxes(a, -1, -2)))
    tr = np.trace(h, axis1=-2, axis2=-1)[..., None, None]
    return h - tr / 3.0 * np.eye(3)


def random_su3(rng, shape, eps):
    return reunitarise(_expm_i_herm(random_hermitian_traceless(rng, shape), eps))


def gauge_field(dims, eps, seed, ape_steps=0, ape_alpha=0.5):
    """Seeded links U = exp(i eps H) on a (Lx, Ly, Lz, T) lattice.

    eps = 0 gives the free field (all links 1).  Generated in slices of
    timeslices to bound the temporary memory on large lattices.
    """
    lx, ly, lz, lt = dims
    rng = np.random.default_rng(seed)
    U = np.empty((lt, lz, ly, lx, 4, 3, 3), dtype=np.complex128)
    if eps == 0.0:
        U[...] = np.eye(3)
    else:
        step = max(1, (1 << 18) // (lx * ly * lz))
        for t0 in range(0, lt, step):
            t1 = min(lt, t0 + step)
            U[t0:t1] = random_su3(rng, (t1 - t0, lz, ly, lx, 4), eps)
    for _ in range(ape_steps):
        U = ape_smear(U, ape_alpha)
    return U


def _shift(a, mu, step):
    """a(x + step * mu) for a field with leading [T, Z, Y, X] axes (periodic)."""
    axis = {0: 3, 1: 2, 2: 1, 3: 0}[mu]
    return np.roll(a, -step, axis=axis)


def ape_smear(U, alpha):
    """One APE step: V = (1 - alpha) U + (alpha / 6) sum of staples, projected to SU(3).

    Staples are built from periodic links (the smearing only shapes the input
    field; the fermion boundary sign is applied later by the operator).
    """
    dag = lambda m: np.conj(np.swapaxes(m, -1, -2))
    new = np.empty_like(U)
    for mu in range(4):
        st = np.zeros(U.shape[:4] + (3, 3), dtype=np.complex128)
        for nu in range(4):
            if nu == mu:
                continue
            u_nu = U[..., nu, :, :]
            u_mu_nu = _shift(U[..., mu, :, :], nu, 1)
            u_nu_mu = _shift(U[..., nu, :, :], mu, 1)
            st += u_nu @ u_mu_nu @ dag(u_nu_mu)
            u_nu_b = _shift(U[..., nu, :, :], nu, -1)
            u_mu_b = _shift(U[..., mu, :, :], nu, -1)
            u_nu_mb = _shift(_shift(U[..., nu, :, :], nu, -1), mu, 1)
            st += dag(u_nu_b) @ u_mu_b @ u_nu_mb
        new[..., mu, :, :] = reunitarise((1.0 - alpha) * U[..., mu, :, :] + alpha / 6.0 * st)
    return new


def gauge_transform(dims, seed, eps=1.0):
    """Random site-local SU(3) matrices G(x): [T, Z, Y, X, 3, 3]."""
    lx, ly, lz, lt = dims
    rng = np.random.default_rng(seed)
    return random_su3(rng, (lt, lz, ly, lx), eps)


def transform_links(U, G):
    """U^G_mu(x) = G(x) U_mu(x) G(x + mu)^dagger."""
    out = np.empty_like(U)
    for mu in range(4):
        g_fwd = _shift(G, mu, 1)
        out[..., mu, :, :] = G @ U[..., mu, :, :] @ np.conj(np.swapaxes(g_fwd, -1, -2))
    return out


def transform_spinor(psi, G):
    """(G psi)(x) = G(x) psi(x), colour acting on the last axis."""
    return np.einsum('tzyxab,...tzyxsb->...tzyxsa', G, psi)


def random_spinor(dims, seed, batch=()):
    lx, ly, lz, lt = dims
    rng = np.random.default_rng(seed)
    shape = tuple(batch) + (lt, lz, ly, lx, 4, 3)
    return rng.standard_normal(shape) + 1j * rng.standard_normal(shape)


def default_momenta(n_q):
    """Momentum lists (integer n, q = 2 pi n / L) used by the synthetic workloads.

    4: {0, e_x, e_y, e_z};  7: {0, +-e_x, +-e_y, +-e_z};
    13: 7 plus {+-(e_x+e_y), +-(e_x+e_z), +-(e_y+e_z)}.
    """
    if n_q == 1:
        return [(0, 0, 0)]
    if n_q == 4:
        return [(0, 0, 0), (1, 0, 0), (0, 1, 0), (0, 0, 1)]
    base = [(0, 0, 0), (1, 0, 0), (-1, 0, 0), (0, 1, 0), (0, -1, 0), (0, 0, 1), (0, 0, -1)]
    if n_q == 7:
        return base
    if n_q == 13:
        return base + [(1, 1, 0), (-1, -1, 0), (1, 0, 1), (-1, 0, -1), (0, 1, 1), (0, -1, -1)]
    raise ValueError("n_q must be 1, 4, 7 or 13")
