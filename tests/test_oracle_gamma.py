"""Pins for oracle.gamma: the Euclidean Clifford algebra and the Gamma basis.

The gamma basis is a reading (the paper does not print one); what any valid
basis must satisfy is fixed by the algebra: {gamma_mu, gamma_nu} = 2 delta,
hermiticity, gamma_5 = gamma_1 gamma_2 gamma_3 gamma_4 anticommuting with all
gamma_mu, and the 16 insertions forming an orthogonal basis of 4x4 matrices.
"""
import numpy as np

from oracle.gamma import gamma_matrices, gamma_list


def test_clifford_and_hermitian():
    g, g5 = gamma_matrices()
    for m in range(4):
        assert np.allclose(g[m], g[m].conj().T)
        for n in range(4):
            anti = g[m] @ g[n] + g[n] @ g[m]
            assert np.allclose(anti, 2.0 * (m == n) * np.eye(4))
        assert np.allclose(g5 @ g[m] + g[m] @ g5, 0)
    assert np.allclose(g5 @ g5, np.eye(4))
    assert np.allclose(g5, g5.conj().T)


def test_gamma5_is_chiral_diagonal():
    # chiral basis: gamma_5 = diag(1, 1, -1, -1), so the twist is a per-spin phase
    _, g5 = gamma_matrices()
    assert np.allclose(g5, np.diag([1, 1, -1, -1]))


def test_gamma_list_is_orthogonal_basis():
    G = gamma_list()
    assert G.shape == (16, 4, 4)
    gram = np.einsum('aij,bij->ab', G.conj(), G)   # tr(G_a^dag G_b)
    assert np.allclose(gram, 4.0 * np.eye(16))
    # every insertion is a signed permutation-like matrix with entries in {0, +-1, +-i}
    for m in G:
        nz = m[np.abs(m) > 1e-12]
        assert nz.size == 4
        assert np.allclose(np.abs(nz), 1.0)
        assert np.allclose(np.minimum(np.abs(nz.real), np.abs(nz.imag)), 0)
        assert np.allclose(m @ m.conj().T, np.eye(4))


def test_gamma_list_order():
    g, g5 = gamma_matrices()
    G = gamma_list()
    assert np.allclose(G[0], np.eye(4))
    for m in range(4):
        assert np.allclose(G[1 + m], g[m])
        assert np.allclose(G[6 + m], g[m] @ g5)
    assert np.allclose(G[5], g5)
    pairs = ((0, 1), (0, 2), (0, 3), (1, 2), (1, 3), (2, 3))
    for k, (m, n) in enumerate(pairs):
        s = G[10 + k]
        assert np.allclose(s, s.conj().T)               # sigma_mu_nu hermitian
        assert np.allclose(s, -0.5j * (g[n] @ g[m] - g[m] @ g[n]))
        assert np.allclose(s, 1j * g[m] @ g[n])          # m != n: gamma_m gamma_n antisymmetric
