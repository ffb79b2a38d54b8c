"""Gamma matrices and the Gamma insertion list (oracle; test infrastructure).

The paper never writes a gamma basis (Sec. 2.3 only says operators are
expressed in the twisted basis).  Reading used here: the Euclidean chiral
basis with hermitian gamma_mu,

    gamma_k = [[0, -i sigma_k], [i sigma_k, 0]]   (k = 1, 2, 3 -> x, y, z)
    gamma_4 = [[0, 1], [1, 0]]                     (t)
    gamma_5 = gamma_1 gamma_2 gamma_3 gamma_4 = diag(1, 1, -1, -1).

Insertion list order (also a reading; the paper is silent):
    0: 1, 1-4: gamma_1..gamma_4, 5: gamma_5, 6-9: gamma_mu gamma_5,
    10-15: sigma_{mu nu} = (i/2)[gamma_mu, gamma_nu] for
           (mu,nu) = (1,2), (1,3), (1,4), (2,3), (2,4), (3,4).
"""
import numpy as np

_SIGMA = (
    np.array([[0, 1], [1, 0]], dtype=np.complex128),
    np.array([[0, -1j], [1j, 0]], dtype=np.complex128),
    np.array([[1, 0], [0, -1]], dtype=np.complex128),
)


def gamma_matrices():
    """Return (gamma_mu for mu = x, y, z, t as a (4, 4, 4) array, gamma_5)."""
    z = np.zeros((2, 2), dtype=np.complex128)
    one = np.eye(2, dtype=np.complex128)
    g = [np.block([[z, -1j * s], [1j * s, z]]) for s in _SIGMA]
    g.append(np.block([[z, one], [one, z]]))
    g = np.array(g)
    g5 = g[0] @ g[1] @ g[2] @ g[3]
    return g, g5


def gamma_list():
    """The 16 insertions Gamma_0..Gamma_15 in the order of the module docstring."""
    g, g5 = gamma_matrices()
    out = [np.eye(4, dtype=np.complex128)]
    out += [g[m] for m in range(4)]
    out.append(g5)
    out += [g[m] @ g5 for m in range(4)]
    for (m, n) in ((0, 1), (0, 2), (0, 3), (1, 2), (1, 3), (2, 3)):
        out.append(0.5j * (g[m] @ g[n] - g[n] @ g[m]))
    return np.array(out)
