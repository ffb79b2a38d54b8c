"""The contraction kernels take the 16 insertions from compiled codes (one
16-bit word per insertion: bits 0-1 the column mask m -- row a has its
non-zero in column a ^ m -- and bits 2 + 2a the power of i of that entry).
This CPU test reads the four code constants from the kernel header as text
and checks every one against the oracle's gamma matrices, so that a wrong
sign, phase or column in the compiled table fails without a GPU.
"""
import os
import re

import numpy as np

from oracle import gamma

HEADER = os.path.join(os.path.dirname(__file__), "..", "paper_1211_0126_gb300", "csrc", "contract.cuh")


def _codes():
    text = open(HEADER).read()
    words = {}
    for k in range(4):
        m = re.search(r"constexpr uint64_t kChiralCodes%d = (0x[0-9a-fA-F]+)ull;" % k, text)
        assert m is not None, "kChiralCodes%d not found" % k
        words[k] = int(m.group(1), 16)
    return [(words[k // 4] >> (16 * (k % 4))) & 0xFFFF for k in range(16)]


def _matrix(code):
    m = code & 3
    out = np.zeros((4, 4), dtype=np.complex128)
    for a in range(4):
        out[a, a ^ m] = 1j ** ((code >> (2 + 2 * a)) & 3)
    return out


def test_compiled_codes_equal_oracle_insertions():
    want = gamma.gamma_list()
    for k, code in enumerate(_codes()):
        assert code >> 10 == 0, k                     # only ten bits in use
        assert np.allclose(_matrix(code), want[k], atol=1e-14), k


def test_every_insertion_is_a_signed_permutation_with_xor_columns():
    # the property the compiled form relies on, checked on the oracle's own matrices
    for k, g in enumerate(gamma.gamma_list()):
        cols = [int(np.flatnonzero(np.abs(g[a]) > 1e-12)[0]) for a in range(4)]
        assert all(np.count_nonzero(np.abs(g[a]) > 1e-12) == 1 for a in range(4)), k
        assert len({a ^ c for a, c in enumerate(cols)}) == 1, k
        for a, c in enumerate(cols):
            assert min(abs(g[a, c] - 1j ** p) for p in range(4)) < 1e-12, k
