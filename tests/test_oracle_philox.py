"""Pins for oracle.philox: the Z4/Z2 noise of Sec. 2.1 (Eq. 2.1).

Eq. 2.1 fixes what the method needs from the noise: components in a Z4 (or
Z2) representation with (1/N) sum eta = O(1/sqrt N) and
(1/N) sum eta eta^dag = 1 + O(1/sqrt N).  The bit stream itself is the
Philox4x32-10 generator (Salmon et al., SC'11).  Its exact bits are pinned by
the known-answer vectors published with the generator (Random123
distribution, philox4x32 with 10 rounds), the noise map by a site decoded by
hand, and the stream's quality by bit statistics, avalanche (full diffusion
of counter and key bits after ten rounds) and the absence of collisions.
"""
import numpy as np

from oracle import philox

DIMS = (4, 4, 4, 4)


# Published known-answer vectors of philox4x32-10 (Salmon, Moraes, Dror and
# Shaw, SC'11; Random123 distribution): counter (c0..c3), key (k0, k1) ->
# output words 0..3.
KAT = [
    ((0x00000000, 0x00000000, 0x00000000, 0x00000000), (0x00000000, 0x00000000),
     (0x6627e8d5, 0xe169c58d, 0xbc57ac4c, 0x9b00dbd8)),
    ((0xffffffff, 0xffffffff, 0xffffffff, 0xffffffff), (0xffffffff, 0xffffffff),
     (0x408f276d, 0x41c83b0e, 0xa20bc7c6, 0x6d5451fd)),
    ((0x243f6a88, 0x85a308d3, 0x13198a2e, 0x03707344), (0xa4093822, 0x299f31d0),
     (0xd16cfe09, 0x94fdcceb, 0x5001e420, 0x24126ea1)),
]


def test_known_answer_vectors():
    for ctr, key, want in KAT:
        got = philox.philox4x32_10(*[np.array([c], dtype=np.uint64) for c in ctr], key[0], key[1])
        assert tuple(int(w[0]) for w in got) == want


def test_known_answer_vectors_vectorised():
    # the same vectors as one array call (the noise map evaluates whole lattices at once)
    ctr = np.array([k[0] for k in KAT], dtype=np.uint64).T
    for i, (_, key, want) in enumerate(KAT):
        got = philox.philox4x32_10(ctr[0], ctr[1], ctr[2], ctr[3], key[0], key[1])
        assert tuple(int(w[i]) for w in got) == want


def test_noise_map_hand_decoded_site():
    """seed -> key (low word, high word), site (x, y, z, t) -> counter word 0 =
    x + Lx (y + Ly (z + Lz t)), source -> counter word 1, and bit 2a (2a + 1)
    of output word 0 -> sign of Re (Im) of component a = 3 spin + colour."""
    dims = (4, 2, 6, 2)                       # Lx, Ly, Lz, T (all different)
    seed = (0x00000005 << 32) | 0x00000007    # key (7, 5)
    x, y, z, t, src = 3, 1, 4, 1, 9
    site = x + 4 * (y + 2 * (z + 6 * t))      # = 71
    w0 = int(philox.philox4x32_10(np.array([site], np.uint64), np.array([src], np.uint64),
                                  np.array([0], np.uint64), np.array([0], np.uint64), 7, 5)[0][0])
    eta4 = philox.noise(seed, src, dims, 4)[t, z, y, x]
    eta2 = philox.noise(seed, src, dims, 2)[t, z, y, x]
    r = 1.0 / np.sqrt(2.0)
    for spin in range(4):
        for colour in range(3):
            a = 3 * spin + colour
            re = -1.0 if (w0 >> (2 * a)) & 1 else 1.0
            im = -1.0 if (w0 >> (2 * a + 1)) & 1 else 1.0
            assert eta4[spin, colour] == complex(re * r, im * r)
            assert eta2[spin, colour] == complex(re, 0.0)
    # the key is (low, high) of the seed, not (high, low)
    swapped = int(philox.philox4x32_10(np.array([site], np.uint64), np.array([src], np.uint64),
                                       np.array([0], np.uint64), np.array([0], np.uint64), 5, 7)[0][0])
    assert swapped != w0
    assert int(philox.noise_bits(seed, np.array([site], np.uint64), src)[0]) == w0


def _many(n_src, kind=4, seed=1234, dims=DIMS):
    return np.array([philox.noise(seed, j, dims, kind).reshape(-1) for j in range(n_src)])


def test_z4_values_and_modulus():
    eta = _many(8)
    assert np.allclose(np.abs(eta), 1.0, atol=0, rtol=1e-15)
    s = np.sqrt(2.0)
    assert set(np.round(eta.real * s).astype(int).ravel()) <= {-1, 1}
    assert set(np.round(eta.imag * s).astype(int).ravel()) <= {-1, 1}


def test_z2_is_real_sign_of_z4():
    z4 = philox.noise(7, 3, DIMS, 4)
    z2 = philox.noise(7, 3, DIMS, 2)
    assert np.all(z2.imag == 0)
    assert np.array_equal(np.sign(z2.real), np.sign(z4.real))


def test_moments_eq_2_1():
    n = 512
    eta = _many(n)                                   # [N, 12V]
    mean = eta.mean(axis=0)
    # each component's mean has variance 1/N: |mean| * sqrt(N) is O(1)
    z = np.abs(mean) * np.sqrt(n)
    assert z.max() < 5.0
    assert 0.6 < np.sqrt(np.mean(z ** 2)) < 1.4
    # (1/N) sum eta eta^dag = 1 + O(1/sqrt N) on a block of components
    blk = eta[:, :96]
    m = blk.T @ blk.conj() / n
    assert np.allclose(np.diag(m), 1.0)               # |eta_a| = 1 exactly
    off = m - np.diag(np.diag(m))
    zo = np.abs(off[~np.eye(96, dtype=bool)]) * np.sqrt(n)
    assert zo.max() < 5.5
    assert 0.8 < np.sqrt(np.mean(zo ** 2)) < 1.2
    # Z4: <eta_a^2> -> 0 ;  Z2: eta_a^2 = 1
    assert np.abs((eta ** 2).mean(axis=0)).max() * np.sqrt(n) < 5.5
    assert np.allclose(_many(4, kind=2) ** 2, 1.0)


def test_bit_frequencies():
    w = philox.noise_bits(99, np.arange(1 << 16, dtype=np.uint64), 5).astype(np.uint64)
    bits = ((w[:, None] >> np.arange(32, dtype=np.uint64)[None, :]) & np.uint64(1)).astype(float)
    freq = bits.mean(axis=0)
    # binomial sd of a frequency over 2^16 draws is 1/512
    assert np.all(np.abs(freq - 0.5) < 5.0 / 512)


def test_avalanche_counter_and_key():
    rng = np.random.default_rng(0)
    base = rng.integers(0, 2 ** 32, size=(4096,), dtype=np.uint64)
    src = rng.integers(0, 2 ** 32, size=(4096,), dtype=np.uint64)
    ref = philox.noise_bits(12345, base, src).astype(np.uint64)
    popcount = lambda v: np.array([bin(int(a)).count("1") for a in v])
    for bit in (0, 7, 19, 31):
        flipped = philox.noise_bits(12345, base ^ np.uint64(1 << bit), src).astype(np.uint64)
        assert abs(popcount(ref ^ flipped).mean() - 16.0) < 0.5
        flipped = philox.noise_bits(12345, base, src ^ np.uint64(1 << bit)).astype(np.uint64)
        assert abs(popcount(ref ^ flipped).mean() - 16.0) < 0.5
    for kbit in (0, 33, 63):
        other = philox.noise_bits(12345 ^ (1 << kbit), base, src).astype(np.uint64)
        assert abs(popcount(ref ^ other).mean() - 16.0) < 0.5


def test_all_four_words_distinct_no_collisions():
    n = 1 << 15
    c = np.arange(n, dtype=np.uint64)
    z = np.zeros_like(c)
    w = philox.philox4x32_10(c, z, z, z, 1, 2)
    full = (w[0].astype(object) << 96) | (w[1].astype(object) << 64) | \
           (w[2].astype(object) << 32) | w[3].astype(object)
    assert len(set(full.tolist())) == n
    assert len(set(w[0].tolist())) > n - 4          # 32-bit birthday bound: ~0.1 expected


def test_sources_and_seeds_independent():
    a = philox.noise(1, 0, DIMS, 4)
    assert not np.array_equal(a, philox.noise(1, 1, DIMS, 4))
    assert not np.array_equal(a, philox.noise(2, 0, DIMS, 4))
    assert np.array_equal(a, philox.noise(1, 0, DIMS, 4))
