"""Philox4x32-10 and the Z4 / Z2 noise map (oracle; test infrastructure).

Sec. 2.1 (Eq. 2.1) asks for sources whose components are drawn from a Z2 or
Z4 representation, with zero mean and unit second moment; Sec. 3 says they are
generated on the fly.  The generator is not named by the paper; the reading
here is the counter-based Philox4x32-10 of Salmon, Moraes, Dror and Shaw,
"Parallel random numbers: as easy as 1, 2, 3" (SC'11), written from that
paper's description:

* state: four 32-bit counter words and a two-word key;
* one round multiplies counter word 0 by M0 and word 2 by M1 (32x32 -> 64
  bits), and returns (hi(M1*c2) ^ c1 ^ k0, lo(M1*c2), hi(M0*c0) ^ c3 ^ k1,
  lo(M0*c0));
* ten rounds; the key is advanced by the Weyl constants (W0, W1) between
  rounds.

Noise map (reading): key = (seed & 0xffffffff, seed >> 32), counter =
(lexicographic site index, source index, 0, 0).  Output word 0 carries the
signs of the 12 spin-colour components a = 3*spin + colour: bit 2a set makes
Re(eta_a) negative, bit 2a+1 set makes Im(eta_a) negative.  Z4 entries are
(+-1 +- i)/sqrt(2) (unit modulus, as Eq. 2.1 needs); Z2 entries are +-1 from
bit 2a alone.

Pins: the round function is checked against the known-answer vectors that
Salmon et al. publish with their Random123 distribution for philox4x32-10
(counter and key all zero, all ones, and the digits of pi); the noise map
(seed -> key, site/source -> counter, word-0 bits -> signs) against a
hand-decoded site; the moments of Eq. 2.1 by statistics.
"""
import numpy as np

M0 = 0xD2511F53
M1 = 0xCD9E8D57
W0 = 0x9E3779B9
W1 = 0xBB67AE85
_MASK = np.uint64(0xFFFFFFFF)


def philox4x32_10(c0, c1, c2, c3, k0, k1):
    """Ten Philox4x32 rounds on arrays of counters (any shape, uint32-valued).

    k0, k1 are Python ints (the key).  Returns four uint32 arrays.
    """
    c0 = np.asarray(c0, dtype=np.uint64)
    c1 = np.asarray(c1, dtype=np.uint64)
    c2 = np.asarray(c2, dtype=np.uint64)
    c3 = np.asarray(c3, dtype=np.uint64)
    key0, key1 = int(k0) & 0xFFFFFFFF, int(k1) & 0xFFFFFFFF
    for rnd in range(10):
        if rnd > 0:
            key0 = (key0 + W0) & 0xFFFFFFFF
            key1 = (key1 + W1) & 0xFFFFFFFF
        p0 = np.uint64(M0) * c0          # exact: both factors < 2**32
        p1 = np.uint64(M1) * c2
        hi0, lo0 = p0 >> np.uint64(32), p0 & _MASK
        hi1, lo1 = p1 >> np.uint64(32), p1 & _MASK
        c0, c1, c2, c3 = (hi1 ^ c1 ^ np.uint64(key0), lo1,
                          hi0 ^ c3 ^ np.uint64(key1), lo0)
    return (c0.astype(np.uint32), c1.astype(np.uint32),
            c2.astype(np.uint32), c3.astype(np.uint32))


def noise_bits(seed, site, source):
    """Word 0 of Philox4x32-10 at counter (site, source, 0, 0), key from seed."""
    site = np.asarray(site, dtype=np.uint64)
    src = np.broadcast_to(np.asarray(source, dtype=np.uint64), site.shape)
    zero = np.zeros_like(site)
    w0, _, _, _ = philox4x32_10(site, src, zero, zero,
                                seed & 0xFFFFFFFF, (seed >> 32) & 0xFFFFFFFF)
    return w0


def noise(seed, source, dims, kind=4):
    """Noise source eta_source on the full lattice.

    dims = (Lx, Ly, Lz, T).  Returns complex128 array [T, Z, Y, X, 4, 3].
    kind = 4 for Z4, 2 for Z2.
    """
    lx, ly, lz, lt = dims
    vol = lx * ly * lz * lt
    w = noise_bits(seed, np.arange(vol, dtype=np.uint64), source)
    w = w.astype(np.uint64)
    a = np.arange(12, dtype=np.uint64)
    re_neg = (w[:, None] >> (2 * a)[None, :]) & np.uint64(1)
    sign_re = 1.0 - 2.0 * re_neg.astype(np.float64)
    if kind == 4:
        im_neg = (w[:, None] >> (2 * a + 1)[None, :]) & np.uint64(1)
        sign_im = 1.0 - 2.0 * im_neg.astype(np.float64)
        eta = (sign_re + 1j * sign_im) / np.sqrt(2.0)
    elif kind == 2:
        eta = sign_re.astype(np.complex128)
    else:
        raise ValueError("noise kind must be 4 (Z4) or 2 (Z2)")
    return eta.reshape(lt, lz, ly, lx, 4, 3)
