"""Philox4x32-10 counter-based generator and Box-Muller normals (oracle side).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

The paper draws the n x l Gaussian test matrix G "using a random number
generator" (Section 3, Step 1) and reports that the quality of the
pseudorandom numbers hardly matters (Section 5, opening paragraphs); when the
same matrix must be regenerated it restarts the generator from the same seed
(Section 5.1, third example).  To make G a function of a seed that two
independent implementations can reproduce, both sides implement Philox4x32-10
from its published definition (Salmon, Moraes, Dror, Shaw, "Parallel random
numbers: as easy as 1, 2, 3", SC'11):

  round:   (hi0, lo0) = mulhilo32(0xD2511F53, c0)
           (hi1, lo1) = mulhilo32(0xCD9E8D57, c2)
           c' = (hi1 ^ c1 ^ k0, lo1, hi0 ^ c3 ^ k1, lo0)
  key bump between rounds: k0 += 0x9E3779B9, k1 += 0xBB67AE85 (mod 2^32)
  10 rounds, 9 key bumps.

Stream layout (shared convention, not arithmetic of the method):
  key      = (seed & 0xffffffff, seed >> 32)
  counter  = (p, 0, domain, 0) for pair index p
  u1 = ((a >> 5) * 2^26 + (b >> 6) + 0.5) / 2^53 from words (a, b)
  u2 likewise from words (c, d)
  z0 = sqrt(-2 ln u1) cos(2 pi u2), z1 = sqrt(-2 ln u1) sin(2 pi u2)
  element 2p <- z0, element 2p+1 <- z1 (row-major over the matrix)
Domain 0 is G.
"""
import numpy as np

_M0 = np.uint64(0xD2511F53)
_M1 = np.uint64(0xCD9E8D57)
_W0 = np.uint32(0x9E3779B9)
_W1 = np.uint32(0xBB67AE85)
_MASK = np.uint64(0xFFFFFFFF)

DOMAIN_G = 0


def philox4x32_10(ctr, key):
    """Apply Philox4x32-10 to counters ``ctr`` (shape (N, 4), uint32) under
    ``key`` (two uint32 words, or arrays of shape (N,)).  Returns (N, 4)."""
    c = [np.asarray(ctr[:, j], dtype=np.uint64) for j in range(4)]
    k0 = np.asarray(key[0], dtype=np.uint32).astype(np.uint64)
    k1 = np.asarray(key[1], dtype=np.uint32).astype(np.uint64)
    for rnd in range(10):
        if rnd > 0:
            k0 = (k0 + np.uint64(_W0)) & _MASK
            k1 = (k1 + np.uint64(_W1)) & _MASK
        p0 = _M0 * c[0]
        p1 = _M1 * c[2]
        hi0, lo0 = p0 >> np.uint64(32), p0 & _MASK
        hi1, lo1 = p1 >> np.uint64(32), p1 & _MASK
        c = [hi1 ^ c[1] ^ k0, lo1, hi0 ^ c[3] ^ k1, lo0]
    return np.stack([x.astype(np.uint32) for x in c], axis=1)


def uniform_pairs(seed, domain, npairs):
    """Two (0,1) uniforms per counter, 53-bit resolution: (u1, u2)."""
    seed = int(seed)
    key = (np.uint32(seed & 0xFFFFFFFF), np.uint32((seed >> 32) & 0xFFFFFFFF))
    p = np.arange(npairs, dtype=np.uint64)
    ctr = np.zeros((npairs, 4), dtype=np.uint32)
    ctr[:, 0] = (p & _MASK).astype(np.uint32)
    ctr[:, 1] = (p >> np.uint64(32)).astype(np.uint32)
    ctr[:, 2] = np.uint32(domain)
    w = philox4x32_10(ctr, key).astype(np.float64)
    scale = 2.0 ** -53
    u1 = (np.floor(w[:, 0] / 32.0) * 67108864.0 + np.floor(w[:, 1] / 64.0) + 0.5) * scale
    u2 = (np.floor(w[:, 2] / 32.0) * 67108864.0 + np.floor(w[:, 3] / 64.0) + 0.5) * scale
    return u1, u2


def gaussian(seed, domain, count):
    """``count`` standard normals (FP64) by Box-Muller on Philox uniforms."""
    npairs = (count + 1) // 2
    u1, u2 = uniform_pairs(seed, domain, npairs)
    r = np.sqrt(-2.0 * np.log(u1))
    t = 2.0 * np.pi * u2
    z = np.empty(2 * npairs, dtype=np.float64)
    z[0::2] = r * np.cos(t)
    z[1::2] = r * np.sin(t)
    return z[:count]


def gaussian_matrix(seed, rows, cols, domain=DOMAIN_G):
    """rows x cols row-major standard-normal matrix (the test matrix G)."""
    return gaussian(seed, domain, rows * cols).reshape(rows, cols)
