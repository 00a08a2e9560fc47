"""Oracle: Philox4x64-10 and the Gaussian test matrix Omega (Alg. RSVD step 1).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

Alg. RSVD (Sec. II.B) starts by drawing an n-by-l test matrix Omega with
independent standard normal entries; the paper notes that the quality of the
random numbers is not crucial.  The paper does not fix a generator, so this
build reads it as follows (one reading, applied identically by the CUDA path):

* Generator: Philox4x64 with 10 rounds, from Salmon, Moraes, Dror, Shaw,
  "Parallel random numbers: as easy as 1, 2, 3" (SC'11).  One bijection of a
  4 x 64-bit counter under a 2 x 64-bit key.  Written here with plain Python
  integers so that every 64 x 64 -> 128-bit product is exact.
* Key = (seed, stream): ``stream`` separates the matrices of a batch.
* Counter = (e // 4, 0, 0, 0) for the linear element index e = c * n + r of
  Omega[r, c] (column-major, so the first l columns of a wider draw equal a
  narrower draw: columns nest as l grows).
* Normal from two words by the Box-Muller transform:
  u = ((w >> 11) + 1/2) 2^-53, evaluated in FP64, lies in (0, 1] (never 0, so
  the logarithm is finite); z = sqrt(-2 ln u_a) cos(2 pi u_b) or ... sin(...).
  Words (w0, w1) give slots 0 (cos) and 1 (sin), words (w2, w3) give slots
  2 (cos) and 3 (sin); slot = e % 4.
"""
import math

import numpy as np

MASK64 = (1 << 64) - 1
# Philox4x64 multipliers and Weyl key increments, as published for Philox-4x64 (SC'11).
PHILOX_M0 = 0xD2E7470EE14C6C93
PHILOX_M1 = 0xCA5A826395121157
PHILOX_W0 = 0x9E3779B97F4A7C15  # golden ratio
PHILOX_W1 = 0xBB67AE8584CAA73B  # sqrt(3) - 1
PHILOX_ROUNDS = 10


def philox4x64(counter, key, rounds=PHILOX_ROUNDS):
    """Philox4x64-R bijection of one 4-word counter under a 2-word key.

    Each round multiplies words 0 and 2 by the two multipliers (full 128-bit
    product), and forms the new state (hi1 ^ x1 ^ k0, lo1, hi0 ^ x3 ^ k1, lo0);
    the key is bumped by the Weyl constants between rounds.
    """
    x0, x1, x2, x3 = (int(v) & MASK64 for v in counter)
    k0, k1 = (int(v) & MASK64 for v in key)
    for r in range(rounds):
        if r > 0:
            k0 = (k0 + PHILOX_W0) & MASK64
            k1 = (k1 + PHILOX_W1) & MASK64
        p0 = PHILOX_M0 * x0
        p1 = PHILOX_M1 * x2
        hi0, lo0 = p0 >> 64, p0 & MASK64
        hi1, lo1 = p1 >> 64, p1 & MASK64
        x0, x1, x2, x3 = hi1 ^ x1 ^ k0, lo1, hi0 ^ x3 ^ k1, lo0
    return (x0, x1, x2, x3)


def word_to_open_unit(w):
    """Top 53 bits of a 64-bit word mapped into (0, 1] (FP64 rounding may give 1)."""
    return ((w >> 11) + 0.5) * (2.0 ** -53)


def box_muller_block(words):
    """The four normals carried by one Philox output block, in slot order."""
    out = []
    for a, b in ((words[0], words[1]), (words[2], words[3])):
        ua = word_to_open_unit(a)
        ub = word_to_open_unit(b)
        rad = math.sqrt(-2.0 * math.log(ua))
        out.append(rad * math.cos(2.0 * math.pi * ub))
        out.append(rad * math.sin(2.0 * math.pi * ub))
    return out


def gaussian_test_matrix(n, l, seed, stream=0):
    """Omega: n-by-l standard normal test matrix (Alg. RSVD step 1), FP64."""
    total = n * l
    flat = np.empty(total, dtype=np.float64)
    for blk in range((total + 3) // 4):
        z = box_muller_block(philox4x64((blk, 0, 0, 0), (seed, stream)))
        for s in range(4):
            e = 4 * blk + s
            if e < total:
                flat[e] = z[s]
    # element e = c * n + r sits at Omega[r, c]
    return flat.reshape(l, n).T.copy()
