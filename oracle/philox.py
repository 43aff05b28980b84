"""Philox-4x32-10 counter-based generator (oracle; test infrastructure only).

Definition: Salmon, Moraes, Dror, Shaw, "Parallel Random Numbers: As Easy as 1, 2, 3"
(SC'11), the Philox-4x32 bijection with 10 rounds.  One round maps the counter
(c0, c1, c2, c3) under key (k0, k1) to

    (hi(M1*c2) ^ c1 ^ k0,  lo(M1*c2),  hi(M0*c0) ^ c3 ^ k1,  lo(M0*c0))

with M0 = 0xD2511F53, M1 = 0xCD9E8D57, and the key is bumped by the Weyl constants
(0x9E3779B9, 0xBB67AE85) between rounds.

The paper keeps source and target processes aligned by seeding one generator stream
RNG_{sigma,tau} identically on both sides (Methods, "Point-to-point MPI
communication").  A counter-based generator keyed by global ids gives the same
alignment with no state at all: the draw for a synapse depends only on its counter.

Pinned by tests/test_oracle_philox.py: published known-answer vectors and curand's
host Philox generator (a library routine), plus bijectivity on a sample.
"""
from __future__ import annotations

import numpy as np

M0 = 0xD2511F53
M1 = 0xCD9E8D57
W0 = 0x9E3779B9
W1 = 0xBB67AE85
MASK = np.uint64(0xFFFFFFFF)

# counter word 3 ("purpose") of each stream the method draws from
PURPOSE_SYNAPSE = 0      # source choice, delay, weight of one synapse / draw
PURPOSE_FT_TARGET = 1    # target choice of a fixed-total draw
PURPOSE_PB_TEST = 2      # inclusion test of pairwise Bernoulli (4 pairs per call)
PURPOSE_POISSON = 3      # Poisson drive counts of four consecutive neurons in one step
PURPOSE_VINIT = 4        # initial membrane potential
PURPOSE_PB_GAP = 5       # gap between kept pairs of pairwise Bernoulli by geometric skipping


def philox4x32_10(c0, c1, c2, c3, k0, k1):
    """Vectorised Philox-4x32-10.  Arguments are integers or uint64 arrays holding
    32-bit values; returns four uint64 arrays of 32-bit words."""
    c0 = np.asarray(c0, dtype=np.uint64) & MASK
    c1 = np.asarray(c1, dtype=np.uint64) & MASK
    c2 = np.asarray(c2, dtype=np.uint64) & MASK
    c3 = np.asarray(c3, dtype=np.uint64) & MASK
    k0 = np.uint64(int(k0) & 0xFFFFFFFF)
    k1 = np.uint64(int(k1) & 0xFFFFFFFF)
    m0, m1 = np.uint64(M0), np.uint64(M1)
    for _ in range(10):
        p0 = m0 * c0            # 32x32 -> 64 bit, exact in uint64
        p1 = m1 * c2
        hi0, lo0 = p0 >> np.uint64(32), p0 & MASK
        hi1, lo1 = p1 >> np.uint64(32), p1 & MASK
        c0, c1, c2, c3 = hi1 ^ c1 ^ k0, lo1, hi0 ^ c3 ^ k1, lo0
        k0 = np.uint64((int(k0) + W0) & 0xFFFFFFFF)
        k1 = np.uint64((int(k1) + W1) & 0xFFFFFFFF)
    return c0, c1, c2, c3


def key_of(seed: int):
    """Key words of a 64-bit seed: (low 32 bits, high 32 bits)."""
    seed = int(seed) & 0xFFFFFFFFFFFFFFFF
    return seed & 0xFFFFFFFF, seed >> 32


def stream(counter, word2: int, purpose: int, seed: int):
    """Draw the stream block for a 64-bit ``counter`` (array) of one stream:
    ctr = (counter lo32, counter hi32, word2, purpose), key = seed."""
    counter = np.asarray(counter, dtype=np.uint64)
    k0, k1 = key_of(seed)
    return philox4x32_10(counter & MASK, counter >> np.uint64(32),
                         np.full(counter.shape, word2, dtype=np.uint64),
                         np.full(counter.shape, purpose, dtype=np.uint64), k0, k1)
