"""Philox4x32-10 counter-based generator, written from its published definition.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

Definition followed: J. K. Salmon, M. A. Moraes, R. O. Dror, D. E. Shaw,
"Parallel random numbers: as easy as 1, 2, 3", SC'11, section 3.2 (the
Philox S-box: two 32x32->64-bit multiplies per round, a Weyl sequence on the
key).  Known-answer vectors from the same authors' distribution pin it in
``tests/test_oracle_philox.py``.

Used by the particle swarm (Algorithm 1 step 3: random initial swarm; step 7:
"p1 and p2 are random constants between 0 and 1").  The counter layout and
the double construction are this project's reading (the paper names no
generator): counter = (generation, particle, dimension, stream), key =
(seed low word, seed high word), and a uniform double in [0, 1) from the
first two output words as ((r0 >> 5) * 2**26 + (r1 >> 6)) * 2**-53.
"""
import numpy as np

# Round multipliers and Weyl key increments of Philox4x32 (SC'11, table 2).
PHILOX_M0 = 0xD2511F53
PHILOX_M1 = 0xCD9E8D57
PHILOX_W0 = 0x9E3779B9
PHILOX_W1 = 0xBB67AE85
MASK32 = 0xFFFFFFFF

# Stream ids of the swarm's draws (fourth counter word).
STREAM_INIT_X = 0
STREAM_INIT_V = 1
STREAM_P1 = 2
STREAM_P2 = 3


def philox4x32_10(counter, key):
    """Philox4x32 with 10 rounds.

    counter: (..., 4) unsigned 32-bit words; key: (..., 2) words (broadcast).
    Returns (..., 4) uint32 output words.
    """
    ctr = np.asarray(counter, dtype=np.uint64) & MASK32
    k = np.asarray(key, dtype=np.uint64) & MASK32
    c0, c1, c2, c3 = (ctr[..., i].copy() for i in range(4))
    k0 = np.broadcast_to(k[..., 0], c0.shape).copy()
    k1 = np.broadcast_to(k[..., 1], c0.shape).copy()
    for rnd in range(10):
        if rnd > 0:
            k0 = (k0 + PHILOX_W0) & MASK32
            k1 = (k1 + PHILOX_W1) & MASK32
        p0 = np.uint64(PHILOX_M0) * c0          # < 2**64, exact in uint64
        p1 = np.uint64(PHILOX_M1) * c2
        hi0, lo0 = p0 >> np.uint64(32), p0 & np.uint64(MASK32)
        hi1, lo1 = p1 >> np.uint64(32), p1 & np.uint64(MASK32)
        c0, c1, c2, c3 = hi1 ^ c1 ^ k0, lo1, hi0 ^ c3 ^ k1, lo0
    return np.stack([c0, c1, c2, c3], axis=-1).astype(np.uint32)


def seed_key(seed):
    """64-bit seed -> Philox key (low word, high word)."""
    s = int(seed) & 0xFFFFFFFFFFFFFFFF
    return np.array([s & MASK32, s >> 32], dtype=np.uint64)


def uniform53(words):
    """Uniform double in [0, 1) from the first two 32-bit words (53 bits)."""
    w = np.asarray(words, dtype=np.uint64)
    hi = (w[..., 0] >> np.uint64(5)).astype(np.float64)   # 27 bits
    lo = (w[..., 1] >> np.uint64(6)).astype(np.float64)   # 26 bits
    return (hi * 67108864.0 + lo) * (1.0 / 9007199254740992.0)


def swarm_uniform(seed, gen, particle, dim, stream):
    """U[0,1) draw for one (generation, particle, dimension, stream) counter."""
    gen, particle, dim, stream = np.broadcast_arrays(
        np.asarray(gen, dtype=np.uint64), np.asarray(particle, dtype=np.uint64),
        np.asarray(dim, dtype=np.uint64), np.asarray(stream, dtype=np.uint64))
    ctr = np.stack([gen, particle, dim, stream], axis=-1)
    return uniform53(philox4x32_10(ctr, seed_key(seed)))
