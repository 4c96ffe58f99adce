"""Pins for the oracle's Philox4x32-10 and uniform-double construction."""
import numpy as np

from conftest import GOLDEN
from oracle import philox


def _kat_rows():
    rows = []
    with open(f"{GOLDEN}/philox4x32_10_kat.txt") as f:
        for line in f:
            line = line.split("#", 1)[0].strip()
            if not line:
                continue
            ctr, key, out = (p.split() for p in line.split(";"))
            rows.append(([int(v, 16) for v in ctr], [int(v, 16) for v in key],
                         [int(v, 16) for v in out]))
    return rows


def test_known_answer_vectors():
    rows = _kat_rows()
    assert len(rows) == 3
    for ctr, key, out in rows:
        got = philox.philox4x32_10(np.array(ctr), np.array(key))
        assert [int(v) for v in got] == out


def test_vectorised_matches_scalar():
    rng = np.random.default_rng(0)
    ctr = rng.integers(0, 2**32, size=(17, 4), dtype=np.uint64)
    key = np.array([0x12345678, 0x9ABCDEF0], dtype=np.uint64)
    batch = philox.philox4x32_10(ctr, key)
    for i in range(17):
        assert np.array_equal(batch[i], philox.philox4x32_10(ctr[i], key))


def test_uniform53_extremes_and_range():
    assert philox.uniform53(np.array([0, 0], dtype=np.uint64)) == 0.0
    top = philox.uniform53(np.array([0xFFFFFFFF, 0xFFFFFFFF], dtype=np.uint64))
    assert top == 1.0 - 2.0 ** -53
    u = philox.swarm_uniform(7, np.arange(1000), 3, 1, philox.STREAM_P1)
    assert np.all((u >= 0) & (u < 1))
    # mean of 1000 U[0,1) draws: within 5 standard errors of 1/2
    assert abs(u.mean() - 0.5) < 5 * (1 / np.sqrt(12 * 1000))


def test_uniform53_takes_the_high_bits_of_r0_then_r1():
    # double = ((r0 >> 5) * 2^26 + (r1 >> 6)) * 2^-53: r0 gives the top 27 bits
    w = lambda r0, r1: np.array([r0, r1], dtype=np.uint64)
    assert philox.uniform53(w(0x80000000, 0)) == 0.5
    assert philox.uniform53(w(0, 0x80000000)) == 2.0 ** -28
    assert philox.uniform53(w(0xFFFFFFFF, 0)) == (2.0 ** 27 - 1) * 2.0 ** -27
    assert philox.uniform53(w(0, 0xFFFFFFFF)) == (2.0 ** 26 - 1) * 2.0 ** -53
    assert philox.uniform53(w(0x00000020, 0x00000040)) == 2.0 ** -27 + 2.0 ** -53
    # the bits dropped by the shifts do not count
    assert philox.uniform53(w(0x1F, 0x3F)) == 0.0


def test_streams_are_distinct():
    a = philox.swarm_uniform(1, 0, np.arange(8), 0, philox.STREAM_P1)
    b = philox.swarm_uniform(1, 0, np.arange(8), 0, philox.STREAM_P2)
    c = philox.swarm_uniform(2, 0, np.arange(8), 0, philox.STREAM_P1)
    assert not np.any(a == b) and not np.any(a == c)
