"""Pins of the bfloat16 storage model in oracle/precision.py.

bfloat16 is the upper 16 bits of IEEE-754 binary32.  A normal value has 8
significant bits, so the nearest-even rounding of the FP64 value x is fixed by
the format alone.  These tests check it against hand-worked values, ties,
the half-ulp error bound, and an independent method: the integer rounding of
the binary32 bit pattern (add 0x7FFF plus the lowest kept bit, then drop the
low 16 bits).  They also check how the model plugs into the IFCM loop.
"""
import numpy as np

from oracle import ifcm as O
from oracle.precision import round_bf16


def test_hand_worked_values():
    # 1/3 = 1.0101010101..b x 2^-2; 8 significant bits 1.0101010, the next bit
    # is 1 and bits follow, so round up to 1.0101011b x 2^-2 = 0.333984375
    assert round_bf16(1.0 / 3.0) == 0.333984375
    # 0.1 = 1.1001100110011..b x 2^-4 -> 1.1001101b x 2^-4 = 0.10009765625
    assert round_bf16(0.1) == 0.10009765625
    assert round_bf16(1.0) == 1.0 and round_bf16(0.0) == 0.0 and round_bf16(-2.5) == -2.5
    # spacing at 1 is 2^-7: 1 + 2^-8 is a tie -> even (1.0); 1 + 3 * 2^-8 is a
    # tie between 1 + 2^-7 (odd) and 1 + 2^-6 (even)
    assert round_bf16(1.0 + 2.0 ** -8) == 1.0
    assert round_bf16(1.0 + 3 * 2.0 ** -8) == 1.0 + 2.0 ** -6
    # just above a tie rounds up
    assert round_bf16(1.0 + 2.0 ** -8 + 2.0 ** -30) == 1.0 + 2.0 ** -7
    # 255/256 needs 8 significant bits and is representable; 511/512 is a
    # tie between 255/256 (odd last bit) and 1 (even)
    assert round_bf16(255.0 / 256.0) == 255.0 / 256.0
    assert round_bf16(511.0 / 512.0) == 1.0


def test_half_ulp_bound_and_idempotence():
    rng = np.random.default_rng(11)
    x = rng.random(100000) * 10.0 ** rng.integers(-12, 3, 100000)
    r = round_bf16(x)
    # x = f 2^e with f in [0.5, 1): the grid spacing is 2^(e-8), so the error
    # is at most half of it, 2^(e-9) (at most 2^-8 |x|)
    _, e = np.frexp(x)
    assert np.all(np.abs(r - x) <= np.ldexp(1.0, e - 9))
    assert np.all(np.abs(r - x) <= 2.0 ** -8 * np.abs(x))
    assert np.array_equal(round_bf16(r), r)
    # monotone
    xs = np.sort(x)
    assert np.all(np.diff(round_bf16(xs)) >= 0)


def test_matches_binary32_integer_rounding():
    rng = np.random.default_rng(12)
    x32 = (rng.random(200000) * 10.0 ** rng.integers(-15, 4, 200000)).astype(np.float32)
    x32[:4] = np.array([1.0 + 2.0 ** -8, 1.0 + 3 * 2.0 ** -8, 0.75, 2.0 ** -20],
                       dtype=np.float32)
    bits = x32.view(np.uint32).astype(np.uint64)
    rounded = ((bits + 0x7FFF + ((bits >> 16) & 1)) & 0xFFFF0000).astype(np.uint32)
    expect = rounded.view(np.float32).astype(np.float64)
    assert np.array_equal(round_bf16(x32.astype(np.float64)), expect)


def test_storage_model_in_the_loop():
    rng = np.random.default_rng(13)
    x = np.clip(np.repeat([0.1, 0.5, 0.9], 32).reshape(3, 4, 8) +
                0.03 * rng.standard_normal((3, 4, 8)), 0, 1)
    c = 3
    U0 = np.full((c,) + x.shape, 1.0 / c)
    C0 = (np.arange(c) + 0.5) / c
    # identity storage changes nothing
    a = O.ifcm_fit(x, U0, C0, 0.3, 0.2, max_iter=6, eps=0.0)
    b = O.ifcm_fit(x, U0, C0, 0.3, 0.2, max_iter=6, eps=0.0, store=lambda u: u)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1]) and a[2] == b[2]
    # bf16 storage: the returned U is representable, close to the FP64 run,
    # and one iteration's centres equal those of the unrounded memberships
    Ub, Cb, Jb, _ = O.ifcm_fit(x, U0, C0, 0.3, 0.2, max_iter=6, eps=0.0, store=round_bf16)
    assert np.array_equal(round_bf16(Ub), Ub)
    assert np.max(np.abs(Ub - a[0])) < 1e-2
    U1, C1, J1, _ = O.ifcm_iteration(x, U0, C0, 0.3, 0.2)
    U1b, C1b, J1b, d1b = O.ifcm_iteration(x, U0, C0, 0.3, 0.2, store=round_bf16)
    assert np.array_equal(C1, C1b) and J1 == J1b
    assert np.array_equal(U1b, round_bf16(U1))
    assert d1b == np.max(np.abs(round_bf16(U1) - U0))
