"""Storage-precision model for the memberships (TEST INFRASTRUCTURE ONLY).

The paper fixes no number format.  The GPU library can store the memberships
between iterations as bfloat16 while computing in FP32.  To model that storage
in the FP64 oracle, ``round_bf16`` maps every FP64 value to the nearest
bfloat16 value (ties to even).  bfloat16 is the upper half of IEEE-754 binary32:
1 sign bit, the 8 exponent bits of binary32 and 7 stored fraction bits.  So a
normal value carries 8 significant bits and its spacing in [2^e, 2^(e+1)) is
2^(e-7).  The rounding is written from that definition: split x = f * 2^e with
f in [0.5, 1) (``frexp``), round f * 2^8 to the nearest integer with ties to
even (``rint``), and scale back.  This is exact in FP64.  Values below the
smallest normal binary32 magnitude (2^-126) are rounded on the subnormal grid
of spacing 2^-133.  Memberships never come near it (u >= ~1e-13 with the d^2
floor), but the rule is complete.
"""
import numpy as np

_MIN_NORMAL_EXP = -125          # frexp exponent of 2^-126 (f = 0.5)


def round_bf16(a):
    """Nearest bfloat16 value of each element of ``a`` (FP64 in, FP64 out)."""
    a = np.asarray(a, dtype=np.float64)
    f, e = np.frexp(a)
    e = np.maximum(e, _MIN_NORMAL_EXP)            # subnormal range: fixed grid
    scale = 2.0 ** (8 - e)
    return np.rint(a * scale) / scale
