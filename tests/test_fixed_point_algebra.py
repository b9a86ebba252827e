"""The arithmetic sc_apply_fixed (include/sc.h) states, checked in exact
rational arithmetic on random tiles: per-tile 53-bit fixed point against the
largest exponent, two 27-bit limbs, exact limb products summed in 64-bit
integers, one FP64 rounding per row.  Its normwise error must stay below
2^-51 * 32 max|T| max|l| per row (the bound the header gives), across a wide
range of magnitudes, with zeros and negative entries.  This checks the
method's claim on the CPU; the kernel itself is checked against the oracle
on the GPU (tests/test_gpu_apply_fixed.py)."""
import struct
from fractions import Fraction

import numpy as np


def _bits(x):
    return struct.unpack("<Q", struct.pack("<d", float(x)))[0]


def _exp(x):
    return (_bits(x) >> 52) & 0x7FF


def _fixed(x, exmax):
    b = _bits(x)
    ex = (b >> 52) & 0x7FF
    if ex == 0:
        return 0
    mant = (b & ((1 << 52) - 1)) | (1 << 52)
    s = exmax - ex + 1
    m = 0 if s > 63 else (mant + (1 << (s - 1))) >> s
    return -m if b >> 63 else m


def _limbs(m):
    return m >> 27, m & ((1 << 27) - 1)      # floor shift: m = hi 2^27 + lo, 0 <= lo < 2^27


def _tile_rows(T, lam):
    exm, exl = max(_exp(v) for v in T.ravel()), max(_exp(v) for v in lam)
    if exm == 0 or exl == 0:
        return np.zeros(T.shape[0])
    L = [_limbs(_fixed(v, exl)) for v in lam]
    out = np.zeros(T.shape[0])
    for i in range(T.shape[0]):
        d0 = d1 = d2 = 0
        for j in range(T.shape[1]):
            mh, ml = _limbs(_fixed(T[i, j], exm))
            lh, ll = L[j]
            d0 += ml * ll
            d1 += mh * ll + ml * lh
            d2 += mh * lh
        for d in (d0, d1, d2):
            assert abs(d) < 2 ** 63                     # fits the kernel's int64 accumulators
        # the kernel fuses these two steps into FMAs; separate roundings are within the same bound
        v = float(d2) + float(d1) * 2.0 ** -27 + float(d0) * 2.0 ** -54
        out[i] = np.ldexp(v, exm + exl - 2094)
    return out


def test_fixed_point_tile_product_error_bound():
    rng = np.random.default_rng(0)
    for trial in range(12):
        scale = 10.0 ** rng.uniform(-150, 150)
        T = rng.standard_normal((32, 32)) * np.exp(rng.uniform(-6, 6, (32, 32))) * scale
        T[rng.random((32, 32)) < 0.15] = 0.0
        lam = rng.standard_normal(32) * 10.0 ** rng.uniform(-40, 40)
        lam[rng.integers(32)] = 0.0
        got = _tile_rows(T, lam)
        bound = 2.0 ** -51 * 32 * np.abs(T).max() * np.abs(lam).max()
        for i in range(32):
            exact = sum(Fraction(T[i, j]) * Fraction(lam[j]) for j in range(32))
            assert abs(Fraction(got[i]) - exact) <= Fraction(bound), (trial, i)


def test_fixed_point_zero_block_and_tile():
    T = np.zeros((32, 32))
    lam = np.ones(32)
    assert np.all(_tile_rows(T, lam) == 0.0)
    assert np.all(_tile_rows(np.ones((32, 32)), np.zeros(32)) == 0.0)


def _balanced_digits(X, S):
    """The recoding of the tcgen05 SYRK's Y planes (yslice_kernel, balanced):
    the S top bytes of a 62-bit magnitude, least significant first, a digit
    above 127 becomes digit - 256 and carries one into the next; the top
    digit takes the last carry without wrapping."""
    dig = [0] * S
    carry = 0
    for d in range(S - 1, -1, -1):
        u = ((X >> (55 - 8 * d)) & 0xFF) + carry
        carry = 1 if (d > 0 and u >= 128) else 0
        dig[d] = u - 256 * carry
    return dig


def test_balanced_digits_reconstruct_and_stay_small():
    """Balanced digits of a magnitude below 2^62 lie in [-128, 128] (so every
    digit product is at most 2^14 and a 32-row block sum of up to 7 digit
    pairs stays below 7 * 32 * 2^14 < 2^22, the range where the kernel's
    FP32-to-integer step v + 1.5 * 2^23 is exact) and represent exactly the
    magnitude truncated to its top S bytes."""
    rng = np.random.default_rng(11)
    cases = [0, 1, (1 << 62) - 1, (1 << 61), 0x7F7F7F7F7F7F7F7F >> 1] + \
        [int(x) for x in rng.integers(0, 1 << 62, size=4000, dtype=np.uint64)]
    for S in (3, 4, 5, 6, 7):
        for X in cases:
            X &= (1 << 62) - 1
            dig = _balanced_digits(X, S)
            assert all(-128 <= d <= 128 for d in dig)
            assert sum(d * 256 ** (S - 1 - t) for t, d in enumerate(dig)) == X >> (55 - 8 * (S - 1))
    assert 7 * 32 * 128 * 128 < 2 ** 22
    # v + 1.5 * 2^23 in FP32 puts v in the low bits for |v| < 2^22
    for v in (0, 1, -1, 3670016, -3670016, 2 ** 22 - 1, -(2 ** 22 - 1)):
        bits = struct.unpack("<I", struct.pack("<f", np.float32(v) + np.float32(12582912.0)))[0]
        assert bits - 0x4B400000 == v
