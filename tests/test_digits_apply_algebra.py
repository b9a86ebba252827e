"""The digit form of F and the tensor-core apply (csrc/sc_apply_digits.cu),
replayed lane by lane on the CPU (tests/digits_emulator.py), against the
plain FP64 products T l_J and T^T l_I of one tile.

Bound: per row and tile, 2^-48 * 32 * max|T| * max|l| -- holding T and l in
55 bits against their largest entries (2^-55 each, rounded), the dropped
digit classes j >= 8 (below 2^-56) and the truncation of the last two classes
to units of 2^-16 of V (2^-72) together stay well inside it; an FP64 GEMV
of the same tile rounds at about 32 * 2^-53 of the same scale.
"""
import numpy as np
import pytest

import digits_emulator as de


def _check(T, lJ, lI, offdiag=True):
    words, eT = de.prepare_tile(T)
    lamJ = de.prepare_lambda(lJ)
    lamI = de.prepare_lambda(lI)
    rows, cols = de.apply_tile(words, eT, lamJ, lamI, offdiag)
    bound_r = 2.0 ** -48 * 32 * np.abs(T).max() * np.abs(lJ).max()
    bound_c = 2.0 ** -48 * 32 * np.abs(T).max() * np.abs(lI).max()
    er = np.abs(rows - T @ lJ).max()
    assert er <= bound_r, (er, bound_r)
    if offdiag:
        ec = np.abs(cols - T.T @ lI).max()
        assert ec <= bound_c, (ec, bound_c)
    else:
        assert not cols.any()
    return er / max(bound_r, 1e-300)


@pytest.mark.parametrize("seed", [0, 1])
def test_random_tile(seed):
    rng = np.random.default_rng(seed)
    T = rng.standard_normal((32, 32))
    r = _check(T, rng.standard_normal(32), rng.standard_normal(32))
    assert r < 0.05          # far inside the bound: an FP64 product's rounding


def test_dynamic_range_signs_and_zeros():
    """Entries spanning 2^-40 .. 2^3 with both signs, exact zeros, a zero
    lambda block, and the largest entry at the top of its binade (the digit
    expansion's range limit)."""
    rng = np.random.default_rng(3)
    T = rng.standard_normal((32, 32)) * 2.0 ** rng.integers(-40, 3, (32, 32))
    T[5, :] = 0.0
    T[:, 7] = 0.0
    T[0, 0] = -np.nextafter(8.0, 0.0)
    l = rng.standard_normal(32) * 2.0 ** rng.integers(-20, 1, 32)
    l[3] = 0.0
    _check(T, l, -l[::-1].copy())
    rows, cols = de.apply_tile(*de.prepare_tile(T), de.prepare_lambda(np.zeros(32)),
                               de.prepare_lambda(np.zeros(32)), True)
    assert not rows.any() and not cols.any()


def test_diagonal_tile_rows_only():
    rng = np.random.default_rng(4)
    A = rng.standard_normal((32, 32))
    T = A + A.T
    l = rng.standard_normal(32)
    _check(T, l, l, offdiag=False)


def test_a_planted_layout_mistake_is_caught():
    """Swapping the two permutes of the column direction (entries of the
    wrong column) must break the column product."""
    rng = np.random.default_rng(5)
    T = rng.standard_normal((32, 32))
    l = rng.standard_normal(32)
    words, eT = de.prepare_tile(T)
    orig = de.prmt
    try:
        de.prmt = lambda a, b, s: orig(a, b, {0x4140: 0x4342, 0x4342: 0x4140}.get(s, s))
        _, cols = de.apply_tile(words, eT, de.prepare_lambda(l), de.prepare_lambda(l), True)
    finally:
        de.prmt = orig
    assert np.abs(cols - T.T @ l).max() > 1e-3
