"""CPU replay of the tensor-core apply from the digit form of F
(csrc/sc_apply_digits.cu), lane by lane: the prepared words of a tile, the
lambda block's B fragments and class constants, the byte permutes that form
the A fragments of either direction, the m16n8k16 MMA in its register
layout (evaluated exactly: every product and partial sum is an integer
multiple of 2^-24 well inside FP32's exact range), the exact integer class
combination with its lane shuffles, and the final scaling.

Test infrastructure: it restates the kernel's index arithmetic so that the
layout can be checked against a plain FP64 product on the CPU; it shares no
code with the library.
"""
from __future__ import annotations

import numpy as np

K = 7                      # digits of F and lambda


def widx(R: int, C: int) -> int:
    return 16 * R + (C ^ (((R & 2) << 2) | (R & 4)))


def biased_exp(x: float) -> int:
    return int((np.float64(x).view(np.uint64) >> np.uint64(52)) & np.uint64(0x7FF))


def fixed55(x: float, emax: int) -> int:
    b = int(np.float64(x).view(np.uint64))
    e = (b >> 52) & 0x7FF
    mant = b & ((1 << 52) - 1)
    if e:
        mant |= 1 << 52
    else:
        e = 1
    sh = e + 1 - emax
    if sh >= 0:
        m = mant << sh
    elif sh > -60:
        m = (mant + (1 << (-sh - 1))) >> (-sh)
    else:
        m = 0
    return -m if b >> 63 else m


def digits7(M: int):
    d = [0] * K
    for k in range(K - 1, -1, -1):
        v = ((M + 128) & 255) - 128
        d[k] = v
        M = (M - v) >> 8
    assert M == 0
    return d


def prepare_tile(T: np.ndarray):
    """words[k][256] (uint32) and the biased e_max of a 32x32 tile (T[r, c])."""
    emax = max(biased_exp(v) for v in T.ravel())
    D = [[digits7(fixed55(T[r, c], emax)) for c in range(32)] for r in range(32)]
    words = np.zeros((K, 256), np.uint64)
    for k in range(K):
        for R in range(16):
            for C in range(16):
                ob = [D[2 * R][2 * C][k] + 128, D[2 * R + 1][2 * C][k] + 128,
                      D[2 * R][2 * C + 1][k] + 128, D[2 * R + 1][2 * C + 1][k] + 128]
                words[k, widx(R, C)] = ob[0] | (ob[1] << 8) | (ob[2] << 16) | (ob[3] << 24)
    return words.astype(np.uint32), emax


def _h(v: int) -> int:
    return int(np.float16(v).view(np.uint16))


def prepare_lambda(l: np.ndarray):
    """The lambda block's digit table wt[14][32] (FP16 bit patterns; row r =
    digit r - 6, zero outside digits 0..6), class constants cj[8] (FP32) and
    the biased e_max of a 32-entry lambda block."""
    emax = max(biased_exp(v) for v in l)
    w = [digits7(fixed55(v, emax)) for v in l]
    wt = np.zeros((14, 32), np.uint32)
    colsum = np.zeros(K, np.int64)
    for c in range(32):
        C = c >> 1
        pos = 2 * (4 * (C & 3) + (C >> 2)) + (c & 1)     # pair C at word 4 (C mod 4) + C / 4 of its row
        for e in range(K):
            wt[e + 6, pos] = _h(w[c][e])
            colsum[e] += w[c][e]
    cj = np.array([12582912.0 - 128.0 * sum(colsum[e] for e in range(K) if 0 <= j - e < K) for j in range(8)],
                  np.float32)
    return wt, cj, emax


def b_fragments(wt):
    """b[k][lane][4]: the B operands the kernel reads from the table, the
    16 bytes at word 4t of row g - k + 6: pairs C = t, 4 + t, 8 + t, 12 + t."""
    b = np.zeros((K, 32, 4), np.uint32)
    for k in range(K):
        for lane in range(32):
            g, t = lane >> 2, lane & 3
            for x in range(4):
                p = 2 * (4 * t + x)
                b[k, lane, x] = int(wt[g - k + 6, p]) | (int(wt[g - k + 6, p + 1]) << 16)
    return b


def prmt(a: int, b: int, sel: int) -> int:
    src = [(a >> (8 * i)) & 0xFF for i in range(4)] + [(b >> (8 * i)) & 0xFF for i in range(4)]
    return sum(src[(sel >> (4 * i)) & 0x7] << (8 * i) for i in range(4))


def _f16pair(r: int):
    return (float(np.uint16(r & 0xFFFF).view(np.float16)), float(np.uint16(r >> 16).view(np.float16)))


def mma(c, a, b):
    """m16n8k16 with the standard register layout: c[lane][4] += A B from
    a[lane][4], b[lane][2] (FP16 pairs), evaluated exactly."""
    A = np.zeros((16, 16))
    B = np.zeros((16, 8))
    for lane in range(32):
        g, t = lane >> 2, lane & 3
        for reg, (row, col) in enumerate([(g, 2 * t), (g + 8, 2 * t), (g, 2 * t + 8), (g + 8, 2 * t + 8)]):
            A[row, col], A[row, col + 1] = _f16pair(a[lane][reg])
        B[2 * t, g], B[2 * t + 1, g] = _f16pair(b[lane][0])
        B[2 * t + 8, g], B[2 * t + 9, g] = _f16pair(b[lane][1])
    D = A @ B              # exact: integer multiples of 2^-24 far below 2^53
    for lane in range(32):
        g, t = lane >> 2, lane & 3
        c[lane][0] += D[g, 2 * t]
        c[lane][1] += D[g, 2 * t + 1]
        c[lane][2] += D[g + 8, 2 * t]
        c[lane][3] += D[g + 8, 2 * t + 1]


def acc_int(d: float, c: float) -> int:
    v = np.float32(np.float64(d) * 16777216.0 + np.float64(c))      # one rounding, as the FMA
    assert float(v) == d * 16777216.0 + float(c), "accumulator not exact"
    return int(np.float32(v).view(np.int32)) - 0x4B400000


def class_sum(d, c0, c1):
    """d[lane][mb][4] -> per lane the integer V of output rho = t (lane = 4 g + t)."""
    v = [[0] * 4 for _ in range(32)]
    for lane in range(32):
        t = lane & 3
        for mb in range(2):
            for h in range(2):
                p = acc_int(d[lane][mb][2 * h], c0[lane]) * 256 + acc_int(d[lane][mb][2 * h + 1], c1[lane])
                v[lane][2 * mb + h] = p << (16 * (2 - t)) if t < 3 else p >> 16
    out = [0] * 32
    for lane in range(32):       # the two shuffle rounds: the sum over the four lanes of this g for rho = t
        g, t = lane >> 2, lane & 3
        out[lane] = sum(v[4 * g + u][t] for u in range(4))
    return out


def apply_tile(words, eT, lamJ, lamI, offdiag: bool):
    """(row contributions T l_J, column contributions T^T l_I) of one tile, in
    tile row / column order, as the kernel forms them."""
    wJ, cJ, eJ = lamJ
    wI, cI, eI = lamI
    bJ, bI = b_fragments(wJ), b_fragments(wI)
    dr = [[[0.0] * 4 for _ in range(2)] for _ in range(32)]
    dc = [[[0.0] * 4 for _ in range(2)] for _ in range(32)]
    for k in range(K):
        pk = words[k]
        for mb in range(2):
            for kb in range(2):
                a, b = [], []
                for lane in range(32):
                    g, t = lane >> 2, lane & 3
                    R = 8 * mb + g
                    w0, w1 = int(pk[widx(R, 8 * kb + t)]), int(pk[widx(R, 8 * kb + 4 + t)])
                    a.append([prmt(w0, 0, 0x4240), prmt(w0, 0, 0x4341), prmt(w1, 0, 0x4240), prmt(w1, 0, 0x4341)])
                    bb = bJ[k, lane]
                    b.append([int(bb[2 * kb]), int(bb[2 * kb + 1])])
                c = [dr[lane][mb] for lane in range(32)]
                mma(c, a, b)
        if offdiag:
            for mb in range(2):
                for kb in range(2):
                    a, b = [], []
                    for lane in range(32):
                        g, t = lane >> 2, lane & 3
                        C = 8 * mb + g
                        w0, w1 = int(pk[widx(8 * kb + t, C)]), int(pk[widx(8 * kb + 4 + t, C)])
                        a.append([prmt(w0, 0, 0x4140), prmt(w0, 0, 0x4342), prmt(w1, 0, 0x4140),
                                  prmt(w1, 0, 0x4342)])
                        bb = bI[k, lane]
                        b.append([int(bb[2 * kb]), int(bb[2 * kb + 1])])
                    c = [dc[lane][mb] for lane in range(32)]
                    mma(c, a, b)
    lanes = range(32)
    myrow = [16 * ((l & 3) >> 1) + 2 * (l >> 2) + (l & 1) for l in lanes]
    Vr = class_sum(dr, [cJ[2 * (l & 3)] for l in lanes], [cJ[2 * (l & 3) + 1] for l in lanes])
    rows = np.zeros(32)
    for l in lanes:
        rows[myrow[l]] = Vr[l] * 2.0 ** (eT + eJ - 2096)
    cols = np.zeros(32)
    if offdiag:
        Vc = class_sum(dc, [cI[2 * (l & 3)] for l in lanes], [cI[2 * (l & 3) + 1] for l in lanes])
        for l in lanes:
            cols[myrow[l]] = Vc[l] * 2.0 ** (eT + eI - 2096)
    return rows, cols
