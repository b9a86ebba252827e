"""Writes tests/golden/config1_anchor.txt from the FP64 oracle alone (no
library code): norms and extreme eigenvalues of F for config 1 (one 16x16 Q1
square, corner node fixed, the 64 boundary dofs glued).  The paper prints no
entries of F, so this is a regression anchor of the oracle; an independent
dense computation (numpy inverse of K_reg gathered by B) printed
||F||_F = 174.9015, trace 266.3118, lambda_min 0.5774, lambda_max 173.8,
which the test checks as well.

    python tests/golden/make_config1_anchor.py
"""
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle  # noqa: E402
import synth  # noqa: E402


def anchor():
    F = oracle.dual_operator(synth.make_config(1).subdomains[0], refine=1)
    ev = np.linalg.eigvalsh(0.5 * (F + F.T))
    return {"frobenius": float(np.linalg.norm(F)), "trace": float(np.trace(F)),
            "lambda_min": float(ev[0]), "lambda_max": float(ev[-1]), "m": int(F.shape[0])}


if __name__ == "__main__":
    a = anchor()
    with open(os.path.join(HERE, "config1_anchor.txt"), "w") as f:
        f.write("# config 1 (16x16 Q1 square, corner fixed, 64 boundary multipliers): F from the FP64 oracle\n")
        f.write("# written by tests/golden/make_config1_anchor.py (oracle only)\n")
        for k, v in a.items():
            f.write(f"{k} {v!r}\n")
    print(a)
