"""Writes tiny_pairs.json: exact likelihoods of tiny pairs by path enumeration.

Calls only oracle/ (oracle/brute.py, exact rational arithmetic over the FP64 values of the
Phred conversions).  Run from the repository root:  python tests/golden/make_golden.py
"""
import json
import math
import os
import sys
from fractions import Fraction

import numpy as np

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__)))))
from oracle import brute  # noqa: E402


def P(q):
    return 10.0 ** (-q / 10.0)


def main():
    rng = np.random.default_rng(20241118)
    cases = []
    for k in range(32):
        m = int(rng.integers(1, 5))
        n = int(rng.integers(1, 6))
        alph = list("ACGTN" if k % 4 == 0 else "ACGT")
        read = "".join(rng.choice(alph, size=m))
        hap = "".join(rng.choice(alph, size=n))
        bq = [int(x) for x in rng.integers(2, 41, size=m)]
        iq = [int(x) for x in rng.integers(10, 46, size=m)]
        dq = [int(x) for x in rng.integers(10, 46, size=m)]
        gcp = 10.0 if k % 2 == 0 else float(rng.integers(3, 30))
        L = brute.likelihood(read, hap, [Fraction(P(q)) for q in bq], [Fraction(P(q)) for q in iq],
                             [Fraction(P(q)) for q in dq], Fraction(P(gcp)))
        cases.append({"read": read, "hap": hap, "bq": bq, "iq": iq, "dq": dq, "gcp": gcp,
                      "log10L": math.log10(L)})
    out = os.path.join(os.path.dirname(os.path.abspath(__file__)), "tiny_pairs.json")
    with open(out, "w") as f:
        json.dump({"source": "exact path enumeration of Eq. 1-3 (Sec. II-A), oracle/brute.py",
                   "cases": cases}, f, indent=1)


if __name__ == "__main__":
    main()
