"""Exact brute-force Pair-HMM likelihood by enumerating every alignment path.

TEST INFRASTRUCTURE ONLY.  Independent of the DP loops of ``phmm_oracle.c``: it walks the
state graph implied by Sec. II-A (Eq. 1-3 and the initialisation line) path by path and sums
path weights in exact rational arithmetic (``fractions.Fraction``).  Only tiny pairs
(m <= 4, n <= 5) are feasible.

State graph (cells (i, j), states M / I / D):
  * a path starts in D at (0, j0) for any 0 <= j0 <= n with weight 1/n (D(0,j) = 1/n);
  * M at (i, j)  -> M at (i+1, j+1): lambda(i+1, j+1) * alpha_{i+1}
  * I or D       -> M at (i+1, j+1): lambda(i+1, j+1) * beta_{i+1}
  * M at (i, j)  -> I at (i+1, j):   delta_{i+1};      I -> I at (i+1, j): eps_{i+1}
  * M at (i, j)  -> D at (i, j+1):   zeta_i (i >= 1);  D -> D at (i, j+1): eps_i (i >= 1)
  (eps_i = eps and beta_i = beta = 1 - eps for one gap-continuation value; a per-base track
  gives each read position its own, every transition into row i taking row i's values)
  * row-0 D states only move to M (row 0 is initialisation, not a recurrence);
  * a path ends in M or I at row m.
"""
from __future__ import annotations

from fractions import Fraction


def _match(r: str, h: str) -> bool:
    r, h = r.upper(), h.upper()
    return r == h or r == "N" or h == "N"


def likelihood(read: str, hap: str, Q, delta, zeta, eps, alpha=None) -> Fraction:
    """Exact L = sum over paths of the product of transition and emission weights.

    Q, delta, zeta: per read position (length m) probabilities (Fraction or anything
    Fraction() accepts exactly, e.g. floats); eps: gap continuation probability, one value or
    one per read position.
    alpha_i = 1 - (delta_i + zeta_i) unless ``alpha`` gives the M -> M probability of every
    read position explicitly (e.g. the alternative 1 - 10^(-(iq_i + dq_i)/10)); beta = 1 - eps.
    """
    m, n = len(read), len(hap)
    Q = [Fraction(x) for x in Q]
    de = [Fraction(x) for x in delta]
    ze = [Fraction(x) for x in zeta]
    if isinstance(eps, (list, tuple)):
        epv = [Fraction(x) for x in eps]
        assert len(epv) == m
    else:
        epv = [Fraction(eps)] * m
    if alpha is None:
        al = [1 - (de[i] + ze[i]) for i in range(m)]
    else:
        al = [Fraction(x) for x in alpha]
        assert len(al) == m
    bev = [1 - x for x in epv]

    def lam(i, j):  # 1-based
        q = Q[i - 1]
        return (1 - q) if _match(read[i - 1], hap[j - 1]) else q / 3

    total = Fraction(0)
    # explicit stack of (state, i, j, weight)
    stack = [("D0", 0, j0, Fraction(1, n)) for j0 in range(0, n + 1)]
    while stack:
        s, i, j, w = stack.pop()
        if i == m and s in ("M", "I"):
            total += w
            # a path may not continue past row m into M/I (row m+1 does not exist), but an
            # M at row m may still step right into D at row m; D never returns to row m's sum.
        # moves to M at (i+1, j+1)
        if i + 1 <= m and j + 1 <= n:
            if s == "M":
                stack.append(("M", i + 1, j + 1, w * lam(i + 1, j + 1) * al[i]))
            else:  # I, D, or row-0 D
                stack.append(("M", i + 1, j + 1, w * lam(i + 1, j + 1) * bev[i]))
        if s == "D0":
            continue
        # moves to I at (i+1, j)
        if i + 1 <= m:
            if s == "M":
                stack.append(("I", i + 1, j, w * de[i]))
            elif s == "I":
                stack.append(("I", i + 1, j, w * epv[i]))
        # moves to D at (i, j+1)
        if i >= 1 and j + 1 <= n:
            if s == "M":
                stack.append(("D", i, j + 1, w * ze[i - 1]))
            elif s == "D":
                stack.append(("D", i, j + 1, w * epv[i - 1]))
    return total
