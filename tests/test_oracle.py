"""Pins of the FP64 oracle to facts the paper and the mathematics fix (no GPU).

Each test checks the oracle against something other than itself: a hand-derived closed form,
exact path enumeration (oracle/brute.py), an arbitrary-range decimal DP, an invariant, or
central finite differences for the adjoint.
"""
import math
from decimal import Decimal, getcontext
from fractions import Fraction

import numpy as np
import pytest

import oracle
from oracle import brute
from paper_2411_11547_gb300 import synth


def P(q):
    return 10.0 ** (-q / 10.0)


def rand_seq(rng, n, alphabet="ACGT"):
    return "".join(rng.choice(list(alphabet), size=n))


# ---------------------------------------------------------------- closed forms -------------

def test_1x1_match_and_mismatch():
    # m = n = 1: L = lambda(1,1) * beta  (M(1,1) = lambda*beta*D(0,0), D(0,0) = 1/n = 1)
    y = oracle.forward_pair("A", [30], [45], [45], "A", gcp=10)
    assert y == pytest.approx(math.log10(0.999 * 0.9), abs=1e-14)
    assert y == pytest.approx(-0.046192002, abs=1e-9)
    y = oracle.forward_pair("A", [30], [45], [45], "C", gcp=10)
    assert y == pytest.approx(math.log10(0.001 / 3 * 0.9), abs=1e-14)


@pytest.mark.parametrize("seed", range(5))
def test_single_row_closed_form(seed):
    # m = 1: I(1,j) = 0, so L = (beta/n) * sum_j lambda(1,j)
    rng = np.random.default_rng(seed)
    n = int(rng.integers(1, 40))
    hap = rand_seq(rng, n, "ACGTN")
    r = rand_seq(rng, 1, "ACGTN")
    q = float(rng.integers(2, 41))
    gcp = float(rng.uniform(3, 30))
    beta = 1 - P(gcp)
    lam = [(1 - P(q)) if (r == h or r == "N" or h == "N") else P(q) / 3 for h in hap]
    want = math.log10(beta / n * sum(lam))
    assert oracle.forward_pair(r, [q], [30], [35], hap, gcp=gcp) == pytest.approx(want, abs=1e-13)


@pytest.mark.parametrize("seed", range(6))
def test_2x3_closed_form(seed):
    # Hand-derived from Eq. 1-3 with D(0,j) = 1/3 for j = 0..3:
    # L = (b/3)[l11 l22 a2 + l23 (l12 a2 + b z1 l11) + d2 (l11 + l12 + l13)]
    rng = np.random.default_rng(100 + seed)
    read, hap = rand_seq(rng, 2), rand_seq(rng, 3)
    bq = rng.integers(5, 41, size=2).astype(float)
    iq = rng.integers(5, 40, size=2).astype(float)
    dq = rng.integers(5, 40, size=2).astype(float)
    gcp = float(rng.uniform(5, 20))
    Q, d, z = P(bq), P(iq), P(dq)
    a = 1 - (d + z)
    b = 1 - P(gcp)

    def lam(i, j):
        return (1 - Q[i - 1]) if read[i - 1] == hap[j - 1] else Q[i - 1] / 3

    L = (b / 3) * (lam(1, 1) * lam(2, 2) * a[1]
                   + lam(2, 3) * (lam(1, 2) * a[1] + b * z[0] * lam(1, 1))
                   + d[1] * (lam(1, 1) + lam(1, 2) + lam(1, 3)))
    got = oracle.forward_pair(read, bq, iq, dq, hap, gcp=gcp)
    assert got == pytest.approx(math.log10(L), abs=1e-13)


@pytest.mark.parametrize("m,n", [(30, 30), (12, 40), (1, 9), (64, 150)])
def test_gapless_closed_form(m, n):
    # delta = zeta = 0 (gap quals +inf): alpha = 1, only diagonal paths remain:
    # L = (beta/n) * sum_{o=0}^{n-m} prod_i lambda(i, o+i)
    rng = np.random.default_rng(m * 1000 + n)
    hap = rand_seq(rng, n)
    o0 = int(rng.integers(0, n - m + 1))
    read = hap[o0:o0 + m]
    bq = rng.integers(10, 41, size=m).astype(float)
    inf = np.full(m, np.inf)
    Q = P(bq)
    beta = 1 - P(10.0)
    tot = 0.0
    for o in range(n - m + 1):
        pr = 1.0
        for i in range(m):
            pr *= (1 - Q[i]) if read[i] == hap[o + i] else Q[i] / 3
        tot += pr
    want = math.log10(beta / n * tot)
    got = oracle.forward_pair(read, bq, inf, inf, hap, gcp=10.0)
    assert got == pytest.approx(want, abs=1e-12)
    if m == n:
        assert got == pytest.approx(math.log10(beta) - math.log10(n) + np.sum(np.log10(1 - Q)),
                                    abs=1e-12)
    # with finite gap quals the diagonal paths keep weight (beta/n) alpha^(m-1) prod lambda and
    # gapped paths only add mass: a lower bound, strict once m > 1 (m = 1 has no gapped path)
    fin = np.full(m, 40.0)
    a = 1 - 2 * P(40.0)
    lower = math.log10(beta / n * tot) + (m - 1) * math.log10(a)
    got_fin = oracle.forward_pair(read, bq, fin, fin, hap, gcp=10.0)
    if m > 1:
        assert got_fin > lower
    else:
        assert got_fin == pytest.approx(lower, abs=1e-14)


# ------------------------------------------------------------ brute-force enumeration -------

@pytest.mark.parametrize("seed", range(40))
def test_brute_force_tiny(seed):
    rng = np.random.default_rng(7000 + seed)
    m = int(rng.integers(1, 5))
    n = int(rng.integers(1, 6))
    alph = "ACGTN" if seed % 3 == 0 else "ACGT"
    read, hap = rand_seq(rng, m, alph), rand_seq(rng, n, alph)
    if seed % 4 == 1:
        read = read.lower()
    bq = rng.integers(0, 41, size=m).astype(float)
    iq = rng.integers(3, 46, size=m).astype(float)
    dq = rng.integers(3, 46, size=m).astype(float)
    gcp = float(rng.integers(1, 40))
    exact = brute.likelihood(read, hap, [Fraction(P(q)) for q in bq],
                             [Fraction(P(q)) for q in iq], [Fraction(P(q)) for q in dq],
                             Fraction(P(gcp)))
    got = oracle.forward_pair(read, bq, iq, dq, hap, gcp=gcp)
    if exact == 0:
        assert got == -math.inf
    else:
        assert got == pytest.approx(math.log10(exact), abs=1e-12)


def test_brute_force_structure_terms():
    # a 2x2 case where only specific transitions can produce mass: read "AC", hap "AC" with
    # bq = 0 (Q = 1: matches emit 0, mismatches 1/3).  Paths through the matching diagonal
    # vanish; everything left uses mismatch emissions, insertions and deletions.
    q = [0.0, 0.0]
    g = [20.0, 25.0]
    exact = brute.likelihood("AC", "AC", [1, 1], [P(x) for x in g], [P(x) for x in g],
                             Fraction(P(10.0)))
    got = oracle.forward_pair("AC", q, g, g, "AC", gcp=10.0)
    assert got == pytest.approx(math.log10(exact), abs=1e-12)


# ------------------------------------------------ arbitrary-range check of the rescaling -----

def _decimal_forward(read, hap, bq, iq, dq, gcp):
    """Eq. 1-3 in 60-digit Decimal (unbounded exponent): no rescaling needed at all."""
    getcontext().prec = 60
    D10 = Decimal(10)
    m, n = len(read), len(hap)

    def p(q):
        return D10 ** (Decimal(-q) / 10)

    Q = [p(q) for q in bq]
    de = [p(q) for q in iq]
    ze = [p(q) for q in dq]
    ep = p(gcp)
    be = 1 - ep
    pm = [Decimal(0)] * (n + 1)
    pi = [Decimal(0)] * (n + 1)
    pd = [Decimal(1) / n] * (n + 1)
    for i in range(1, m + 1):
        cm = [Decimal(0)] * (n + 1)
        ci = [Decimal(0)] * (n + 1)
        cd = [Decimal(0)] * (n + 1)
        al = 1 - (de[i - 1] + ze[i - 1])
        for j in range(1, n + 1):
            r, h = read[i - 1], hap[j - 1]
            lam = (1 - Q[i - 1]) if (r == h or r == "N" or h == "N") else Q[i - 1] / 3
            cm[j] = lam * (al * pm[j - 1] + be * (pi[j - 1] + pd[j - 1]))
            ci[j] = de[i - 1] * pm[j] + ep * pi[j]
            cd[j] = ze[i - 1] * cm[j - 1] + ep * cd[j - 1]
        pm, pi, pd = cm, ci, cd
    L = sum(pm[1:]) + sum(pi[1:])
    return float(L.log10())


@pytest.mark.parametrize("case", ["unrelated_high_q", "beyond_double"])
def test_renormalisation_against_decimal(case):
    rng = np.random.default_rng(11)
    if case == "unrelated_high_q":
        m, n, q, gq, gcp = 60, 70, 40, (30, 46), 10.0
    else:
        # high base and gap quals, rare gap extension: L far below the double range
        m, n, q, gq, gcp = 150, 160, 60, (60, 61), 40.0
    read, hap = rand_seq(rng, m), rand_seq(rng, n)
    bq = np.full(m, float(q))
    iq = rng.integers(gq[0], gq[1], size=m).astype(float)
    dq = rng.integers(gq[0], gq[1], size=m).astype(float)
    want = _decimal_forward(read, hap, bq, iq, dq, gcp)
    got = oracle.forward_pair(read, bq, iq, dq, hap, gcp=gcp)
    if case == "beyond_double":
        assert want < -330
    assert got == pytest.approx(want, abs=1e-10)


# ------------------------------------------------------------------------- invariants -------

@pytest.mark.parametrize("seed", range(4))
def test_N_symmetry(seed):
    # an all-N haplotype and an all-N read both make every emission 1 - Q_i
    rng = np.random.default_rng(300 + seed)
    m, n = int(rng.integers(3, 30)), int(rng.integers(3, 40))
    bq = rng.integers(10, 41, size=m)
    iq = rng.integers(30, 46, size=m)
    dq = rng.integers(30, 46, size=m)
    a = oracle.forward_pair(rand_seq(rng, m), bq, iq, dq, "N" * n)
    b = oracle.forward_pair("N" * m, bq, iq, dq, rand_seq(rng, n))
    c = oracle.forward_pair("N" * m, bq, iq, dq, "N" * n)
    assert a == b == c
    # an N at read position i equals that row matching every column: compare with a read that
    # carries N against a haplotype whose column j holds N instead
    read = rand_seq(rng, m)
    hap = rand_seq(rng, n)
    rN = read[:1] + "N" + read[2:] if m > 1 else "N"
    assert np.isfinite(oracle.forward_pair(rN, bq, iq, dq, hap))


@pytest.mark.parametrize("seed", range(8))
def test_mismatch_monotonicity(seed):
    # H over {A,C,G}; substituting a read base by T (absent from H) turns every emission of
    # that row into the mismatch value Q/3 <= 1-Q (Q < 3/4): L cannot increase.
    rng = np.random.default_rng(400 + seed)
    m, n = int(rng.integers(2, 60)), int(rng.integers(2, 80))
    hap = rand_seq(rng, n, "ACG")
    read = list(rand_seq(rng, m, "ACG"))
    bq = rng.integers(2, 41, size=m)
    iq = rng.integers(20, 46, size=m)
    dq = rng.integers(20, 46, size=m)
    prev = oracle.forward_pair("".join(read), bq, iq, dq, hap)
    for i in rng.permutation(m)[: min(m, 6)]:
        read[i] = "T"
        cur = oracle.forward_pair("".join(read), bq, iq, dq, hap)
        assert cur <= prev + 1e-13
        prev = cur


@pytest.mark.parametrize("seed", range(6))
def test_alpha_mode_1_2x3_closed_form(seed):
    # The hand-derived 2x3 closed form of test_2x3_closed_form with the alternative
    # M -> M probability alpha_i = 1 - 10^(-(iq_i + dq_i)/10) (alpha_mode 1):
    # L = (b/3)[l11 l22 a2 + l23 (l12 a2 + b z1 l11) + d2 (l11 + l12 + l13)], a2 replaced.
    rng = np.random.default_rng(400 + seed)
    read, hap = rand_seq(rng, 2), rand_seq(rng, 3)
    bq = rng.integers(5, 41, size=2).astype(float)
    iq = rng.integers(3, 20, size=2).astype(float)   # low gap quals: the two alphas differ
    dq = rng.integers(3, 20, size=2).astype(float)   # by ~(delta + zeta) / ln 10 per row
    gcp = float(rng.uniform(5, 20))
    Q, d, z = P(bq), P(iq), P(dq)
    a1 = 1 - 10.0 ** (-(iq + dq) / 10.0)
    b = 1 - P(gcp)

    def lam(i, j):
        return (1 - Q[i - 1]) if read[i - 1] == hap[j - 1] else Q[i - 1] / 3

    L1 = (b / 3) * (lam(1, 1) * lam(2, 2) * a1[1]
                    + lam(2, 3) * (lam(1, 2) * a1[1] + b * z[0] * lam(1, 1))
                    + d[1] * (lam(1, 1) + lam(1, 2) + lam(1, 3)))
    got = oracle.forward_pair(read, bq, iq, dq, hap, gcp=gcp, alpha_mode=1)
    assert got == pytest.approx(math.log10(L1), abs=1e-13)
    # the default reading gives a different value on the same pair (the pin separates them)
    got0 = oracle.forward_pair(read, bq, iq, dq, hap, gcp=gcp, alpha_mode=0)
    assert abs(got0 - got) > 1e-9


@pytest.mark.parametrize("seed", range(24))
def test_alpha_mode_1_brute_force(seed):
    # alpha_mode 1 against exact path enumeration with alpha_i = 1 - 10^(-(iq_i+dq_i)/10)
    # passed to the enumerator explicitly (everything else as in test_brute_force_tiny)
    rng = np.random.default_rng(9100 + seed)
    m = int(rng.integers(1, 5))
    n = int(rng.integers(1, 6))
    alph = "ACGTN" if seed % 3 == 0 else "ACGT"
    read, hap = rand_seq(rng, m, alph), rand_seq(rng, n, alph)
    bq = rng.integers(0, 41, size=m).astype(float)
    iq = rng.integers(2, 30, size=m).astype(float)
    dq = rng.integers(2, 30, size=m).astype(float)
    gcp = float(rng.integers(1, 40))
    alpha = [Fraction(1.0 - 10.0 ** (-(i + d) / 10.0)) for i, d in zip(iq, dq)]
    exact = brute.likelihood(read, hap, [Fraction(P(q)) for q in bq],
                             [Fraction(P(q)) for q in iq], [Fraction(P(q)) for q in dq],
                             Fraction(P(gcp)), alpha=alpha)
    got = oracle.forward_pair(read, bq, iq, dq, hap, gcp=gcp, alpha_mode=1)
    if exact == 0:
        assert got == -math.inf
    else:
        assert got == pytest.approx(math.log10(exact), abs=1e-12)


# ------------------------------------------------- per-base gap-continuation track -------

@pytest.mark.parametrize("seed", range(24))
def test_per_base_gcp_brute_force(seed):
    # a per-read-position gap continuation (eps_i, beta_i of the row being entered) against
    # exact path enumeration with one eps per read position
    rng = np.random.default_rng(9500 + seed)
    m = int(rng.integers(1, 5))
    n = int(rng.integers(1, 6))
    alph = "ACGTN" if seed % 3 == 0 else "ACGT"
    read, hap = rand_seq(rng, m, alph), rand_seq(rng, n, alph)
    bq = rng.integers(0, 41, size=m).astype(float)
    iq = rng.integers(3, 30, size=m).astype(float)
    dq = rng.integers(3, 30, size=m).astype(float)
    gq = rng.integers(1, 40, size=m).astype(float)
    exact = brute.likelihood(read, hap, [Fraction(P(q)) for q in bq],
                             [Fraction(P(q)) for q in iq], [Fraction(P(q)) for q in dq],
                             [Fraction(P(q)) for q in gq])
    got = oracle.forward_pair(read, bq, iq, dq, hap, gcp=10.0, gcp_q=gq)
    if exact == 0:
        assert got == -math.inf
    else:
        assert got == pytest.approx(math.log10(exact), abs=1e-12)


@pytest.mark.parametrize("seed", range(4))
def test_per_base_gcp_2x3_closed_form(seed):
    # The 2x3 closed form with row-indexed beta: the start enters row 1 through beta_1, the
    # deletion path M(1,1) -> D(1,2) -> M(2,3) returns to M through beta_2:
    # L = (b1/3)[l11 l22 a2 + l23 (l12 a2 + b2 z1 l11) + d2 (l11 + l12 + l13)]
    rng = np.random.default_rng(600 + seed)
    read, hap = rand_seq(rng, 2), rand_seq(rng, 3)
    bq = rng.integers(5, 41, size=2).astype(float)
    iq = rng.integers(5, 40, size=2).astype(float)
    dq = rng.integers(5, 40, size=2).astype(float)
    gq = rng.uniform(2, 20, size=2)
    Q, d, z = P(bq), P(iq), P(dq)
    a = 1 - (d + z)
    b1, b2 = 1 - P(gq[0]), 1 - P(gq[1])

    def lam(i, j):
        return (1 - Q[i - 1]) if read[i - 1] == hap[j - 1] else Q[i - 1] / 3

    L = (b1 / 3) * (lam(1, 1) * lam(2, 2) * a[1]
                    + lam(2, 3) * (lam(1, 2) * a[1] + b2 * z[0] * lam(1, 1))
                    + d[1] * (lam(1, 1) + lam(1, 2) + lam(1, 3)))
    got = oracle.forward_pair(read, bq, iq, dq, hap, gcp=10.0, gcp_q=gq)
    assert got == pytest.approx(math.log10(L), abs=1e-13)


def test_per_base_gcp_uniform_track_is_the_scalar():
    # a track holding the scalar value everywhere gives the scalar path's results exactly, and
    # its per-position gradients sum to the scalar d/dgcp
    b = synth.random_pairs(51, 20, (1, 40), (1, 60), alphabet=b"ACGTN", qual_dtype=np.float32)
    tot = int(b["read_off"][-1])
    bt = dict(b, gcp_q=np.full(tot, b["gcp"], dtype=np.float32))
    assert np.array_equal(oracle.forward_batch(bt), oracle.forward_batch(b))
    dy = np.random.default_rng(1).uniform(-1, 1, len(b["pair_read"]))
    y0, b0, i0, d0, g0 = oracle.backward_batch(b, dy)
    y1, b1, i1, d1, gq = oracle.backward_batch(bt, dy)
    for u, v in ((y0, y1), (b0, b1), (i0, i1), (d0, d1)):
        assert np.array_equal(u, v)
    assert gq.shape == (tot,)
    assert np.sum(gq) == pytest.approx(g0, rel=1e-12, abs=1e-12)


@pytest.mark.parametrize("seed", range(4))
def test_per_base_gcp_adjoint_vs_central_differences(seed):
    rng = np.random.default_rng(950 + seed)
    m, n = int(rng.integers(1, 20)), int(rng.integers(1, 30))
    hap = rand_seq(rng, n, "ACGTN")
    read = hap[:m] if (seed % 2 == 0 and m <= n) else rand_seq(rng, m, "ACGTN")
    bq = rng.uniform(2, 40, size=m)
    iq = rng.uniform(15, 45, size=m)
    dq = rng.uniform(15, 45, size=m)
    gq = rng.uniform(3, 25, size=m)
    y, gb, gi, gd, gg = oracle.backward_pair(read, bq, iq, dq, hap, gcp=10.0, dy=1.0, gcp_q=gq)
    assert gg.shape == (m,)
    for arr, g in ((bq, gb), (iq, gi), (dq, gd), (gq, gg)):
        for i in range(m):
            def fi(v, arr=arr, i=i):
                a = arr.copy()
                a[i] = v
                args = [a if arr is x else x for x in (bq, iq, dq, gq)]
                return oracle.forward_pair(read, args[0], args[1], args[2], hap, gcp=10.0,
                                           gcp_q=args[3])
            assert g[i] == pytest.approx(_fd(fi, arr[i]), rel=2e-5, abs=1e-9)


def test_invalid_inputs_give_nan():
    assert math.isnan(oracle.forward_pair("AXG", [30] * 3, [45] * 3, [45] * 3, "ACG"))
    assert math.isnan(oracle.forward_pair("ACG", [30] * 3, [45] * 3, [45] * 3, "AC-"))
    assert math.isnan(oracle.forward_pair("", [], [], [], "ACG"))
    assert math.isnan(oracle.forward_pair("A", [30], [45], [45], ""))
    assert math.isnan(oracle.forward_pair("A", [30], [45], [45], "A", gcp=0.0))
    assert math.isnan(oracle.forward_pair("A", [30], [1.0], [2.0], "A"))  # delta+zeta > 1
    assert math.isnan(oracle.forward_pair("A", [-1.0], [45], [45], "A"))


def test_batch_driver_matches_pairs():
    b = synth.random_pairs(21, 30, (1, 40), (1, 60), alphabet=b"ACGTN")
    got = oracle.forward_batch(b, nthreads=3)
    for p in range(30):
        r, h = b["pair_read"][p], b["pair_hap"][p]
        r0, r1 = b["read_off"][r], b["read_off"][r + 1]
        h0, h1 = b["hap_off"][h], b["hap_off"][h + 1]
        want = oracle.forward_pair(b["read_bases"][r0:r1], b["base_q"][r0:r1],
                                   b["ins_q"][r0:r1], b["del_q"][r0:r1],
                                   b["hap_bases"][h0:h1], gcp=b["gcp"])
        assert got[p] == want


# ---------------------------------------------------------------------------- adjoint -------

def test_adjoint_single_row_closed_form():
    # m = 1: L = (beta/n)(c_match (1-Q) + c_mis Q/3)
    hap = "ACGTAAGT"
    n = len(hap)
    q, gcp = 27.0, 12.0
    Q, eps = P(q), P(gcp)
    beta = 1 - eps
    cm = hap.count("A")
    cx = n - cm
    L = beta / n * (cm * (1 - Q) + cx * Q / 3)
    dQ = -math.log(10) / 10 * Q
    want_bq = (beta / (n * L * math.log(10))) * (cx / 3 - cm) * dQ
    want_gcp = (1 / (beta * math.log(10))) * (math.log(10) / 10) * eps
    y, gb, gi, gd, gg = oracle.backward_pair("A", [q], [33.0], [35.0], hap, gcp=gcp)
    assert y == pytest.approx(math.log10(L), abs=1e-14)
    assert gb[0] == pytest.approx(want_bq, rel=1e-12)
    assert gg == pytest.approx(want_gcp, rel=1e-12)
    assert gi[0] == 0.0 and gd[0] == 0.0


def _fd(fun, x, h=1e-4):
    return (fun(x + h) - fun(x - h)) / (2 * h)


@pytest.mark.parametrize("seed", range(6))
@pytest.mark.parametrize("alpha_mode", [0, 1])
def test_adjoint_vs_central_differences(seed, alpha_mode):
    rng = np.random.default_rng(900 + seed)
    m, n = int(rng.integers(1, 25)), int(rng.integers(1, 35))
    hap = rand_seq(rng, n, "ACGTN")
    read = hap[:m] if (seed % 2 == 0 and m <= n) else rand_seq(rng, m, "ACGTN")
    bq = rng.uniform(2, 40, size=m)
    iq = rng.uniform(15, 45, size=m)
    dq = rng.uniform(15, 45, size=m)
    gcp = float(rng.uniform(5, 25))
    dy = 1.7
    y, gb, gi, gd, gg = oracle.backward_pair(read, bq, iq, dq, hap, gcp=gcp,
                                             alpha_mode=alpha_mode, dy=dy)

    def f(bq_=bq, iq_=iq, dq_=dq, gcp_=gcp):
        return dy * oracle.forward_pair(read, bq_, iq_, dq_, hap, gcp=gcp_, alpha_mode=alpha_mode)

    for i in range(m):
        for arr, g in ((bq, gb), (iq, gi), (dq, gd)):
            def fi(v, arr=arr, i=i):
                a = arr.copy()
                a[i] = v
                kw = {"bq_": bq, "iq_": iq, "dq_": dq}
                key = "bq_" if arr is bq else ("iq_" if arr is iq else "dq_")
                kw[key] = a
                return f(**kw)
            fd = _fd(fi, arr[i])
            assert g[i] == pytest.approx(fd, rel=2e-5, abs=1e-9)
    fd = _fd(lambda v: f(gcp_=v), gcp)
    assert gg == pytest.approx(fd, rel=2e-5, abs=1e-9)


def test_adjoint_deep_underflow_regime():
    # an unrelated long pair whose likelihood is far below the FP32 and near the FP64 range:
    # the normalised adjoint must still match finite differences
    rng = np.random.default_rng(77)
    m, n = 120, 160
    read, hap = rand_seq(rng, m), rand_seq(rng, n)
    bq = rng.uniform(35, 40, size=m)
    iq = np.full(m, 40.0)
    dq = np.full(m, 40.0)
    y, gb, gi, gd, gg = oracle.backward_pair(read, bq, iq, dq, hap, gcp=10.0)
    assert y < -100
    for i in (0, 37, m - 1):
        def fb(v, i=i):
            a = bq.copy()
            a[i] = v
            return oracle.forward_pair(read, a, iq, dq, hap, gcp=10.0)
        assert gb[i] == pytest.approx(_fd(fb, bq[i]), rel=1e-5, abs=1e-9)


def test_backward_batch_sums_per_read():
    b = synth.random_pairs(31, 12, (2, 20), (2, 30), alphabet=b"ACGT")
    # make two pairs share read 0
    b["pair_read"] = b["pair_read"].copy()
    b["pair_read"][5] = 0
    dy = np.linspace(0.5, 2.0, 12)
    y, gb, gi, gd, gg = oracle.backward_batch(b, dy, nthreads=2)
    m0 = b["read_off"][1] - b["read_off"][0]
    acc = np.zeros(m0)
    tot_g = 0.0
    for p in range(12):
        r, h = b["pair_read"][p], b["pair_hap"][p]
        r0, r1 = b["read_off"][r], b["read_off"][r + 1]
        h0, h1 = b["hap_off"][h], b["hap_off"][h + 1]
        yy, g1, _, _, g4 = oracle.backward_pair(b["read_bases"][r0:r1], b["base_q"][r0:r1],
                                                b["ins_q"][r0:r1], b["del_q"][r0:r1],
                                                b["hap_bases"][h0:h1], gcp=b["gcp"], dy=dy[p])
        assert yy == y[p]
        if r == 0:
            acc += g1
        tot_g += g4
    np.testing.assert_allclose(gb[:m0], acc, rtol=1e-13, atol=0)
    assert gg == pytest.approx(tot_g, rel=1e-13)


def test_golden_tiny_pairs():
    import json
    import os
    path = os.path.join(os.path.dirname(__file__), "golden", "tiny_pairs.json")
    for c in json.load(open(path))["cases"]:
        got = oracle.forward_pair(c["read"], c["bq"], c["iq"], c["dq"], c["hap"], gcp=c["gcp"])
        assert got == pytest.approx(c["log10L"], abs=1e-12)
