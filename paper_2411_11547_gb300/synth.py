"""Seeded synthetic Pair-HMM batches shaped like the paper's workloads.

This module only draws inputs: bases, Phred qualities, offsets and the pair list.  It holds
none of the method's arithmetic and serves both the CUDA path and the CPU oracle.

Every batch is a dict of host numpy arrays:
  read_bases  uint8[sum m]    ASCII bases of all reads, concatenated
  base_q, ins_q, del_q        Phred per read base: uint8 (or float32 for differentiable runs)
  read_off    int64[R+1]      read r occupies read_bases[read_off[r]:read_off[r+1]]
  hap_bases   uint8[sum n]    ASCII haplotype bases, concatenated
  hap_off     int64[H+1]
  pair_read, pair_hap int32[P] the (read, haplotype) pairs to score
  gcp         float           Phred gap-continuation penalty (one scalar per batch)

Read model (used by every workload): haplotypes are uniform i.i.d. ACGT.  A read picks a
haplotype of its region at random (one at least as long as the read) and a uniform start
offset, then copies bases with 1% substitutions (the new base uniform over the other three)
and 0.1%-per-base indel events (length uniform 1..3, insertion or deletion with equal odds,
inserted bases uniform), until m bases are emitted (random bases pad the end if the
haplotype runs out).  Regions are scored all-vs-all (every read against every haplotype),
as in the paper's batches B_q = (R_q, H_q) (Sec. II-A).
"""
from __future__ import annotations

import numpy as np

ACGT = np.frombuffer(b"ACGT", dtype=np.uint8)

# Workload names, in the order they are described in the design notes.
WORKLOADS = ("c0_plain", "c1_batched", "c2_stress", "c3_grad", "c4_persistent")


def _sample_reads(rng, hap_seqs, m, src_hap):
    """Reads of lengths m[k] sampled from hap_seqs[src_hap[k]] with the error model."""
    nreads = len(m)
    out = []
    n_src = np.array([len(hap_seqs[h]) for h in src_hap], dtype=np.int64)
    offs = (rng.random(nreads) * (n_src - m + 1)).astype(np.int64)
    n_events = rng.binomial(m, 0.001)
    for k in range(nreads):
        h = hap_seqs[src_hap[k]]
        mk = int(m[k])
        if n_events[k] == 0:
            seg = h[offs[k]:offs[k] + mk].copy()
        else:
            # event positions (in emitted-base index) and their kinds
            pos = np.sort(rng.choice(mk, size=int(n_events[k]), replace=False))
            kinds = rng.random(len(pos)) < 0.5  # True = insertion
            lens = rng.integers(1, 4, size=len(pos))
            parts = []
            p = int(offs[k])
            emitted = 0
            for e_pos, ins, ln in zip(pos, kinds, lens):
                take = int(e_pos) - emitted
                if take > 0:
                    chunk = h[p:p + take]
                    parts.append(chunk)
                    emitted += len(chunk)
                    p += take
                if ins:
                    parts.append(ACGT[rng.integers(0, 4, size=int(ln))])
                    emitted += int(ln)
                else:
                    p += int(ln)
            rest = mk - emitted
            if rest > 0:
                parts.append(h[p:p + rest])
            seg = np.concatenate(parts)[:mk] if parts else np.empty(0, np.uint8)
        if len(seg) < mk:
            seg = np.concatenate([seg, ACGT[rng.integers(0, 4, size=mk - len(seg))]])
        seg = np.array(seg, dtype=np.uint8)
        # substitutions: new base uniform among the other three
        sub = rng.random(mk) < 0.01
        if sub.any():
            cur = np.searchsorted(ACGT, seg[sub])
            cur = np.where(cur < 4, cur, 0)
            seg[sub] = ACGT[(cur + rng.integers(1, 4, size=int(sub.sum()))) % 4]
        out.append(seg)
    return out


def _assemble(regions, gcp, name, qual_dtype=np.uint8):
    """regions: list of (hap_seqs, read_seqs, bq, iq, dq) -> batch dict, all-vs-all pairs."""
    haps, reads, bqs, iqs, dqs = [], [], [], [], []
    pr, ph = [], []
    h_base = r_base = 0
    for hap_seqs, read_seqs, bq, iq, dq in regions:
        H, R = len(hap_seqs), len(read_seqs)
        haps.extend(hap_seqs)
        reads.extend(read_seqs)
        bqs.extend(bq)
        iqs.extend(iq)
        dqs.extend(dq)
        rr, hh = np.meshgrid(np.arange(R), np.arange(H), indexing="ij")
        pr.append((rr.ravel() + r_base).astype(np.int32))
        ph.append((hh.ravel() + h_base).astype(np.int32))
        h_base += H
        r_base += R
    read_len = np.array([len(r) for r in reads], dtype=np.int64)
    hap_len = np.array([len(h) for h in haps], dtype=np.int64)
    return {
        "name": name,
        "read_bases": np.concatenate(reads).astype(np.uint8),
        "base_q": np.concatenate(bqs).astype(qual_dtype),
        "ins_q": np.concatenate(iqs).astype(qual_dtype),
        "del_q": np.concatenate(dqs).astype(qual_dtype),
        "read_off": np.concatenate([[0], np.cumsum(read_len)]).astype(np.int64),
        "hap_bases": np.concatenate(haps).astype(np.uint8),
        "hap_off": np.concatenate([[0], np.cumsum(hap_len)]).astype(np.int64),
        "pair_read": np.concatenate(pr),
        "pair_hap": np.concatenate(ph),
        "gcp": float(gcp),
    }


def _region(rng, hap_lens, read_lens, bq_fn, gap_fn):
    hap_seqs = [ACGT[rng.integers(0, 4, size=int(n))] for n in hap_lens]
    hl = np.array(hap_lens)
    src = np.empty(len(read_lens), dtype=np.int64)
    for k, mk in enumerate(read_lens):
        ok = np.nonzero(hl >= mk)[0]
        src[k] = ok[rng.integers(0, len(ok))]
    read_seqs = _sample_reads(rng, hap_seqs, np.asarray(read_lens, dtype=np.int64), src)
    bq = [bq_fn(rng, len(r)) for r in read_seqs]
    iq = [gap_fn(rng, len(r)) for r in read_seqs]
    dq = [gap_fn(rng, len(r)) for r in read_seqs]
    return hap_seqs, read_seqs, bq, iq, dq


def _bq_uniform(lo, hi):
    return lambda rng, m: rng.integers(lo, hi + 1, size=m)


def _const(v):
    return lambda rng, m: np.full(m, v)


def c0_plain(seed=0, n_haps=16, n_reads=64, m=150, n=300):
    """One region: 16 haplotypes (length 300) x 64 reads (length 150), all-vs-all = 1,024
    pairs (46.08 M cells).  bq uniform 10..40, ins/del gap-open quals 45, GCP 10."""
    rng = np.random.default_rng(seed)
    reg = _region(rng, [n] * n_haps, [m] * n_reads, _bq_uniform(10, 40), _const(45))
    return _assemble([reg], 10.0, "c0_plain")


def _bq_mixture(rng, m):
    lo = rng.random(m) < 0.2
    return np.where(lo, rng.integers(2, 16, size=m), rng.integers(25, 41, size=m))


def c1_batched(seed=1, regions=2000):
    """Uneven-length batch: per region 2..16 haplotypes (length uniform 100..600) and 20..200
    reads (length lognormal, mean 150, sigma_log 0.35, redrawn outside 50..250); bq a mixture
    (80% uniform 25..40, 20% uniform 2..15), ins/del quals uniform 30..45, GCP 10."""
    rng = np.random.default_rng(seed)
    sig = 0.35
    mu = np.log(150.0) - sig * sig / 2
    regs = []
    for _ in range(regions):
        H = int(rng.integers(2, 17))
        R = int(rng.integers(20, 201))
        hl = rng.integers(100, 601, size=H)
        rl = []
        while len(rl) < R:
            v = int(round(float(rng.lognormal(mu, sig))))
            if 50 <= v <= 250 and v <= hl.max():
                rl.append(v)
        regs.append(_region(rng, hl, rl, _bq_mixture, _bq_uniform(30, 45)))
    return _assemble(regs, 10.0, "c1_batched")


def c2_stress(seed=2, regions=12500):
    """Underflow / long-pair stress: per region 4 haplotypes (length 500..1500) x 1 read
    (length 250..500) = 50,000 pairs.  bq uniform 10..40; 30% of reads get 1-2 runs of
    50..150 bases with bq 2..6; 5% of reads get 1-5 'N' bases; ins/del 30..45; GCP 10."""
    rng = np.random.default_rng(seed)
    regs = []
    for _ in range(regions):
        hl = rng.integers(500, 1501, size=4)
        mk = int(rng.integers(250, 501))
        hap_seqs, read_seqs, bq, iq, dq = _region(rng, hl, [mk], _bq_uniform(10, 40),
                                                  _bq_uniform(30, 45))
        if rng.random() < 0.30:
            for _ in range(int(rng.integers(1, 3))):
                ln = int(rng.integers(50, 151))
                st = int(rng.integers(0, max(1, mk - ln + 1)))
                bq[0][st:st + ln] = rng.integers(2, 7, size=min(ln, mk - st))
        if rng.random() < 0.05:
            k = int(rng.integers(1, 6))
            pos = rng.choice(mk, size=k, replace=False)
            read_seqs[0] = read_seqs[0].copy()
            read_seqs[0][pos] = ord("N")
        regs.append((hap_seqs, read_seqs, bq, iq, dq))
    return _assemble(regs, 10.0, "c2_stress")


def c3_grad(seed=3, pairs=100_000):
    """Differentiation workload: C0-shaped groups (16 haplotypes x 64 reads, m=150, n=300)
    repeated up to 100,000 pairs (97 full groups and one of 16 x 42); quals as float32."""
    rng = np.random.default_rng(seed)
    regs = []
    left = pairs
    while left > 0:
        R = min(64, left // 16)
        regs.append(_region(rng, [300] * 16, [150] * R, _bq_uniform(10, 40), _const(45)))
        left -= 16 * R
    return _assemble(regs, 10.0, "c3_grad", qual_dtype=np.float32)


def _log_uniform_int(rng, lo, hi, size):
    return np.floor(np.exp(rng.uniform(np.log(lo), np.log(hi + 1), size=size))).astype(np.int64)


def _bulk(rng, hap_len, hap_region, read_len, read_region, n_regions, bq, iq, dq, gcp, name,
          qual_dtype=np.uint8):
    """Vectorised batch of many regions (same read model as _sample_reads): haplotype and
    read lengths and region ids are given; bases, sources, offsets and errors are drawn here.
    Pairs are all-vs-all within each region."""
    H, R = len(hap_len), len(read_len)
    hap_off = np.concatenate([[0], np.cumsum(hap_len)]).astype(np.int64)
    hap_bases = ACGT[rng.integers(0, 4, size=int(hap_off[-1]))]
    # source haplotype: uniform among the region's haplotypes at least as long as the read
    order = np.argsort(hap_region, kind="stable")
    reg_first = np.searchsorted(hap_region[order], np.arange(n_regions))
    reg_count = np.bincount(hap_region, minlength=n_regions)
    maxh = int(reg_count.max())
    cand = np.full((R, maxh), -1, dtype=np.int64)
    for k in range(maxh):
        has = k < reg_count[read_region]
        h = order[np.minimum(reg_first[read_region] + k, H - 1)]
        ok = has & (hap_len[h] >= read_len)
        cand[:, k] = np.where(ok, h, -1)
    n_ok = (cand >= 0).sum(axis=1)
    assert np.all(n_ok > 0), "every read needs a haplotype at least as long"
    pick = np.floor(rng.random(R) * n_ok).astype(np.int64)
    srt = np.sort(np.where(cand >= 0, cand, np.iinfo(np.int64).max), axis=1)
    src = srt[np.arange(R), pick]
    offs = np.floor(rng.random(R) * (hap_len[src] - read_len + 1)).astype(np.int64)
    read_off = np.concatenate([[0], np.cumsum(read_len)]).astype(np.int64)
    tot = int(read_off[-1])
    within = np.arange(tot) - np.repeat(read_off[:-1], read_len)
    gidx = np.repeat(hap_off[src] + offs, read_len) + within
    read_bases = hap_bases[gidx].copy()
    # indel events (rare): redraw those reads with the per-read sampler
    n_events = rng.binomial(read_len, 0.001)
    for r in np.nonzero(n_events)[0]:
        h = src[r]
        seg = _sample_reads(rng, [hap_bases[hap_off[h]:hap_off[h + 1]]],
                            np.array([read_len[r]]), np.array([0]))[0]
        read_bases[read_off[r]:read_off[r + 1]] = seg
    # substitutions on the reads without indel events (the redrawn ones carry their own)
    sub = (rng.random(tot) < 0.01) & ~np.repeat(n_events > 0, read_len)
    if sub.any():
        cur = np.searchsorted(ACGT, read_bases[sub])
        read_bases[sub] = ACGT[(cur + rng.integers(1, 4, size=int(sub.sum()))) % 4]
    # all-vs-all pairs within each region
    r_order = np.argsort(read_region, kind="stable")
    pr, ph = [], []
    for k in range(maxh):
        sel = k < reg_count[read_region[r_order]]
        rr = r_order[sel]
        pr.append(rr)
        ph.append(order[reg_first[read_region[rr]] + k])
    pr = np.concatenate(pr)
    ph = np.concatenate(ph)
    o = np.lexsort((ph, pr))  # read-major, then haplotype
    return {
        "name": name,
        "read_bases": read_bases.astype(np.uint8),
        "base_q": bq(tot).astype(qual_dtype),
        "ins_q": iq(tot).astype(qual_dtype),
        "del_q": dq(tot).astype(qual_dtype),
        "read_off": read_off,
        "hap_bases": hap_bases.astype(np.uint8),
        "hap_off": hap_off,
        "pair_read": pr[o].astype(np.int32),
        "pair_hap": ph[o].astype(np.int32),
        "gcp": float(gcp),
    }


def c4_persistent(seed=4, regions=65536, n_haps=4, n_reads=16):
    """Persistent-kernel batch: 65,536 regions x 4 haplotypes x 16 reads = 2^22 pairs; read
    length log-uniform 36..300, haplotype length log-uniform 64..2048; quals as C0."""
    rng = np.random.default_rng(seed)
    hl = np.minimum(_log_uniform_int(rng, 64, 2048, regions * n_haps), 2048)
    rl = np.minimum(_log_uniform_int(rng, 36, 300, regions * n_reads), 300)
    hap_region = np.repeat(np.arange(regions), n_haps)
    read_region = np.repeat(np.arange(regions), n_reads)
    rl = np.minimum(rl, hl.reshape(regions, n_haps).max(axis=1)[read_region])
    return _bulk(rng, hl, hap_region, rl, read_region, regions,
                 lambda k: rng.integers(10, 41, size=k), lambda k: np.full(k, 45),
                 lambda k: np.full(k, 45), 10.0, "c4_persistent")


def na12878_like(seed=5, regions=100_000):
    """Stand-in for the end-to-end scoring workload of Table I (NA12878: 55.1 M pairs in
    998,837 batches, reads 10..151 with mean 58, haplotypes 30..521): per region 1..6
    haplotypes and 2..30 reads (about 55 pairs per region), read length log-uniform 10..151,
    haplotype length log-uniform 30..521 with each region's first haplotype at least as long
    as its longest read; quals as C1.  100,000 regions is about a tenth of the dataset."""
    rng = np.random.default_rng(seed)
    nh = rng.integers(1, 7, size=regions)
    nr = rng.integers(2, 31, size=regions)
    hap_region = np.repeat(np.arange(regions), nh)
    read_region = np.repeat(np.arange(regions), nr)
    rl = np.minimum(_log_uniform_int(rng, 10, 151, int(nr.sum())), 151)
    hl = np.minimum(_log_uniform_int(rng, 30, 521, int(nh.sum())), 521)
    maxr = np.zeros(regions, dtype=np.int64)
    np.maximum.at(maxr, read_region, rl)
    first = np.concatenate([[0], np.cumsum(nh)[:-1]])
    hl[first] = np.maximum(hl[first], maxr)

    def bq(k):
        lo = rng.random(k) < 0.2
        return np.where(lo, rng.integers(2, 16, size=k), rng.integers(25, 41, size=k))

    return _bulk(rng, hl, hap_region, rl, read_region, regions, bq,
                 lambda k: rng.integers(30, 46, size=k), lambda k: rng.integers(30, 46, size=k),
                 10.0, "na12878_like")


def make(name: str, **kw):
    return {"c0_plain": c0_plain, "c1_batched": c1_batched, "c2_stress": c2_stress,
            "c3_grad": c3_grad, "c4_persistent": c4_persistent,
            "na12878_like": na12878_like}[name](**kw)


def subset_pairs(batch, idx):
    """A batch holding only the pairs idx (reads and haplotypes are shared, not copied)."""
    out = dict(batch)
    out["pair_read"] = np.ascontiguousarray(batch["pair_read"][idx])
    out["pair_hap"] = np.ascontiguousarray(batch["pair_hap"][idx])
    return out


def cells(batch) -> int:
    """Sum over pairs of m * n (real, unpadded lengths): the numerator of Eq. 5."""
    rl = np.diff(batch["read_off"])
    hl = np.diff(batch["hap_off"])
    return int(np.sum(rl[batch["pair_read"]] * hl[batch["pair_hap"]]))


def random_pairs(seed, n_pairs, m_range, n_range, q_range=(10, 40), gap_q=(30, 45),
                 alphabet=b"ACGT", related=0.5, qual_dtype=np.uint8, gcp=10.0):
    """Independent random pairs (one read, one haplotype each) for edge-case and parity tests.
    A fraction `related` of reads is sampled from its haplotype with the error model."""
    rng = np.random.default_rng(seed)
    alph = np.frombuffer(alphabet, dtype=np.uint8)
    regs = []
    for _ in range(n_pairs):
        n = int(rng.integers(n_range[0], n_range[1] + 1))
        m = int(rng.integers(m_range[0], m_range[1] + 1))
        hap = alph[rng.integers(0, len(alph), size=n)]
        if rng.random() < related and n >= m:
            rd = _sample_reads(rng, [hap], np.array([m]), np.array([0]))[0]
        else:
            rd = alph[rng.integers(0, len(alph), size=m)]
        bq = rng.integers(q_range[0], q_range[1] + 1, size=m)
        iq = rng.integers(gap_q[0], gap_q[1] + 1, size=m)
        dq = rng.integers(gap_q[0], gap_q[1] + 1, size=m)
        regs.append(([hap], [rd], [bq], [iq], [dq]))
    return _assemble(regs, gcp, "random_pairs", qual_dtype=qual_dtype)
