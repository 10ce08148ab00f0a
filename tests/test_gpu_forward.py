"""GPU parity of the forward pass against the FP64 oracle, through the C ABI.

Bars: |d log10 L| <= 1e-3 for pairs scored by an FP32 wavefront, <= 1e-9 for pairs the FP64
rescue recomputed (checked by flag).  Inputs are seeded synthetic batches.
"""
import json
import os

import numpy as np
import pytest

import oracle
from paper_2411_11547_gb300 import synth

pytestmark = pytest.mark.gpu

TOL32, TOL64 = 1e-3, 1e-9


@pytest.fixture(scope="module")
def phmm():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2411_11547_gb300 import _build, phmm as ph
    _build.build()
    ph.lib()
    return ph


def run(ph, batch, **opt):
    import torch
    plan = ph.Plan(ph.DeviceBatch(batch), ph.options(**opt))
    out, flags = plan.forward()
    torch.cuda.synchronize()
    return out.cpu().numpy(), flags.cpu().numpy(), plan


def check(got, flags, want, ph, allow_invalid=False):
    assert got.shape == want.shape
    fp32 = (flags & ph.FLAG_FP32) != 0
    r64 = (flags & ph.FLAG_RESCUED64) != 0
    inv = (flags & ph.FLAG_INVALID) != 0
    if not allow_invalid:
        assert not inv.any()
    assert np.all(fp32 | r64 | inv), "pair without a result flag"
    fin = np.isfinite(want)
    e = np.abs(got - want)
    if (fp32 & fin).any():
        assert e[fp32 & fin].max() <= TOL32, f"FP32 path max err {e[fp32 & fin].max():.3g}"
    if (r64 & fin).any():
        assert e[r64 & fin].max() <= TOL64, f"rescued max err {e[r64 & fin].max():.3g}"
    # pairs with L == 0 exactly: both sides -inf
    assert np.all(got[~fin & ~inv] == want[~fin & ~inv])
    return e


@pytest.mark.parametrize("first_line", [0, 1])
def test_random_pairs_binned(phmm, first_line):
    b = synth.random_pairs(5, 600, (1, 300), (1, 700), alphabet=b"ACGTN", related=0.5)
    got, flags, _ = run(phmm, b, first_line=first_line)
    check(got, flags, oracle.forward_batch(b), phmm)
    if first_line == 0:
        assert (flags & phmm.FLAG_RESCUED64).any(), "expected some FP64 rescues"


@pytest.mark.parametrize("lanes", [4, 8, 16, 32])
@pytest.mark.parametrize("rows", [4, 6, 8, 10, 12, 14, 16, 18, 20])
@pytest.mark.parametrize("ext", [0, 1])
def test_every_fixed_group(phmm, lanes, rows, ext):
    cap = min(lanes * rows, 512)
    b = synth.random_pairs(lanes * 100 + rows + ext, 70, (1, cap), (1, 400), alphabet=b"ACGTN")
    got, flags, _ = run(phmm, b, binning=0, lanes=lanes, rows=rows, first_line=ext, rescue=1,
                        persistent=lanes % 8 == 0)
    check(got, flags, oracle.forward_batch(b), phmm)


def test_plain_kernel_without_rescue_flags_everything_fp32(phmm):
    b = synth.c0_plain()
    got, flags, _ = run(phmm, b, binning=0, lanes=16, rows=12, first_line=0, rescue=0,
                        persistent=0, use_graph=0)
    assert np.all(flags == phmm.FLAG_FP32)
    want = oracle.forward_batch(b)
    ok = want > -60  # within the FP32 range of K0 = 2^120
    assert np.abs(got[ok] - want[ok]).max() <= TOL32


def test_c0_full_all_paths(phmm):
    b = synth.c0_plain()
    want = oracle.forward_batch(b)
    for fl in (0, 1):
        got, flags, _ = run(phmm, b, first_line=fl)
        check(got, flags, want, phmm)


def test_golden_tiny_pairs(phmm):
    path = os.path.join(os.path.dirname(__file__), "golden", "tiny_pairs.json")
    cases = json.load(open(path))["cases"]
    regs = []
    for c in cases:
        regs.append(([np.frombuffer(c["hap"].encode(), np.uint8)],
                     [np.frombuffer(c["read"].encode(), np.uint8)],
                     [np.array(c["bq"])], [np.array(c["iq"])], [np.array(c["dq"])]))
    # one batch per gcp value
    for gcp in sorted({c["gcp"] for c in cases}):
        sel = [i for i, c in enumerate(cases) if c["gcp"] == gcp]
        b = synth._assemble([regs[i] for i in sel], gcp, "golden")
        want = np.array([cases[i]["log10L"] for i in sel])
        for fl in (0, 1):
            got, flags, _ = run(phmm, b, first_line=fl)
            check(got, flags, want, phmm)


def test_edge_lengths(phmm):
    rng = np.random.default_rng(3)
    regs = []
    for m, n in [(1, 1), (1, 2000), (512, 512), (512, 3000), (300, 1), (4, 4), (33, 17),
                 (160, 160), (161, 5000), (500, 8)]:
        hap = synth.ACGT[rng.integers(0, 4, n)]
        read = hap[:m].copy() if m <= n else synth.ACGT[rng.integers(0, 4, m)]
        regs.append(([hap], [read], [rng.integers(10, 41, m)], [rng.integers(30, 46, m)],
                     [rng.integers(30, 46, m)]))
    b = synth._assemble(regs, 10.0, "edges")
    want = oracle.forward_batch(b)
    for fl in (0, 1):
        got, flags, _ = run(phmm, b, first_line=fl)
        check(got, flags, want, phmm)


def test_float_quals_and_alpha_mode(phmm):
    b = synth.random_pairs(8, 200, (5, 250), (5, 400), qual_dtype=np.float32, related=0.7)
    rng = np.random.default_rng(1)
    b["base_q"] = (b["base_q"] + rng.uniform(0, 1, b["base_q"].shape)).astype(np.float32)
    for am in (0, 1):
        bb = dict(b, alpha_mode=am)
        got, flags, _ = run(phmm, bb)
        check(got, flags, oracle.forward_batch(bb), phmm)


def test_stress_low_quals_and_N(phmm):
    full = synth.c2_stress(regions=150)
    got, flags, _ = run(phmm, full, first_line=0)
    check(got, flags, oracle.forward_batch(full), phmm)
    got2, flags2, _ = run(phmm, full, first_line=1)
    check(got2, flags2, oracle.forward_batch(full), phmm)


def test_empty_pair_list(phmm):
    b = synth.random_pairs(1, 3, (5, 10), (5, 10))
    b["pair_read"] = b["pair_read"][:0]
    b["pair_hap"] = b["pair_hap"][:0]
    got, flags, _ = run(phmm, b)
    assert got.shape == (0,)


def test_graph_replay_and_determinism(phmm):
    import torch
    b = synth.c1_batched(regions=12)
    plan = phmm.Plan(phmm.DeviceBatch(b), phmm.options())
    o1, f1 = plan.forward()
    o1 = o1.clone()
    o2, f2 = plan.forward()
    torch.cuda.synchronize()
    assert torch.equal(o1, o2) and torch.equal(f1, f2)
    plan2 = phmm.Plan(phmm.DeviceBatch(b), phmm.options(use_graph=0))
    o3, _ = plan2.forward()
    torch.cuda.synchronize()
    assert torch.equal(o1, o3)
    # batch order invariance: permuted pair list gives permuted results
    perm = np.random.default_rng(0).permutation(len(b["pair_read"]))
    bp = synth.subset_pairs(b, perm)
    plan3 = phmm.Plan(phmm.DeviceBatch(bp), phmm.options())
    o4, _ = plan3.forward()
    torch.cuda.synchronize()
    assert torch.equal(o4.cpu(), o1.cpu()[perm])


def test_invalid_inputs_are_rejected(phmm):
    b = synth.random_pairs(2, 4, (5, 10), (5, 10))
    bad = dict(b, read_bases=b["read_bases"].copy())
    bad["read_bases"][0] = ord("X")
    with pytest.raises(phmm.PhmmError) as e:
        phmm.Plan(phmm.DeviceBatch(bad))
    assert e.value.status == phmm.PHMM_EINVAL
    bad = dict(b, pair_hap=b["pair_hap"].copy())
    bad["pair_hap"][1] = 99
    with pytest.raises(phmm.PhmmError) as e:
        phmm.Plan(phmm.DeviceBatch(bad))
    assert e.value.status == phmm.PHMM_EINVAL
    bad = dict(b, gcp=0.0)
    with pytest.raises(phmm.PhmmError):
        phmm.Plan(phmm.DeviceBatch(bad))
    bad = dict(b, ins_q=np.zeros_like(b["ins_q"]))  # delta + zeta > 1
    with pytest.raises(phmm.PhmmError):
        phmm.Plan(phmm.DeviceBatch(bad))
    long = synth.random_pairs(2, 2, (2049, 2060), (600, 700))
    with pytest.raises(phmm.PhmmError) as e:
        phmm.Plan(phmm.DeviceBatch(long))
    assert e.value.status == phmm.PHMM_ETOOLONG
    plan = phmm.Plan(phmm.DeviceBatch(b))
    import ctypes
    import torch
    P = len(b["pair_read"])
    out = torch.empty(P, dtype=torch.float64, device="cuda")
    fl = torch.empty(P, dtype=torch.uint8, device="cuda")
    ws = ctypes.c_void_p(plan._ws_ptr)
    # a workspace one byte short of phmm_workspace_bytes, everything else valid: PHMM_ENOMEM
    for fn in (phmm.lib().phmm_forward, phmm.lib().phmm_forward_partials):
        rc = fn(plan.handle, ws, plan.ws_bytes - 1, ctypes.c_void_p(out.data_ptr()),
                ctypes.c_void_p(fl.data_ptr()), None)
        assert rc == phmm.PHMM_ENOMEM
    # enough workspace but no output arrays: PHMM_EINVAL; a misaligned workspace: PHMM_EINVAL
    rc = phmm.lib().phmm_forward(plan.handle, ws, plan.ws_bytes, ctypes.c_void_p(0),
                                 ctypes.c_void_p(0), None)
    assert rc == phmm.PHMM_EINVAL
    rc = phmm.lib().phmm_forward(plan.handle, ctypes.c_void_p(plan._ws_ptr + 16), plan.ws_bytes,
                                 ctypes.c_void_p(out.data_ptr()), ctypes.c_void_p(fl.data_ptr()),
                                 None)
    assert rc == phmm.PHMM_EINVAL
    # the same plan with the full workspace works
    rc = phmm.lib().phmm_forward(plan.handle, ws, plan.ws_bytes, ctypes.c_void_p(out.data_ptr()),
                                 ctypes.c_void_p(fl.data_ptr()), None)
    assert rc == phmm.PHMM_OK
    torch.cuda.synchronize()
    check(out.cpu().numpy(), fl.cpu().numpy(), oracle.forward_batch(b), phmm)


def test_extended_range_fp64_untiled(phmm):
    """Pairs beyond the FP64 range of K0 = 2^1020 (log10 L < -597) under the paper's plain
    FP32 first line: FP32 underflows, the FP64 rescue underflows too, and the per-lane-
    exponent FP64 kernels (32 lanes x 4 / 8 / 16 rows, no row tiles) finish them.  Unrelated
    reads with Phred-150 bases and gap opens and a Phred-150 gap continuation cost about 7
    log10 units per row (a mismatch 15.5, a gap 15 plus 15 per base)."""
    rng = np.random.default_rng(77)
    regs = []
    for m in [100, 120, 128, 140, 200, 256, 300, 380, 450, 512]:
        for rep in range(3):
            n = int(rng.integers(200, 700))
            hap = synth.ACGT[rng.integers(0, 4, n)]
            read = synth.ACGT[rng.integers(0, 4, m)]
            regs.append(([hap], [read], [np.full(m, 150)], [np.full(m, 150)], [np.full(m, 150)]))
    # and some ordinary related pairs in the same batch (FP32 or plain FP64 rescue)
    short = synth.random_pairs(78, 40, (30, 300), (300, 500), related=1.0)
    b = synth._assemble(regs, 150.0, "deep")
    for k in ("read_bases", "base_q", "ins_q", "del_q", "hap_bases"):
        b[k] = np.concatenate([b[k], short[k]])
    b["read_off"] = np.concatenate([b["read_off"], b["read_off"][-1] + short["read_off"][1:]])
    b["hap_off"] = np.concatenate([b["hap_off"], b["hap_off"][-1] + short["hap_off"][1:]])
    b["pair_read"] = np.concatenate([b["pair_read"], short["pair_read"] + len(regs)]).astype(np.int32)
    b["pair_hap"] = np.concatenate([b["pair_hap"], short["pair_hap"] + len(regs)]).astype(np.int32)
    want = oracle.forward_batch(b)
    deep = np.arange(len(regs))
    assert np.all(want[deep] < -597.1), want[deep].max()
    got, flags, plan = run(phmm, b, first_line=0, use_graph=0)
    counts = plan.rescue_counts()
    assert counts[1] >= len(regs), counts
    ext64 = phmm.FLAG_RESCUED64 | phmm.FLAG_EXTENDED
    assert np.all(flags[deep] == ext64), np.unique(flags[deep])
    # every untiled FP64 group ran: reads up to 128, 256 and 512 rows
    rl = np.diff(b["read_off"])[b["pair_read"]]
    for lo, hi in ((1, 128), (129, 256), (257, 512)):
        assert np.any((flags == ext64) & (rl >= lo) & (rl <= hi)), (lo, hi)
    check(got, flags, want, phmm)


def test_c4_sampled_pairs_full_size_launch(phmm):
    """C4 at full size (2^22 pairs) in the bench's launch configuration (autotuned group
    tables); a stratified sample of pairs (every length bin, the longest ones) is compared
    with the oracle."""
    b = synth.c4_persistent()
    db = phmm.DeviceBatch(b)
    o = phmm.autotune(db, which=1)
    plan = phmm.Plan(db, o)
    out, fl = plan.forward()
    got, flags = out.cpu().numpy(), fl.cpu().numpy()
    assert np.all((flags & phmm.FLAG_INVALID) == 0)
    rl = np.diff(b["read_off"])[b["pair_read"]]
    hl = np.diff(b["hap_off"])[b["pair_hap"]]
    rng = np.random.default_rng(44)
    idx = list(rng.choice(len(rl), 3000, replace=False))
    idx += list(np.argsort(rl * hl)[-200:])  # the largest pairs
    idx = np.unique(np.array(idx))
    sb = synth.subset_pairs(b, idx)
    check(got[idx], flags[idx], oracle.forward_batch(sb), phmm)


@pytest.mark.parametrize("first_line", [0, 1])
def test_long_reads_in_row_tiles(phmm, first_line):
    # reads longer than one group (512 rows) are swept in row tiles of 512, alone and mixed
    # with short reads in one binned batch; the plain first line sends them through the
    # tiled FP64 and per-lane-exponent FP64 kernels
    rng = np.random.default_rng(31)
    regs = []
    for m, n in [(513, 700), (600, 40), (1024, 1100), (1500, 300), (2048, 2100), (777, 777),
                 (1025, 5), (520, 1)]:
        hap = synth.ACGT[rng.integers(0, 4, n)]
        if n >= m and rng.random() < 0.7:
            o = int(rng.integers(0, n - m + 1))
            read = hap[o:o + m].copy()
            sub = rng.random(m) < 0.01
            read[sub] = synth.ACGT[rng.integers(0, 4, int(sub.sum()))]
        else:
            read = synth.ACGT[rng.integers(0, 4, m)]
        regs.append(([hap], [read], [rng.integers(10, 41, m)], [rng.integers(30, 46, m)],
                     [rng.integers(30, 46, m)]))
    short = synth.random_pairs(32, 60, (1, 512), (1, 600), related=0.5)
    b = synth._assemble(regs, 10.0, "long_reads")
    for k in ("read_bases", "base_q", "ins_q", "del_q", "hap_bases"):
        b[k] = np.concatenate([b[k], short[k]])
    b["read_off"] = np.concatenate([b["read_off"], b["read_off"][-1] + short["read_off"][1:]])
    b["hap_off"] = np.concatenate([b["hap_off"], b["hap_off"][-1] + short["hap_off"][1:]])
    nr, nh = len(regs), len(regs)
    b["pair_read"] = np.concatenate([b["pair_read"], short["pair_read"] + nr]).astype(np.int32)
    b["pair_hap"] = np.concatenate([b["pair_hap"], short["pair_hap"] + nh]).astype(np.int32)
    got, flags, plan = run(phmm, b, first_line=first_line)
    check(got, flags, oracle.forward_batch(b), phmm)
    # the adjoint sweeps the same row tiles (bottom to top): gradients against the oracle's,
    # through phmm_backward and through the fused step, in FP32 and with every pair in FP64
    from test_gpu_backward import check_against_oracle
    dy = np.random.default_rng(first_line).uniform(-1, 1, len(got))
    bf = dict(b, base_q=b["base_q"].astype(np.float32), ins_q=b["ins_q"].astype(np.float32),
              del_q=b["del_q"].astype(np.float32))
    check_against_oracle(phmm, bf, dy, first_line=first_line,
                         adjoint_rescue=2 if first_line == 0 else 1)


def test_metamorphic_order_blocks_and_bins(phmm):
    """The result of a pair does not depend on the batch order, on pairs per block (warps per
    block) or on bin edges that keep its group: bitwise.  Across groups: within tolerance."""
    b = synth.c1_batched(regions=5)
    base, bflags, _ = run(phmm, b)
    perm = np.random.default_rng(8).permutation(len(b["pair_read"]))
    pb = dict(b, pair_read=b["pair_read"][perm].copy(), pair_hap=b["pair_hap"][perm].copy())
    for wpb in (1, 2, 4):
        got, flags, _ = run(phmm, pb, warps_per_block=wpb)
        assert np.array_equal(got, base[perm]) and np.array_equal(flags, bflags[perm])
    # bin edges moved: reads of every length scored by the wider 32 x 16 group
    got, flags, _ = run(phmm, b, bin_rows=[phmm.cfg_index(32, 16)] * 129)
    assert np.max(np.abs(got - base)) <= 2e-4
