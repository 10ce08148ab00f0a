"""The seeded synthetic workloads (CPU): sizes, length ranges, quality recipes and determinism.

These batches stand in for the paper's datasets in every parity test and in the benchmark, so
their shapes are pinned here: a change to a generator shows up as a failing test, not as a
silently different benchmark workload.
"""
import numpy as np
import pytest

from paper_2411_11547_gb300 import synth


def lengths(b):
    return np.diff(b["read_off"]), np.diff(b["hap_off"])


def test_c0_one_all_vs_all_region():
    b = synth.make("c0_plain")
    rl, hl = lengths(b)
    assert len(rl) == 64 and len(hl) == 16 and len(b["pair_read"]) == 1024
    assert np.all(rl == 150) and np.all(hl == 300)
    assert synth.cells(b) == 1024 * 150 * 300
    # every read meets every haplotype exactly once
    pairs = set(zip(b["pair_read"].tolist(), b["pair_hap"].tolist()))
    assert len(pairs) == 1024
    bq = np.asarray(b["base_q"])
    assert bq.min() >= 10 and bq.max() <= 40
    assert np.all(np.asarray(b["ins_q"]) == 45) and np.all(np.asarray(b["del_q"]) == 45)
    assert b["gcp"] == 10.0


def test_reads_are_sampled_from_their_region():
    # each read is a copy of one of its region's haplotypes with ~1% substitutions and rare
    # indels: its best ungapped window on some haplotype of the region matches far above the
    # 25% of an unrelated sequence
    b = synth.make("c0_plain")
    ro, ho = b["read_off"], b["hap_off"]
    haps = [b["hap_bases"][ho[h]:ho[h + 1]] for h in range(len(ho) - 1)]
    for r in range(0, 64, 9):
        read = b["read_bases"][ro[r]:ro[r + 1]]
        best = 0.0
        for hap in haps:
            for off in range(len(hap) - len(read) + 1):
                best = max(best, float(np.mean(hap[off:off + len(read)] == read)))
        assert best > 0.6, (r, best)


def test_c3_float_quals_and_size():
    b = synth.make("c3_grad")
    rl, hl = lengths(b)
    assert len(b["pair_read"]) == 100_000
    assert np.all(rl == 150) and np.all(hl == 300)
    assert synth.cells(b) == 4_500_000_000
    assert np.asarray(b["base_q"]).dtype == np.float32


def test_c2_stress_lengths_low_quality_runs_and_N():
    b = synth.make("c2_stress")
    rl, hl = lengths(b)
    assert len(b["pair_read"]) == 50_000
    assert rl.min() >= 250 and rl.max() <= 500 and hl.min() >= 500 and hl.max() <= 1500
    bq = np.asarray(b["base_q"])
    assert (bq <= 6).any() and bq.max() <= 40
    assert (np.asarray(b["read_bases"]) == ord("N")).any()


@pytest.mark.parametrize("name, pairs, cells, mr, nr", [
    ("c1_batched", 2_009_144, 100_498_586_203, (50, 250), (100, 600)),
    ("c4_persistent", 4_194_304, 298_596_557_711, (36, 300), (64, 2048)),
    ("na12878_like", 5_610_137, 52_553_929_341, (10, 151), (30, 521)),
])
def test_large_workloads_exact_sizes(name, pairs, cells, mr, nr):
    b = synth.make(name)
    rl, hl = lengths(b)
    assert len(b["pair_read"]) == pairs
    assert synth.cells(b) == cells
    assert rl.min() >= mr[0] and rl.max() <= mr[1]
    assert hl.min() >= nr[0] and hl.max() <= nr[1]
    # pairs are listed read by read (what the host pipeline's fast path relies on)
    assert np.all(np.diff(b["pair_read"]) >= 0)


def test_generators_are_seeded():
    for name in ("c0_plain", "c3_grad"):
        a, b = synth.make(name), synth.make(name)
        for k in ("read_bases", "base_q", "ins_q", "del_q", "read_off", "hap_bases", "hap_off",
                  "pair_read", "pair_hap"):
            assert np.array_equal(np.asarray(a[k]), np.asarray(b[k])), (name, k)
