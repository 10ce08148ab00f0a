"""phmm_score_host: a batch in host memory scored end to end in pipelined subsets."""
import numpy as np
import pytest

import oracle
from paper_2411_11547_gb300 import synth
from test_gpu_forward import check

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def phmm():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2411_11547_gb300 import _build, phmm as ph
    _build.build()
    ph.lib()
    return ph


@pytest.mark.parametrize("subset_cells", [1, 200_000, 1 << 40])
def test_host_subsets_match_oracle_and_device_path(phmm, subset_cells):
    # one read per subset, a few hundred subsets, and the whole batch in one subset
    b = synth.c1_batched(regions=5)
    got, flags = phmm.score_host(b, subset_cells=subset_cells)
    check(got, flags, oracle.forward_batch(b), phmm)
    dev, dflags = phmm.forward(b)
    # the same groups score each pair whatever the subset: results are identical
    assert np.array_equal(got, dev.cpu().numpy())
    assert np.array_equal(flags, dflags.cpu().numpy())


def test_host_pipeline_float_quals_long_reads_and_plain_tier(phmm):
    b = synth.random_pairs(17, 300, (1, 700), (1, 800), related=0.5, qual_dtype=np.float32)
    got, flags = phmm.score_host(b, phmm.options(first_line=0), subset_cells=3_000_000)
    check(got, flags, oracle.forward_batch(b), phmm)


def test_host_pipeline_unsorted_pairs(phmm):
    # pairs in random order and haplotypes shared across distant reads: the general path
    # (counting sort by read, haplotypes gathered one by one, results scattered)
    b = synth.c1_batched(regions=4)
    perm = np.random.default_rng(3).permutation(len(b["pair_read"]))
    b = dict(b, pair_read=b["pair_read"][perm].copy(), pair_hap=b["pair_hap"][perm].copy())
    b["pair_hap"][::7] = b["pair_hap"][::7][::-1]  # some pairs meet far-away haplotypes
    for sc in (1, 5_000_000):
        got, flags = phmm.score_host(b, subset_cells=sc)
        dev, dflags = phmm.forward(b)
        assert np.array_equal(got, dev.cpu().numpy())
        assert np.array_equal(flags, dflags.cpu().numpy())


def test_host_pipeline_buffers_are_reused_then_released(phmm):
    b = synth.random_pairs(5, 50, (10, 120), (20, 200), related=0.5)
    r1 = phmm.score_host(b, subset_cells=20_000)
    r2 = phmm.score_host(b, subset_cells=20_000)  # cached buffers
    phmm.lib().phmm_score_host_release()
    r3 = phmm.score_host(b, subset_cells=20_000)  # fresh buffers
    for x in (r2, r3):
        assert np.array_equal(r1[0], x[0]) and np.array_equal(r1[1], x[1])
    phmm.lib().phmm_score_host_release()
