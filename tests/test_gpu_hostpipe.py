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


def fused_device(ph, b, dL):
    """The fused step on the whole batch on the device (reference for phmm_grad_host)."""
    import torch
    plan = ph.Plan(ph.DeviceBatch(b))
    y, fl = plan.forward_partials()
    gb, gi, gd, gg = plan.backward_partials(torch.as_tensor(dL, device="cuda"))
    return (y.cpu().numpy(), fl.cpu().numpy(), gb.cpu().numpy(), gi.cpu().numpy(),
            gd.cpu().numpy(), float(gg.cpu().numpy()[0]))


@pytest.mark.parametrize("subset_cells", [1, 300_000, 1 << 40])
def test_grad_host_matches_oracle_and_whole_batch(phmm, subset_cells):
    """Per subset the same groups compute each pair's partials and each read's pairs are
    summed in the same order, so log10 L, flags and the per-read gradients equal the
    whole-batch fused step bit for bit; d/dgcp is summed over subsets (rounding only)."""
    from test_gpu_backward import grad_close
    b = synth.c1_batched(regions=4)
    b = dict(b, base_q=b["base_q"].astype(np.float32), ins_q=b["ins_q"].astype(np.float32),
             del_q=b["del_q"].astype(np.float32))
    dL = np.random.default_rng(8).uniform(-1, 1, len(b["pair_read"]))
    y, fl, gb, gi, gd, gg = phmm.grad_host(b, dL, subset_cells=subset_cells)
    ref = fused_device(phmm, b, dL)
    for got, want in zip((y, fl, gb, gi, gd), ref[:5]):
        assert np.array_equal(got, want)
    assert abs(gg - ref[5]) <= 1e-12 * max(1.0, abs(ref[5]))
    if subset_cells == 300_000:
        wy, wb, wi, wd, wg = oracle.backward_batch(b, dL)
        assert np.all(np.abs(y - wy) <= 1e-3)
        grad_close(gb, wb, "d/dbq", b["read_off"])
        grad_close(gi, wi, "d/diq", b["read_off"])
        grad_close(gd, wd, "d/ddq", b["read_off"])
        assert abs(gg - wg) <= 1e-3 * abs(wg) + 1e-9


def test_grad_host_unsorted_pairs_and_reads_without_pairs(phmm):
    # pairs in random order; the last read has no pair (its gradients are 0); u8 quals
    b = synth.random_pairs(23, 60, (5, 200), (5, 300), related=0.5)
    perm = np.random.default_rng(4).permutation(len(b["pair_read"]))
    keep = perm[perm != np.nonzero(b["pair_read"] == b["pair_read"].max())[0][0]]
    b = dict(b, pair_read=b["pair_read"][keep].copy(), pair_hap=b["pair_hap"][keep].copy())
    dL = np.linspace(-2, 2, len(b["pair_read"]))
    y, fl, gb, gi, gd, gg = phmm.grad_host(b, dL, subset_cells=40_000)
    ref = fused_device(phmm, b, dL)
    for got, want in zip((y, fl, gb, gi, gd), ref[:5]):
        assert np.array_equal(got, want)
    last = slice(int(b["read_off"][-2]), int(b["read_off"][-1]))
    assert not gb[last].any() and not gi[last].any() and not gd[last].any()
    # a subset made only of reads without pairs is skipped (scoring path too)
    for sc in (1, 40_000):
        got, flags = phmm.score_host(b, subset_cells=sc)
        dev, dflags = phmm.forward(b)
        assert np.array_equal(got, dev.cpu().numpy())
        assert np.array_equal(flags, dflags.cpu().numpy())
    phmm.lib().phmm_score_host_release()


def test_grad_host_long_reads_in_row_tiles(phmm):
    """Reads longer than one wavefront group (512 rows) go through the row-tiled adjoint in
    the host pipeline too; gradients against the oracle, and bitwise equal to the device
    fused step."""
    from test_gpu_backward import grad_close
    b = synth.random_pairs(2, 6, (600, 1100), (600, 1200), related=1.0, qual_dtype=np.float32)
    dL = np.random.default_rng(3).uniform(-1, 1, 6)
    y, fl, gb, gi, gd, gg = phmm.grad_host(b, dL, subset_cells=1 << 40)
    ref = fused_device(phmm, b, dL)
    for got, want in zip((y, fl, gb, gi, gd), ref[:5]):
        assert np.array_equal(got, want)
    wy, wb, wi, wd, wg = oracle.backward_batch(b, dL)
    assert np.all(np.abs(y - wy) <= 1e-3)
    grad_close(gb, wb, "d/dbq", b["read_off"])
    grad_close(gi, wi, "d/diq", b["read_off"])
    grad_close(gd, wd, "d/ddq", b["read_off"])
    assert abs(gg - wg) <= 1e-3 * abs(wg) + 1e-9
    phmm.lib().phmm_score_host_release()
