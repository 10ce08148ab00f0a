"""Sharding one batch over two ranks (gloo, CPU): every read's pairs stay on one rank, and the
per-read gradients and the one cross-rank sum (d/dgcp) reproduce the unsharded result.  The
per-rank computation is the oracle (CPU); on GPUs each rank runs the library instead."""
import os
import socket

import numpy as np
import pytest

import oracle
from paper_2411_11547_gb300 import shard, synth


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out_dir):
    import torch
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        b = synth.c1_batched(regions=6)
        sub, pairs, (lo, hi) = shard.shard(b, rank, world)
        dy = np.random.default_rng(0).uniform(-1, 1, len(b["pair_read"]))
        y, gb, gi, gd, gg = oracle.backward_batch(sub, dy[pairs], nthreads=2)
        tot = int(b["read_off"][-1])
        P = len(b["pair_read"])
        # place the shard's results in global arrays and sum over ranks
        full = torch.zeros(P + 3 * tot, dtype=torch.float64)
        full[torch.as_tensor(pairs)] = torch.as_tensor(y)
        r0, r1 = int(b["read_off"][lo]), int(b["read_off"][hi])
        full[P + r0:P + r1] = torch.as_tensor(gb)
        full[P + tot + r0:P + tot + r1] = torch.as_tensor(gi)
        full[P + 2 * tot + r0:P + 2 * tot + r1] = torch.as_tensor(gd)
        dist.all_reduce(full)
        dgcp = shard.allreduce_scalar(gg)
        if rank == 0:
            np.save(os.path.join(out_dir, "sharded.npy"), full.numpy())
            np.save(os.path.join(out_dir, "dgcp.npy"), np.array([dgcp]))
    finally:
        dist.destroy_process_group()


def test_partition_keeps_reads_whole_and_balances_cells():
    b = synth.c1_batched(regions=8)
    parts = shard.partition_by_read(b, 3)
    assert parts[0][0] == 0 and parts[-1][1] == len(b["read_off"]) - 1
    assert all(parts[k][1] == parts[k + 1][0] for k in range(2))
    ro, ho = b["read_off"], b["hap_off"]
    pr, ph = b["pair_read"], b["pair_hap"]
    c = (ro[pr + 1] - ro[pr]) * (ho[ph + 1] - ho[ph])
    per = [c[(pr >= lo) & (pr < hi)].sum() for lo, hi in parts]
    assert sum(per) == c.sum()
    assert max(per) <= 1.5 * c.sum() / 3  # balanced to within a region's size
    seen = np.zeros(len(pr), dtype=int)
    for k in range(3):
        sub, pairs, _ = shard.shard(b, k, 3)
        seen[pairs] += 1
        # renumbered pairs point at the same sequences
        i = len(pairs) // 2
        p = pairs[i]
        so, sh = sub["read_off"], sub["hap_off"]
        r, h = sub["pair_read"][i], sub["pair_hap"][i]
        assert np.array_equal(sub["read_bases"][so[r]:so[r + 1]],
                              b["read_bases"][ro[pr[p]]:ro[pr[p] + 1]])
        assert np.array_equal(sub["hap_bases"][sh[h]:sh[h + 1]],
                              b["hap_bases"][ho[ph[p]]:ho[ph[p] + 1]])
    assert np.all(seen == 1)


def test_two_ranks_gloo_match_unsharded(tmp_path):
    import torch.multiprocessing as mp
    port = _free_port()
    mp.start_processes(_worker, args=(2, port, str(tmp_path)), nprocs=2, join=True,
                       start_method="spawn")
    b = synth.c1_batched(regions=6)
    dy = np.random.default_rng(0).uniform(-1, 1, len(b["pair_read"]))
    y, gb, gi, gd, gg = oracle.backward_batch(b, dy, nthreads=2)
    full = np.load(tmp_path / "sharded.npy")
    P, tot = len(y), int(b["read_off"][-1])
    np.testing.assert_allclose(full[:P], y, rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(full[P:P + tot], gb, rtol=1e-10, atol=1e-14)
    np.testing.assert_allclose(full[P + tot:P + 2 * tot], gi, rtol=1e-10, atol=1e-14)
    np.testing.assert_allclose(full[P + 2 * tot:], gd, rtol=1e-10, atol=1e-14)
    assert abs(float(np.load(tmp_path / "dgcp.npy")[0]) - gg) <= 1e-10 * abs(gg)


def _worker_step(rank, world, port, out_dir):
    """The library's orchestration (shard.sharded_step) with the oracle as each rank's compute:
    partition, per-rank step, placement of the results and the d/dgcp sum over ranks."""
    import torch
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        b = synth.c1_batched(regions=7)
        dy = np.random.default_rng(1).uniform(-1, 1, len(b["pair_read"]))
        r = shard.sharded_step(b, dy, rank, world,
                               lambda sub, d: oracle.backward_batch(sub, d, nthreads=2))
        np.savez(os.path.join(out_dir, f"rank{rank}.npz"), pairs=r["pairs"],
                 bases=np.array(r["bases"]), y=r["log10"], gb=r["d_base_q"], gi=r["d_ins_q"],
                 gd=r["d_del_q"], gg=np.array([r["d_gcp"]]))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_sharded_step_orchestration_gloo(tmp_path, world):
    import torch.multiprocessing as mp
    port = _free_port()
    mp.start_processes(_worker_step, args=(world, port, str(tmp_path)), nprocs=world,
                       join=True, start_method="spawn")
    b = synth.c1_batched(regions=7)
    dy = np.random.default_rng(1).uniform(-1, 1, len(b["pair_read"]))
    y, gb, gi, gd, gg = oracle.backward_batch(b, dy, nthreads=2)
    tot = int(b["read_off"][-1])
    got_y = np.full(len(y), np.nan)
    got = [np.full(tot, np.nan) for _ in range(3)]
    for k in range(world):
        r = np.load(tmp_path / f"rank{k}.npz")
        assert np.all(np.isnan(got_y[r["pairs"]]))  # every pair on exactly one rank
        got_y[r["pairs"]] = r["y"]
        b0, b1 = (int(x) for x in r["bases"])
        for arr, part in zip(got, (r["gb"], r["gi"], r["gd"])):
            assert np.all(np.isnan(arr[b0:b1]))  # every read base on exactly one rank
            arr[b0:b1] = part
        # every rank holds the same d/dgcp: the sum over the ranks
        assert abs(float(r["gg"][0]) - gg) <= 1e-10 * abs(gg)
    np.testing.assert_allclose(got_y, y, rtol=1e-12, atol=1e-12)
    for a, want in zip(got, (gb, gi, gd)):
        np.testing.assert_allclose(a, want, rtol=1e-10, atol=1e-14)
