"""Autotuned group tables (phmm_autotune): valid entries, and results unchanged against the
FP64 oracle when the tuned tables are used."""
import numpy as np
import pytest

import oracle
from paper_2411_11547_gb300 import synth
from test_gpu_backward import grad_close, RTOL

pytestmark = pytest.mark.gpu

# adjoint groups with odd rows per lane
ODD_BWD = ((4, 9), (4, 11), (8, 7), (8, 9), (8, 11), (16, 7), (16, 9), (16, 11), (16, 13),
           (32, 7), (32, 9))


@pytest.fixture(scope="module")
def phmm():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2411_11547_gb300 import _build, phmm as ph
    _build.build()
    ph.lib()
    return ph




def test_autotune_tables_and_parity(phmm):
    import torch
    b = synth.random_pairs(123, 400, (1, 320), (1, 400), related=0.5, qual_dtype=np.float32)
    db = phmm.DeviceBatch(b)
    o = phmm.autotune(db, which=3, sample_pairs=48)
    m = np.diff(b["read_off"])
    for tab, built, valid in ((o.bin_rows, None, o.bin_table_valid),
                              (o.bwd_rows, "bwd", o.bwd_table_valid)):
        if not valid:  # no tuned group beat the built-in ones
            continue
        tuned = 0
        for k in range(1, 129):
            c = tab[k]
            if c < 0:
                continue
            L, K = phmm.cfg_shape(c)
            assert L * K >= 4 * k, (k, c)
            if built == "bwd":
                assert K in (4, 6, 8, 10, 12) or (L, K) in ((16, 14), (32, 16)) or \
                    (L, K) in ODD_BWD
            else:
                assert K % 2 == 0  # the forward kernels have even rows per lane
            tuned += 1
        # entries only in 16-row ranges that hold pairs (others keep the built-in groups)
        ranges = set(((m - 1) // 16).tolist())
        assert tuned <= 4 * len(ranges)
        assert all(tab[k] < 0 for k in range(1, 129) if (4 * k - 1) // 16 not in ranges)
    plan = phmm.Plan(db, o)
    out, flags = plan.forward()
    want = oracle.forward_batch(b)
    assert np.max(np.abs(out.cpu().numpy() - want)) <= 1e-3
    dy = np.random.default_rng(1).uniform(-1, 1, len(b["pair_read"]))
    gb, gi, gd, gg = plan.backward(torch.as_tensor(dy, device="cuda"))
    wy, wb, wi, wd, wg = oracle.backward_batch(b, dy)
    grad_close(gb.cpu().numpy(), wb, "d/dbq", b["read_off"])
    grad_close(gi.cpu().numpy(), wi, "d/diq", b["read_off"])
    grad_close(gd.cpu().numpy(), wd, "d/ddq", b["read_off"])
    assert abs(float(gg.cpu()[0]) - wg) <= RTOL * abs(wg) + 1e-9
