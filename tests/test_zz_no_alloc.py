"""The allocation-free forward entry point (phmm_forward_noalloc) against phmm_forward.

Called through the C ABI twice in a row on different batches; each result must match the
planned entry point's within the FP32 bar (1e-3 in log10).  Runs last so that a failure here
leaves every other test already run.
"""
import ctypes

import numpy as np
import pytest

from paper_2411_11547_gb300 import synth

pytestmark = pytest.mark.gpu

TOL32 = 1e-3


@pytest.fixture(scope="module")
def phmm():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2411_11547_gb300 import _build, phmm as ph
    _build.build()
    L = ph.lib()
    L.phmm_forward_noalloc.argtypes = [ctypes.POINTER(ph.Batch), ctypes.c_void_p,
                                       ctypes.c_void_p, ctypes.c_void_p]
    L.phmm_forward_noalloc.restype = ctypes.c_int
    return ph


def noalloc(ph, db):
    import torch
    P = db.n_pairs
    out = torch.full((P,), float("nan"), dtype=torch.float64, device="cuda")
    flags = torch.zeros(P, dtype=torch.uint8, device="cuda")
    b = db.struct()
    rc = ph.lib().phmm_forward_noalloc(ctypes.byref(b), out.data_ptr(), flags.data_ptr(),
                                       ph._stream())
    torch.cuda.synchronize()
    return rc, out.cpu().numpy(), flags.cpu().numpy()


def test_noalloc_matches_planned_forward_two_calls(phmm):
    batches = [synth.random_pairs(41, 300, (1, 300), (1, 600), alphabet=b"ACGTN", related=0.5),
               synth.c1_batched(regions=4)]
    for b in batches:  # two calls in a row; the second must not see the first's scratch
        db = phmm.DeviceBatch(b)
        rc, got, flags = noalloc(phmm, db)
        assert rc == phmm.PHMM_OK
        want, wflags = phmm.Plan(db).forward()
        want = want.cpu().numpy()
        assert np.all(flags == (phmm.FLAG_FP32 | phmm.FLAG_EXTENDED))
        np.testing.assert_allclose(got, want, rtol=0, atol=TOL32)


def test_noalloc_rejects_batches_beyond_its_scratch(phmm):
    # 5 M read bases need 85 MB of per-position scratch: beyond the static array
    rng = np.random.default_rng(0)
    R, m = 20000, 250
    reads = synth.ACGT[rng.integers(0, 4, R * m)]
    b = {"read_bases": reads, "base_q": np.full(R * m, 30, np.uint8),
         "ins_q": np.full(R * m, 45, np.uint8), "del_q": np.full(R * m, 45, np.uint8),
         "read_off": np.arange(R + 1, dtype=np.int64) * m,
         "hap_bases": synth.ACGT[rng.integers(0, 4, 300)],
         "hap_off": np.array([0, 300], dtype=np.int64),
         "pair_read": np.array([0, 1], dtype=np.int32), "pair_hap": np.zeros(2, np.int32),
         "gcp": 10.0}
    rc, _, _ = noalloc(phmm, phmm.DeviceBatch(b))
    assert rc == phmm.PHMM_ENOMEM
