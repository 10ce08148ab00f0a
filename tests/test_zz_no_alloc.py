"""The allocation-free forward entry point (phmm_forward_noalloc) against phmm_forward.

Some callers cannot allocate device memory (a framework that owns every allocation through
its own pool, a request path where cudaMalloc is not allowed, a plug-in handed only its
buffers); phmm_forward_noalloc keeps its scratch in a static device array instead.  It is
called through the C ABI twice in a row on different batches; each result must match the
planned entry point's within the FP32 bar (1e-3 in log10), and the FP64 oracle's too.  Its
rejections (bad offsets, reads too long, scratch too small) and its per-pair INVALID flag
are checked with host-built inputs that it rejects or flags without any out-of-bounds
access.  Runs last so that a failure here leaves every other test already run.
"""
import ctypes

import numpy as np
import pytest

import oracle
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
        np.testing.assert_allclose(got, oracle.forward_batch(b), rtol=0, atol=TOL32)


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


def _small(rng, m_list, n_list):
    """A batch of one read per length in m_list and one haplotype per length in n_list,
    every read paired with every haplotype."""
    reads = [synth.ACGT[rng.integers(0, 4, m)] for m in m_list]
    haps = [synth.ACGT[rng.integers(0, 4, n)] for n in n_list]
    sm = sum(m_list)
    R, H = len(m_list), len(n_list)
    pr, ph = np.meshgrid(np.arange(R, dtype=np.int32), np.arange(H, dtype=np.int32),
                         indexing="ij")
    return {"read_bases": np.concatenate(reads), "base_q": rng.integers(10, 41, sm).astype(np.uint8),
            "ins_q": np.full(sm, 45, np.uint8), "del_q": np.full(sm, 45, np.uint8),
            "read_off": np.concatenate([[0], np.cumsum(m_list)]).astype(np.int64),
            "hap_bases": np.concatenate(haps),
            "hap_off": np.concatenate([[0], np.cumsum(n_list)]).astype(np.int64),
            "pair_read": pr.ravel(), "pair_hap": ph.ravel(), "gcp": 10.0}


def test_noalloc_rejects_reads_beyond_one_group(phmm):
    b = _small(np.random.default_rng(1), [100, 513], [600])
    rc, _, _ = noalloc(phmm, phmm.DeviceBatch(b))
    assert rc == phmm.PHMM_ETOOLONG


def test_noalloc_batch_without_pairs(phmm):
    b = _small(np.random.default_rng(2), [20, 30], [40])
    b = dict(b, pair_read=b["pair_read"][:0], pair_hap=b["pair_hap"][:0])
    rc, got, _ = noalloc(phmm, phmm.DeviceBatch(b))
    assert rc == phmm.PHMM_OK and got.shape == (0,)


def test_noalloc_flags_out_of_range_pair_ids(phmm):
    b = _small(np.random.default_rng(3), [50, 60], [80, 90])
    ph = b["pair_hap"].copy()
    ph[1] = 2  # == n_haps: out of range
    pr = b["pair_read"].copy()
    pr[2] = -1
    b = dict(b, pair_hap=ph, pair_read=pr)
    rc, got, flags = noalloc(phmm, phmm.DeviceBatch(b))
    assert rc == phmm.PHMM_OK
    assert flags[1] == phmm.FLAG_INVALID and np.isnan(got[1])
    assert flags[2] == phmm.FLAG_INVALID and np.isnan(got[2])
    ok = np.array([0, 3])
    assert np.all(flags[ok] == (phmm.FLAG_FP32 | phmm.FLAG_EXTENDED))
    want = oracle.forward_batch(dict(b, pair_read=b["pair_read"][ok], pair_hap=b["pair_hap"][ok]))
    np.testing.assert_allclose(got[ok], want, rtol=0, atol=TOL32)


@pytest.mark.parametrize("which", ["hap_not_monotone", "read_not_monotone", "hap_start",
                                   "read_start", "empty_read"])
def test_noalloc_rejects_bad_offsets(phmm, which):
    # every offset stays within the arrays' sizes, so even an unchecked call would read and
    # write only inside its buffers and the static scratch
    b = _small(np.random.default_rng(4), [10, 20, 30], [10, 20, 30])
    ro, ho = b["read_off"].copy(), b["hap_off"].copy()   # [0 10 30 60] both
    if which == "hap_not_monotone":
        ho[2] = 5                                         # lengths 10, -5, 55
    elif which == "read_not_monotone":
        ro[2] = 5
    elif which == "hap_start":
        ho[0] = 2
    elif which == "read_start":
        ro[0] = 2
    else:
        ro[2] = ro[1]                                     # an empty read
    rc, _, _ = noalloc(phmm, phmm.DeviceBatch(dict(b, read_off=ro, hap_off=ho)))
    assert rc == phmm.PHMM_EINVAL
    # the same call with the offsets restored succeeds
    rc, got, _ = noalloc(phmm, phmm.DeviceBatch(b))
    assert rc == phmm.PHMM_OK
    np.testing.assert_allclose(got, oracle.forward_batch(b), rtol=0, atol=TOL32)
