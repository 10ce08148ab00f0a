"""Per-base gap-continuation track (eps_i and beta_i per read position) on the GPU, through the
C ABI, against the FP64 oracle: forward log10 L, the adjoint's per-position gradients
(including d/dgcp_i) in the two-call and the fused paths, the FP64 adjoint, row tiles of
long reads, the autograd Function and the host pipeline.  Bars as in the other parity tests.
"""
import numpy as np
import pytest

import oracle
from paper_2411_11547_gb300 import synth

from test_gpu_backward import RTOL, grad_close
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


def with_track(b, seed, lo=3.0, hi=30.0):
    """The batch with a per-base gap-continuation track drawn uniformly in [lo, hi] (Phred),
    in the batch's quality dtype."""
    rng = np.random.default_rng(seed)
    sm = int(b["read_off"][-1])
    qd = np.asarray(b["base_q"]).dtype
    if qd == np.float32:
        gq = rng.uniform(lo, hi, sm).astype(np.float32)
    else:
        gq = rng.integers(int(lo), int(hi) + 1, sm).astype(np.uint8)
    return dict(b, gcp_q=gq)


def run_grad(ph, b, dy, fused, **opt):
    import torch
    plan = ph.Plan(ph.DeviceBatch(b), ph.options(**opt))
    y, fl = plan.forward_partials() if fused else plan.forward()
    res = (plan.backward_partials if fused else plan.backward)(
        torch.as_tensor(dy, dtype=torch.float64, device="cuda"))
    torch.cuda.synchronize()
    assert len(res) == 5  # d_gcp_q returned for a batch with a track
    gb, gi, gd, gg, gq = (x.cpu().numpy() for x in res)
    return y.cpu().numpy(), fl.cpu().numpy(), gb, gi, gd, float(gg[0]), gq, plan


def check_grad(ph, b, dy, **opt):
    wy, wb, wi, wd, wq = oracle.backward_batch(b, dy)
    assert np.asarray(wq).shape == (int(b["read_off"][-1]),)
    ro = b["read_off"]
    for fused in (False, True):
        y, fl, gb, gi, gd, gg, gq, _ = run_grad(ph, b, dy, fused, **opt)
        assert np.all(np.abs(y - wy) <= 1e-3), (fused, np.abs(y - wy).max())
        grad_close(gb, wb, f"d/dbq fused={fused}", ro)
        grad_close(gi, wi, f"d/diq fused={fused}", ro)
        grad_close(gd, wd, f"d/ddq fused={fused}", ro)
        grad_close(gq, wq, f"d/dgcp_q fused={fused}", ro)
        # the scalar d/dgcp of a batch with a track is the sum over every position
        assert abs(gg - wq.sum()) <= RTOL * np.abs(wq).sum() + 1e-9, (fused, gg, wq.sum())


@pytest.mark.parametrize("qual_dtype", [np.float32, np.uint8])
def test_forward_with_track(phmm, qual_dtype):
    # read lengths across every group of the track's table (16x4 .. 32x16)
    b = with_track(synth.random_pairs(201, 300, (1, 512), (1, 600), alphabet=b"ACGTN",
                                      related=0.5, qual_dtype=qual_dtype), 5)
    import torch
    plan = phmm.Plan(phmm.DeviceBatch(b))
    out, fl = plan.forward()
    torch.cuda.synchronize()
    check(out.cpu().numpy(), fl.cpu().numpy(), oracle.forward_batch(b), phmm)
    # the track changes the result (it is not ignored)
    assert np.max(np.abs(out.cpu().numpy() - oracle.forward_batch(
        dict(b, gcp_q=None)))) > 1e-2


def test_uniform_track_matches_the_scalar_path(phmm):
    import torch
    b = synth.random_pairs(202, 120, (1, 400), (1, 500), related=0.6, qual_dtype=np.float32)
    sm = int(b["read_off"][-1])
    bt = dict(b, gcp_q=np.full(sm, b["gcp"], dtype=np.float32))
    dy = np.random.default_rng(2).uniform(-1, 1, len(b["pair_read"]))
    dyt = torch.as_tensor(dy, device="cuda")
    p0 = phmm.Plan(phmm.DeviceBatch(b))
    y0, _ = p0.forward_partials()
    g0 = [x.cpu().numpy() for x in p0.backward_partials(dyt)]
    p1 = phmm.Plan(phmm.DeviceBatch(bt))
    y1, _ = p1.forward_partials()
    g1 = [x.cpu().numpy() for x in p1.backward_partials(dyt)]
    assert np.max(np.abs(y0.cpu().numpy() - y1.cpu().numpy())) <= 2e-5
    for a, c in zip(g0[:3], g1[:3]):
        np.testing.assert_allclose(a, c, rtol=1e-4, atol=1e-4 * np.abs(a).max())
    assert abs(float(g0[3][0]) - float(g1[3][0])) <= 1e-4 * abs(float(g0[3][0]))
    assert abs(float(g1[4].astype(np.float64).sum()) - float(g1[3][0])) <= 1e-4 * abs(float(g1[3][0]))


@pytest.mark.parametrize("seed", [0, 1])
def test_adjoint_with_track(phmm, seed):
    b = with_track(synth.random_pairs(210 + seed, 150, (1, 512), (1, 500), alphabet=b"ACGTN",
                                      related=0.5, qual_dtype=np.float32), 11 + seed)
    dy = np.random.default_rng(seed).uniform(-1.5, 2.0, len(b["pair_read"]))
    check_grad(phmm, b, dy)


def test_adjoint_with_track_shared_reads(phmm):
    # C3-shaped regions: every read in 16 pairs, per-read sums of the per-base gradients
    b = with_track(synth.c3_grad(pairs=16 * 64 * 2), 13)
    check_grad(phmm, b, np.ones(len(b["pair_read"])))


def test_adjoint_with_track_in_fp64(phmm):
    b = with_track(synth.random_pairs(220, 60, (1, 500), (1, 400), related=0.6,
                                      qual_dtype=np.float32), 17)
    dy = np.random.default_rng(5).uniform(-1, 1, len(b["pair_read"]))
    wy, wb, wi, wd, wq = oracle.backward_batch(b, dy)
    y, fl, gb, gi, gd, gg, gq, plan = run_grad(phmm, b, dy, True, adjoint_rescue=2)
    assert plan.rescue_counts()[2] == len(dy)
    assert np.all(np.abs(y - wy) <= 1e-9)
    ro = b["read_off"]
    for got, want, name in ((gb, wb, "bq"), (gi, wi, "iq"), (gd, wd, "dq"), (gq, wq, "gq")):
        grad_close(got, want, name, ro)


def test_long_reads_with_track(phmm):
    rng = np.random.default_rng(41)
    regs = []
    for m, n in [(700, 800), (1030, 1100), (600, 300)]:
        hap = synth.ACGT[rng.integers(0, 4, n)]
        if n >= m:
            o = int(rng.integers(0, n - m + 1))
            read = hap[o:o + m].copy()
        else:
            read = synth.ACGT[rng.integers(0, 4, m)]
        regs.append(([hap], [read], [rng.integers(10, 41, m)], [rng.integers(30, 46, m)],
                     [rng.integers(30, 46, m)]))
    b = with_track(synth._assemble(regs, 10.0, "long", qual_dtype=np.float32), 19)
    check_grad(phmm, b, np.random.default_rng(6).uniform(-1, 1, len(b["pair_read"])))


def test_autograd_with_per_base_gcp(phmm):
    import torch
    from paper_2411_11547_gb300.autograd import PairHMMLogLik, layout_from_host
    b = with_track(synth.random_pairs(230, 80, (1, 250), (1, 400), related=0.6,
                                      qual_dtype=np.float32), 23)
    w = np.random.default_rng(4).normal(size=len(b["pair_read"]))
    layout, (bq, iq, dq) = layout_from_host(b)
    gcp = torch.as_tensor(b["gcp_q"], device="cuda").requires_grad_(True)
    for t in (bq, iq, dq):
        t.requires_grad_(True)
    y, _ = PairHMMLogLik.apply(bq, iq, dq, gcp, layout)
    (y * torch.as_tensor(w, device=y.device)).sum().backward()
    wy, wb, wi, wd, wq = oracle.backward_batch(b, w)
    assert np.all(np.abs(y.detach().cpu().numpy() - wy) <= 1e-3)
    ro = b["read_off"]
    grad_close(gcp.grad.cpu().numpy(), wq, "d/dgcp_q", ro)
    grad_close(bq.grad.cpu().numpy(), wb, "d/dbq", ro)


def test_host_pipeline_with_track(phmm):
    import torch
    b = with_track(synth.c1_batched(regions=3), 29)
    b = dict(b, base_q=b["base_q"].astype(np.float32), ins_q=b["ins_q"].astype(np.float32),
             del_q=b["del_q"].astype(np.float32), gcp_q=b["gcp_q"].astype(np.float32))
    dL = np.random.default_rng(8).uniform(-1, 1, len(b["pair_read"]))
    y, fl, gb, gi, gd, gg, gq = phmm.grad_host(b, dL, subset_cells=200_000)
    plan = phmm.Plan(phmm.DeviceBatch(b))
    yd, fd = plan.forward_partials()
    ref = [x.cpu().numpy() for x in plan.backward_partials(torch.as_tensor(dL, device="cuda"))]
    assert np.array_equal(y, yd.cpu().numpy()) and np.array_equal(fl, fd.cpu().numpy())
    for got, want in zip((gb, gi, gd, gq), (ref[0], ref[1], ref[2], ref[4])):
        assert np.array_equal(got, want)
    wy, wb, wi, wd, wq = oracle.backward_batch(b, dL)
    grad_close(gq, wq, "d/dgcp_q", b["read_off"])
    phmm.lib().phmm_score_host_release()


def test_track_rejections(phmm):
    b = with_track(synth.random_pairs(240, 4, (5, 10), (5, 10), qual_dtype=np.float32), 31)
    with pytest.raises(phmm.PhmmError) as e:  # the plain FP32 first line has no track kernels
        phmm.Plan(phmm.DeviceBatch(b), phmm.options(first_line=phmm.FIRST_PLAIN32))
    assert e.value.status == phmm.PHMM_EINVAL
    bad = dict(b, gcp_q=b["gcp_q"].copy())
    bad["gcp_q"][3] = 0.0  # eps = 1: no gap continuation probability below 1
    with pytest.raises(phmm.PhmmError) as e:
        phmm.Plan(phmm.DeviceBatch(bad))
    assert e.value.status == phmm.PHMM_EINVAL
    # the allocation-free entry point takes the scalar gap continuation only
    import ctypes
    import torch
    db = phmm.DeviceBatch(b)
    out = torch.empty(4, dtype=torch.float64, device="cuda")
    fl = torch.empty(4, dtype=torch.uint8, device="cuda")
    L = phmm.lib()
    L.phmm_forward_noalloc.argtypes = [ctypes.POINTER(phmm.Batch), ctypes.c_void_p,
                                       ctypes.c_void_p, ctypes.c_void_p]
    s = db.struct()
    assert L.phmm_forward_noalloc(ctypes.byref(s), out.data_ptr(), fl.data_ptr(),
                                  None) == phmm.PHMM_EINVAL
