"""GPU adjoint vs the FP64 oracle adjoint, through the C ABI.

Bar: gradients within 1e-3 relative.  An element whose reference is tiny compared with the
rest of ITS READ is compared with an absolute floor of 1e-4 x the largest |reference| of the
same track over the same read.  The floor follows from the arithmetic: each element is a
difference of sums of posterior-scale products (e.g. d/dbq = 0.1 (A1 Q/(1-Q) - A2) with
A1 + A2 the M occupancy of the row), and the FP32 forward and adjoint values behind those
products carry relative errors that grow with the columns swept, up to about n 2^-24
(2e-5 at n = 300; 1.2e-5 of the read's largest element was measured on a 3-row read).  An
element that nearly cancels keeps that error in absolute terms, so it cannot meet a
relative bar; the floor is five times the measured error.
"""
import numpy as np
import pytest

import oracle
from paper_2411_11547_gb300 import synth

pytestmark = pytest.mark.gpu

RTOL, FLOOR = 1e-3, 1e-4


@pytest.fixture(scope="module")
def phmm():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2411_11547_gb300 import _build, phmm as ph
    _build.build()
    ph.lib()
    return ph


def read_floor(want, read_off):
    """FLOOR x max |want| over each element's own read (read_off: that read's offsets into
    `want`)."""
    a = np.abs(np.asarray(want, dtype=np.float64))
    ro = np.asarray(read_off, dtype=np.int64)
    lens = np.diff(ro)
    keep = lens > 0
    mx = np.zeros(len(lens))
    mx[keep] = np.maximum.reduceat(a, ro[:-1][keep])
    return FLOOR * np.maximum(np.repeat(mx, lens), 1e-300)


def grad_close(got, want, name, read_off):
    got = np.asarray(got, dtype=np.float64)
    want = np.asarray(want, dtype=np.float64)
    assert np.all(np.isfinite(got)), f"{name}: non-finite"
    tol = RTOL * np.abs(want) + read_floor(want, read_off)
    bad = np.abs(got - want) > tol
    if bad.any():
        i = np.argmax(np.abs(got - want) - tol)
        raise AssertionError(f"{name}: {bad.sum()} of {bad.size} outside tolerance; worst at {i}:"
                             f" got {got[i]:.6g} want {want[i]:.6g}")


def run_grad(ph, batch, dy, fused=False, **opt):
    """log10 L, gradients and flags through phmm_forward + phmm_backward, or (fused) through
    phmm_forward_partials + phmm_backward_partials."""
    import torch
    plan = ph.Plan(ph.DeviceBatch(batch), ph.options(**opt))
    out, flags = plan.forward_partials() if fused else plan.forward()
    dyt = torch.as_tensor(dy, dtype=torch.float64, device="cuda")
    gb, gi, gd, gg = plan.backward_partials(dyt) if fused else plan.backward(dyt)
    torch.cuda.synchronize()
    return (out.cpu().numpy(), gb.cpu().numpy(), gi.cpu().numpy(), gd.cpu().numpy(),
            float(gg.cpu().numpy()[0]), plan, flags.cpu().numpy())


def check_against_oracle(ph, b, dy, **opt):
    """Both the two-call path and the fused path against the oracle's log10 L (1e-3) and
    adjoint (1e-3 relative)."""
    wy, wb, wi, wd, wg = oracle.backward_batch(b, dy)
    for fused in (False, True):
        y, gb, gi, gd, gg, plan, fl = run_grad(ph, b, dy, fused=fused, **opt)
        assert np.all(np.abs(y - wy) <= 1e-3), (fused, np.abs(y - wy).max())
        if fused:
            ext = (fl & ph.FLAG_EXTENDED) != 0
            one = ((fl & ph.FLAG_FP32) != 0) ^ ((fl & ph.FLAG_RESCUED64) != 0)
            assert np.all(ext & one & ((fl & ph.FLAG_INVALID) == 0)), np.unique(fl)
        ro = b["read_off"]
        grad_close(gb, wb, f"d/dbq fused={fused}", ro)
        grad_close(gi, wi, f"d/diq fused={fused}", ro)
        grad_close(gd, wd, f"d/ddq fused={fused}", ro)
        assert abs(gg - wg) <= RTOL * abs(wg) + 1e-9, (fused, gg, wg)


@pytest.mark.parametrize("seed", [0, 1])
def test_random_pairs(phmm, seed):
    b = synth.random_pairs(60 + seed, 150, (1, 300), (1, 500), alphabet=b"ACGTN", related=0.5,
                           qual_dtype=np.float32)
    dy = np.random.default_rng(seed).uniform(-1.5, 2.0, len(b["pair_read"]))
    check_against_oracle(phmm, b, dy)


def test_shared_reads_all_vs_all(phmm):
    # C3-shaped: regions of 16 haplotypes x 64 reads (here 3 regions), reads shared by pairs
    b = synth.c3_grad(pairs=16 * 64 * 2 + 16 * 5)
    dy = np.ones(len(b["pair_read"]))
    check_against_oracle(phmm, b, dy)


def test_alpha_mode_and_u8_quals(phmm):
    b = synth.random_pairs(77, 80, (5, 200), (5, 300), related=0.6)
    for am in (0, 1):
        bb = dict(b, alpha_mode=am)
        dy = np.linspace(-1, 1, len(b["pair_read"]))
        check_against_oracle(phmm, bb, dy)


def test_every_backward_group(phmm):
    # read lengths that land in each backward group (rows per lane 4/8/12/16)
    rng = np.random.default_rng(5)
    regs = []
    for m in [3, 16, 17, 32, 40, 48, 60, 64, 90, 96, 120, 128, 150, 192, 200, 256, 300, 384, 400,
              512]:
        n = int(rng.integers(max(m, 20), m + 200))
        hap = synth.ACGT[rng.integers(0, 4, n)]
        read = hap[:m].copy()
        regs.append(([hap], [read], [rng.integers(10, 41, m)], [rng.integers(30, 46, m)],
                     [rng.integers(30, 46, m)]))
        regs.append(([synth.ACGT[rng.integers(0, 4, n)]], [read], [rng.integers(10, 41, m)],
                     [rng.integers(30, 46, m)], [rng.integers(30, 46, m)]))
    b = synth._assemble(regs, 10.0, "groups", qual_dtype=np.float32)
    dy = np.ones(len(b["pair_read"]))
    check_against_oracle(phmm, b, dy)


def test_backward_requires_forward(phmm):
    import torch
    b = synth.random_pairs(1, 4, (5, 10), (5, 10))
    plan = phmm.Plan(phmm.DeviceBatch(b))
    with pytest.raises(phmm.PhmmError) as e:
        plan.backward(torch.ones(4, dtype=torch.float64, device="cuda"))
    assert e.value.status == phmm.PHMM_ESTATE
    # the fused reduction needs the fused forward's partials, and phmm_backward replaces them
    with pytest.raises(phmm.PhmmError) as e:
        plan.backward_partials(torch.ones(4, dtype=torch.float64, device="cuda"))
    assert e.value.status == phmm.PHMM_ESTATE
    plan.forward_partials()
    plan.backward_partials(torch.ones(4, dtype=torch.float64, device="cuda"))
    plan.backward(torch.ones(4, dtype=torch.float64, device="cuda"))
    with pytest.raises(phmm.PhmmError) as e:
        plan.backward_partials(torch.ones(4, dtype=torch.float64, device="cuda"))
    assert e.value.status == phmm.PHMM_ESTATE


def test_fused_partials_are_linear_in_dL(phmm):
    """The fused reduction weights fixed per-pair partials: gradients for dL1, dL2 and
    dL1 + 3 dL2 from one phmm_forward_partials satisfy g(dL1 + 3 dL2) = g(dL1) + 3 g(dL2) up
    to the final FP32 rounding, and equal the two-call path's for the same dL."""
    import torch
    b = synth.random_pairs(17, 90, (10, 200), (10, 300), related=0.5, qual_dtype=np.float32)
    P = len(b["pair_read"])
    rng = np.random.default_rng(3)
    d1 = torch.as_tensor(rng.uniform(-1, 1, P), device="cuda")
    d2 = torch.as_tensor(rng.uniform(-1, 1, P), device="cuda")
    plan = phmm.Plan(phmm.DeviceBatch(b))
    plan.forward_partials()
    g1 = [x.double().cpu().numpy() for x in plan.backward_partials(d1)]
    g2 = [x.double().cpu().numpy() for x in plan.backward_partials(d2)]
    g3 = [x.double().cpu().numpy() for x in plan.backward_partials(d1 + 3 * d2)]
    for a, c, s3 in zip(g1, g2, g3):
        lin = a + 3 * c
        assert np.allclose(s3, lin, rtol=1e-5, atol=1e-6 * np.abs(lin).max()), np.abs(s3 - lin).max()
    two = phmm.Plan(phmm.DeviceBatch(b))
    two.forward()
    h = [x.double().cpu().numpy() for x in two.backward(d1 + 3 * d2)]
    for a, c in zip(h, g3):
        assert np.allclose(a, c, rtol=1e-5, atol=1e-6 * np.abs(a).max()), np.abs(a - c).max()


def test_backward_deterministic(phmm):
    import torch
    b = synth.c1_batched(regions=6)
    b = dict(b, base_q=b["base_q"].astype(np.float32), ins_q=b["ins_q"].astype(np.float32),
             del_q=b["del_q"].astype(np.float32))
    dy = np.random.default_rng(2).normal(size=len(b["pair_read"]))
    for fused in (False, True):
        r1 = run_grad(phmm, b, dy, fused=fused)
        r2 = run_grad(phmm, b, dy, fused=fused)
        for x, y in zip(r1[:5], r2[:5]):
            assert np.array_equal(np.asarray(x), np.asarray(y))


def test_reads_much_longer_than_haplotypes(phmm):
    # m >> n forces long insertion runs: forward and adjoint mass sit in disjoint cells of a
    # lane, beyond what one FP32 exponent per lane spans; such pairs are finished in FP64
    rng = np.random.default_rng(9)
    regs = []
    for m, n in [(261, 37), (300, 64), (200, 30), (120, 20), (500, 90), (64, 8)]:
        hap = synth.ACGT[rng.integers(0, 4, n)]
        read = synth.ACGT[rng.integers(0, 4, m)]
        regs.append(([hap], [read], [rng.integers(10, 41, m)], [rng.integers(30, 46, m)],
                     [rng.integers(30, 46, m)]))
    b = synth._assemble(regs, 10.0, "long_reads", qual_dtype=np.float32)
    check_against_oracle(phmm, b, np.ones(len(b["pair_read"])))


def test_autograd_function(phmm):
    import torch
    from paper_2411_11547_gb300.autograd import PairHMMLogLik, layout_from_host
    b = synth.random_pairs(91, 120, (1, 250), (1, 400), related=0.6, qual_dtype=np.float32)
    w = np.random.default_rng(4).normal(size=len(b["pair_read"]))
    layout, (bq, iq, dq) = layout_from_host(b)
    for t in (bq, iq, dq):
        t.requires_grad_(True)
    gcp = torch.tensor(float(b["gcp"]), dtype=torch.float64, requires_grad=True)
    y, flags = PairHMMLogLik.apply(bq, iq, dq, gcp, layout)
    loss = (y * torch.as_tensor(w, device=y.device)).sum()
    loss.backward()
    wy, wb, wi, wd, wg = oracle.backward_batch(b, w)
    assert np.all(np.abs(y.detach().cpu().numpy() - wy) <= 1e-3)
    assert flags.dtype == torch.uint8 and not flags.requires_grad
    ro = b["read_off"]
    grad_close(bq.grad.cpu().numpy(), wb, "d/dbq", ro)
    grad_close(iq.grad.cpu().numpy(), wi, "d/diq", ro)
    grad_close(dq.grad.cpu().numpy(), wd, "d/ddq", ro)
    assert abs(float(gcp.grad) - wg) <= RTOL * abs(wg) + 1e-9


BWD_SHAPES = ([(L, K) for L in (4, 8, 16, 32) for K in (4, 6, 8, 10, 12)] + [(16, 14), (32, 16)]
              + [(4, 9), (4, 11), (8, 7), (8, 9), (8, 11), (16, 7), (16, 9), (16, 11), (16, 13),
                 (32, 7), (32, 9)])


@pytest.mark.parametrize("L,K", BWD_SHAPES)
def test_every_backward_shape(phmm, L, K):
    # every built adjoint group, forced by a backward table; reads from 1 row up to capacity
    import torch
    cap = L * K
    b = synth.random_pairs(300 + cap + K, 24, (max(1, cap // 3), cap), (1, 260), related=0.6,
                           qual_dtype=np.float32)
    assert np.diff(b["read_off"]).max() <= cap
    c = phmm.cfg_index(L, K)
    dy = np.random.default_rng(cap).uniform(-1, 1, len(b["pair_read"]))
    check_against_oracle(phmm, b, dy, bwd_rows=[c] * 129)


def test_c4_adjoint_full_size_sampled_regions(phmm):
    """The adjoint of the full 2^22-pair batch in the bench's launch configuration (autotuned
    forward and adjoint tables); the per-read gradients of 40 sampled regions (every pair of
    those reads, 2,560 pairs) are compared with the oracle's adjoint of those regions."""
    import torch
    b = synth.c4_persistent()
    db = phmm.DeviceBatch(b)
    o = phmm.autotune(db, which=3)
    plan = phmm.Plan(db, o)
    plan.forward()
    P = len(b["pair_read"])
    dy = np.random.default_rng(12).uniform(-1, 1, P)
    gb, gi, gd, gg = plan.backward(torch.as_tensor(dy, device="cuda"))
    gb, gi, gd = gb.cpu().numpy(), gi.cpu().numpy(), gd.cpu().numpy()
    # regions hold reads 16 r .. 16 r + 15; every pair of a sampled read is taken
    regions = np.random.default_rng(13).choice(65536, 40, replace=False)
    reads = np.sort(np.concatenate([np.arange(16 * r, 16 * r + 16) for r in regions]))
    pairs = np.nonzero(np.isin(b["pair_read"], reads))[0]
    assert len(pairs) == 40 * 64
    sb = synth.subset_pairs(b, pairs)
    # the oracle over the sampled pairs only: the sampled reads' gradients are complete there
    wy, wb, wi, wd, wg = oracle.backward_batch(sb, dy[pairs])
    ro = b["read_off"]
    idx = np.concatenate([np.arange(ro[r], ro[r + 1]) for r in reads])
    sro = np.concatenate([[0], np.cumsum(ro[reads + 1] - ro[reads])])
    grad_close(gb[idx], wb[idx], "d/dbq", sro)
    grad_close(gi[idx], wi[idx], "d/diq", sro)
    grad_close(gd[idx], wd[idx], "d/ddq", sro)
    # the fused step on the same plan: log10 L of the sampled pairs and the same gradients
    y, _ = plan.forward_partials()
    fb, fi, fd, fg = plan.backward_partials(torch.as_tensor(dy, device="cuda"))
    assert np.all(np.abs(y.cpu().numpy()[pairs] - wy) <= 1e-3)
    grad_close(fb.cpu().numpy()[idx], wb[idx], "fused d/dbq", sro)
    grad_close(fi.cpu().numpy()[idx], wi[idx], "fused d/diq", sro)
    grad_close(fd.cpu().numpy()[idx], wd[idx], "fused d/ddq", sro)


def test_fused_step_empty_batch(phmm):
    import torch
    # no pairs: log10 L is empty, every gradient is 0
    b = synth.random_pairs(2, 3, (5, 10), (5, 10), qual_dtype=np.float32)
    b = dict(b, pair_read=b["pair_read"][:0], pair_hap=b["pair_hap"][:0])
    plan = phmm.Plan(phmm.DeviceBatch(b))
    y, fl = plan.forward_partials()
    gb, gi, gd, gg = plan.backward_partials(torch.zeros(0, dtype=torch.float64, device="cuda"))
    assert y.shape == (0,) and fl.shape == (0,)
    for g in (gb, gi, gd):
        assert not g.cpu().numpy().any()
    assert float(gg.cpu()[0]) == 0.0


@pytest.mark.parametrize("fused", [False, True])
def test_every_pair_in_fp64(phmm, fused):
    """adjoint_rescue = 2 sends every pair to the FP64 adjoint (32 lanes x 4 / 8 / 16 rows, by
    read length): the FP64 kernels that otherwise run only on hand-offs, against the oracle;
    the fused call's log10 L then comes from FP64 too (the rescued-pair bar, 1e-9)."""
    b = synth.random_pairs(44, 60, (1, 500), (1, 400), related=0.6, qual_dtype=np.float32)
    rl = np.diff(b["read_off"])[b["pair_read"]]
    assert (rl <= 128).any() and ((rl > 128) & (rl <= 256)).any() and (rl > 256).any()
    P = len(b["pair_read"])
    dy = np.random.default_rng(5).uniform(-1, 1, P)
    wy, wb, wi, wd, wg = oracle.backward_batch(b, dy)
    y, gb, gi, gd, gg, plan, fl = run_grad(phmm, b, dy, fused=fused, adjoint_rescue=2)
    assert plan.rescue_counts()[2] == P
    if fused:
        assert np.all(fl == (phmm.FLAG_RESCUED64 | phmm.FLAG_EXTENDED))
        assert np.all(np.abs(y - wy) <= 1e-9)
    ro = b["read_off"]
    grad_close(gb, wb, "d/dbq", ro)
    grad_close(gi, wi, "d/diq", ro)
    grad_close(gd, wd, "d/ddq", ro)
    assert abs(gg - wg) <= 1e-6 * abs(wg) + 1e-9, (gg, wg)


def test_fused_step_graph_replay(phmm):
    """On a small batch the fused step's two calls replay captured CUDA graphs: results equal
    the eager launches bit for bit, replays repeat them, new output pointers recapture, and
    the launch count is reported either way."""
    import torch
    b = synth.c3_grad(pairs=16 * 64)  # one C0-shaped region, 1,024 pairs
    P = len(b["pair_read"])
    dy = torch.as_tensor(np.random.default_rng(4).uniform(-1, 1, P), device="cuda")
    res = {}
    for g in (0, 1):
        plan = phmm.Plan(phmm.DeviceBatch(b), phmm.options(use_graph=g))
        y = torch.empty(P, dtype=torch.float64, device="cuda")
        fl = torch.empty(P, dtype=torch.uint8, device="cuda")
        sm = int(b["read_off"][-1])
        gout = tuple(torch.empty(sm, dtype=torch.float32, device="cuda") for _ in range(3)) + (
            torch.empty(1, dtype=torch.float64, device="cuda"),)
        outs = []
        for _ in range(3):  # the 2nd call repeats the pointers (capture), the 3rd replays
            plan.forward_partials(y, fl)
            gr = plan.backward_partials(dy, out=gout)
            torch.cuda.synchronize()
            outs.append([y.cpu().numpy(), fl.cpu().numpy()] + [x.cpu().numpy() for x in gr])
            assert plan.launch_count(0) > 10 and plan.launch_count(1) > 3
        assert plan.backward_ms()[0] == (-1.0 if g else plan.backward_ms()[0])
        for o in outs[1:]:
            for u, v in zip(outs[0], o):
                assert np.array_equal(u, v)
        res[g] = outs[0]
    for u, v in zip(res[0], res[1]):
        assert np.array_equal(u, v)
    wy, wb, wi, wd, wg = oracle.backward_batch(b, dy.cpu().numpy())
    assert np.all(np.abs(res[1][0] - wy) <= 1e-3)
    grad_close(res[1][2], wb, "d/dbq graph", b["read_off"])
