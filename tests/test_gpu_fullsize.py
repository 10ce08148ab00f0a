"""Full-size parity of the workloads C1, C2 and C3 against the FP64 oracle, through the C ABI.

Each batch is launched whole, in the configuration that scores it (binned, autotuned where the
bench tunes, FP64 rescue on), so binning, rescue lists and persistent work queues run at their
real sizes; the oracle then checks a stratified sample: every 16-row read-length range, every
result flag present (all rescued pairs up to a cap), and the largest pairs.  Bars as in the
other parity tests: 1e-3 in log10 L for FP32 results, 1e-9 for FP64-rescued ones, gradients
1e-3 relative with the per-read floor of test_gpu_backward.  The last test compares the GPU
gradient with FP64 central finite differences (h = 1e-4) of the oracle's log10 L on 200
sampled C3 pairs.
"""
import numpy as np
import pytest

import oracle
from paper_2411_11547_gb300 import synth

from test_gpu_backward import grad_close, read_floor
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


def stratified(b, flags, seed, per_bucket=120, per_flag=1000, top=1000):
    """Pair indices: up to per_bucket pairs of every 16-row read-length range, up to per_flag
    pairs of every flag value (all of a rarer one), and the `top` largest pairs (m * n)."""
    rng = np.random.default_rng(seed)
    rl = np.diff(b["read_off"])[b["pair_read"]]
    hl = np.diff(b["hap_off"])[b["pair_hap"]]
    idx = []
    bucket = (rl - 1) // 16
    for k in np.unique(bucket):
        sel = np.nonzero(bucket == k)[0]
        idx.append(rng.choice(sel, min(per_bucket, len(sel)), replace=False))
    for f in np.unique(flags):
        sel = np.nonzero(flags == f)[0]
        idx.append(rng.choice(sel, min(per_flag, len(sel)), replace=False))
    idx.append(np.argsort(rl.astype(np.int64) * hl)[-top:])
    return np.unique(np.concatenate(idx))


def forward_full(ph, b, autotune=False, **opt):
    import torch
    db = ph.DeviceBatch(b)
    o = ph.options(**opt)
    if autotune:
        o = ph.autotune(db, o, which=1)
    plan = ph.Plan(db, o)
    out, fl = plan.forward()
    torch.cuda.synchronize()
    return out.cpu().numpy(), fl.cpu().numpy(), plan


@pytest.mark.parametrize("first_line", [1, 0])
def test_c1_full_size(phmm, first_line):
    """C1: 2,000 regions, ~2.0 M pairs; the default extended-range first line (autotuned
    tables), and the paper's plain FP32 scheme with ~87% of pairs rescued in FP64."""
    b = synth.c1_batched()
    got, flags, plan = forward_full(phmm, b, autotune=first_line == 1, first_line=first_line)
    assert np.all((flags & phmm.FLAG_INVALID) == 0)
    if first_line == 0:
        assert plan.rescue_counts()[0] > len(got) // 2
    idx = stratified(b, flags, 11 + first_line, top=600)
    check(got[idx], flags[idx], oracle.forward_batch(synth.subset_pairs(b, idx)), phmm)


@pytest.mark.parametrize("first_line", [0, 1])
def test_c2_full_size(phmm, first_line):
    """C2: 50,000 long pairs with low-quality runs and N bases; under the plain first line
    most pairs take the FP64 rescue and some the per-lane-exponent FP64 kernels."""
    b = synth.c2_stress()
    got, flags, plan = forward_full(phmm, b, first_line=first_line)
    assert np.all((flags & phmm.FLAG_INVALID) == 0)
    if first_line == 0:
        counts = plan.rescue_counts()
        assert counts[0] > len(got) // 2, counts
    idx = stratified(b, flags, 21 + first_line, top=500)
    check(got[idx], flags[idx], oracle.forward_batch(synth.subset_pairs(b, idx)), phmm)


def test_c3_full_size_fused_step(phmm):
    """C3: the fused training step over all 100,000 pairs (autotuned adjoint tables); log10 L
    of a stratified sample and the per-read gradients of 24 sampled reads (every pair of each,
    from 24 regions, plus the short last region) against the oracle."""
    import torch
    b = synth.c3_grad()
    P = len(b["pair_read"])
    db = phmm.DeviceBatch(b)
    plan = phmm.Plan(db, phmm.autotune(db, which=2))
    dy = np.random.default_rng(31).uniform(-1, 1, P)
    y, fl = plan.forward_partials()
    gb, gi, gd, gg = plan.backward_partials(torch.as_tensor(dy, device="cuda"))
    y, fl = y.cpu().numpy(), fl.cpu().numpy()
    gb, gi, gd = gb.cpu().numpy(), gi.cpu().numpy(), gd.cpu().numpy()
    idx = stratified(b, fl, 32, top=200)
    check(y[idx], fl[idx], oracle.forward_batch(synth.subset_pairs(b, idx)), phmm)
    R = len(b["read_off"]) - 1
    rng = np.random.default_rng(33)
    reads = np.unique(np.concatenate([rng.choice(R - 42, 23, replace=False), [R - 1]]))
    pairs = np.nonzero(np.isin(b["pair_read"], reads))[0]
    assert len(pairs) == 16 * len(reads)
    wy, wb, wi, wd, wg = oracle.backward_batch(synth.subset_pairs(b, pairs), dy[pairs])
    ro = b["read_off"]
    pos = np.concatenate([np.arange(ro[r], ro[r + 1]) for r in reads])
    sro = np.concatenate([[0], np.cumsum(ro[reads + 1] - ro[reads])])
    grad_close(gb[pos], wb[pos], "d/dbq", sro)
    grad_close(gi[pos], wi[pos], "d/diq", sro)
    grad_close(gd[pos], wd[pos], "d/ddq", sro)


def test_c3_gradient_vs_central_differences(phmm):
    """The GPU gradient of sum_{p in S} log10 L_p over 200 sampled C3 pairs S (seed 33), from
    the fused step over the whole batch with dL = 1 on S and 0 elsewhere, against FP64 central
    finite differences (h = 1e-4) of the oracle's log10 L: three positions of each sampled
    read in each quality track (its largest |gradient| and two random ones), and d/dgcp."""
    import torch
    b = synth.c3_grad()
    P = len(b["pair_read"])
    rng = np.random.default_rng(33)
    S = np.sort(rng.choice(P, 200, replace=False))
    dy = np.zeros(P)
    dy[S] = 1.0
    plan = phmm.Plan(phmm.DeviceBatch(b))
    plan.forward_partials()
    gb, gi, gd, gg = plan.backward_partials(torch.as_tensor(dy, device="cuda"))
    got = {"base_q": gb.cpu().numpy(), "ins_q": gi.cpu().numpy(), "del_q": gd.cpu().numpy()}
    gg = float(gg.cpu().numpy()[0])
    # the oracle adjoint of the sampled pairs sets each read's floor (per-read, as elsewhere)
    wy, wb, wi, wd, wg = oracle.backward_batch(synth.subset_pairs(b, S), np.ones(len(S)))
    ref = {"base_q": wb, "ins_q": wi, "del_q": wd}
    ro, hoff = b["read_off"], b["hap_off"]
    h = 1e-4

    def loglik(r, track, pos, delta):
        """sum over the sampled pairs of read r of log10 L with quality track[pos] + delta."""
        tot = 0.0
        q = {k: np.asarray(b[k][ro[r]:ro[r + 1]], dtype=np.float64).copy()
             for k in ("base_q", "ins_q", "del_q")}
        if track is not None:
            q[track][pos] += delta
        read = b["read_bases"][ro[r]:ro[r + 1]]
        for p in S[b["pair_read"][S] == r]:
            hp = b["pair_hap"][p]
            tot += oracle.forward_pair(read, q["base_q"], q["ins_q"], q["del_q"],
                                       b["hap_bases"][hoff[hp]:hoff[hp + 1]], gcp=b["gcp"])
        return tot

    n_checked = 0
    for r in np.unique(b["pair_read"][S]):
        m = int(ro[r + 1] - ro[r])
        for track in ("base_q", "ins_q", "del_q"):
            g_read = got[track][ro[r]:ro[r + 1]]
            w_read = ref[track][ro[r]:ro[r + 1]]
            floor = read_floor(w_read, [0, m])[0]
            for pos in {int(np.argmax(np.abs(w_read))), *rng.choice(m, 2, replace=False).tolist()}:
                fd = (loglik(r, track, pos, h) - loglik(r, track, pos, -h)) / (2 * h)
                tol = 1e-3 * abs(fd) + floor + 2e-9
                assert abs(g_read[pos] - fd) <= tol, (r, track, pos, g_read[pos], fd)
                n_checked += 1
    assert n_checked >= 3 * 3 * 150
    # d/dgcp: the whole sampled set
    def total(gcp):
        return float(np.sum(oracle.forward_batch(dict(synth.subset_pairs(b, S), gcp=gcp))))
    fd = (total(b["gcp"] + h) - total(b["gcp"] - h)) / (2 * h)
    assert abs(gg - fd) <= 1e-3 * abs(fd) + 1e-9, (gg, fd)
