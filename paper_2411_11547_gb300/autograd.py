"""torch.autograd.Function over the library's forward and adjoint (include/phmm.h).

y_p = log10 P(read | haplotype) of every pair (Eq. 1-4 summed over the last row); the gradient
flows to the three Phred quality tracks (float32, treated as continuous) and to the
gap-continuation Phred quality: one scalar, or a per-base track of one value per read base.  Both directions run in the CUDA kernels behind the C ABI; the
gradient sums over the pairs sharing a read are taken in FP64 on the device, deterministic.
"""
from __future__ import annotations

import torch

from . import phmm as _ph


class PairHMMLogLik(torch.autograd.Function):
    """log10 L for every pair; backward gives d/d(base_q, ins_q, del_q, gcp).

    Arguments: float32 quality tensors `base_q, ins_q, del_q` [sum m] (device), `gcp` (a 0-d
    float64/float32 tensor, or a float32 device tensor [sum m]: a per-base gap-continuation
    track), and `layout`, a dict of device tensors with keys
    read_bases, read_off, hap_bases, hap_off, pair_read, pair_hap (and optionally
    alpha_mode).  Returns (log10L float64 [pairs], flags uint8 [pairs]); flags are not
    differentiable.  One plan (validation, binning, workspace) is built per call.  When a
    gradient is wanted the forward is the fused call (phmm_forward_partials: the adjoint sweep
    yields log10 L and every pair's partials at once) and backward only weights the partials
    by dy and reduces them; otherwise it is the plain forward.
    """

    @staticmethod
    def forward(ctx, base_q, ins_q, del_q, gcp, layout, opts=None):
        track = torch.is_tensor(gcp) and gcp.numel() > 1
        if track:
            g, gq = 10.0, gcp.detach().to(base_q.dtype).contiguous()
        else:
            g = float(gcp.detach().reshape(()).item()) if torch.is_tensor(gcp) else float(gcp)
            gq = None
        db = _ph.DeviceBatch.from_tensors(
            layout["read_bases"], base_q.detach().contiguous(), ins_q.detach().contiguous(),
            del_q.detach().contiguous(), layout["read_off"], layout["hap_bases"],
            layout["hap_off"], layout["pair_read"], layout["pair_hap"], g,
            layout.get("alpha_mode", 0), gcp_q=gq)
        ctx.track = track
        plan = _ph.Plan(db, opts)
        ctx.fused = any(ctx.needs_input_grad[:4])
        out, flags = plan.forward_partials() if ctx.fused else plan.forward()
        ctx.plan = plan
        ctx.gcp_like = gcp if torch.is_tensor(gcp) else None
        ctx.mark_non_differentiable(flags)
        return out, flags

    @staticmethod
    def backward(ctx, dy, _dflags):
        plan = ctx.plan
        if dy is None:
            return None, None, None, None, None, None
        dy = dy.contiguous()
        res = plan.backward_partials(dy) if ctx.fused else plan.backward(dy)
        dbq, diq, ddq, dgcp = res[:4]
        gg = None
        if ctx.gcp_like is not None and ctx.needs_input_grad[3]:
            src = res[4] if ctx.track else dgcp
            gg = src.reshape(ctx.gcp_like.shape).to(ctx.gcp_like.dtype)
        ctx.plan = None
        return dbq, diq, ddq, gg, None, None


def pair_hmm_loglik(base_q, ins_q, del_q, gcp, layout, opts=None):
    """Functional form of PairHMMLogLik.apply."""
    return PairHMMLogLik.apply(base_q, ins_q, del_q, gcp, layout, opts)


def layout_from_host(batch, device="cuda"):
    """(layout dict, float32 quals on the device) from a host batch dict (synth.py format)."""
    import numpy as np

    def dev(a, dt):
        return torch.from_numpy(np.ascontiguousarray(a)).to(device=device, dtype=dt)

    layout = {"read_bases": dev(batch["read_bases"], torch.uint8),
              "read_off": dev(batch["read_off"], torch.int64),
              "hap_bases": dev(batch["hap_bases"], torch.uint8),
              "hap_off": dev(batch["hap_off"], torch.int64),
              "pair_read": dev(batch["pair_read"], torch.int32),
              "pair_hap": dev(batch["pair_hap"], torch.int32),
              "alpha_mode": int(batch.get("alpha_mode", 0))}
    quals = tuple(dev(np.asarray(batch[k], dtype=np.float32), torch.float32)
                  for k in ("base_q", "ins_q", "del_q"))
    return layout, quals
