"""Thin Python binding of libphmm (include/phmm.h): argument marshalling only.

Every step of the Pair-HMM path runs in the library's CUDA kernels; PyTorch provides device
memory and the current stream.  There is no CPU fallback: if the shared library cannot be
loaded, importing the binding's entry points raises.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

PHMM_OK, PHMM_EINVAL, PHMM_ETOOLONG, PHMM_ENOMEM, PHMM_ECUDA, PHMM_ESTATE = 0, -1, -2, -3, -4, -5
PHMM_EGUARD = -6  # debug builds: a guard region or a kernel index check failed
PHMM_MAX_READ_LEN = 512
FLAG_FP32, FLAG_RESCUED64, FLAG_EXTENDED, FLAG_INVALID = 1, 2, 4, 8


def cfg_index(lanes: int, rows: int) -> int:
    """Group index held by the options' bin_rows / bwd_rows tables (lanes 4/8/16/32, rows per
    lane 4..20), as the library encodes it."""
    return {4: 0, 8: 1, 16: 2, 32: 3}[lanes] * 17 + (rows - 4)


def cfg_shape(c: int) -> tuple:
    """(lanes, rows) of group index c."""
    return 4 << (c // 17), 4 + c % 17
QUAL_U8, QUAL_F32 = 0, 1
FIRST_PLAIN32, FIRST_EXT32 = 0, 1

_PKG = os.path.dirname(os.path.abspath(__file__))
# PHMM_DEBUG=1: the debug build (guard regions and kernel index checks, see _build.py)
_LIB_PATH = os.path.join(_PKG, "libphmm_debug.so" if os.environ.get("PHMM_DEBUG") == "1"
                         else "libphmm.so")
_lock = threading.Lock()
_lib = None


class PhmmError(RuntimeError):
    def __init__(self, status, what=""):
        self.status = status
        msg = lib().phmm_status_str(status).decode() if _lib is not None else str(status)
        if status == PHMM_ECUDA and _lib is not None:
            msg += f" (cudaError {_lib.phmm_last_cuda_error()})"
        super().__init__(f"{what}: {msg} [{status}]")


class Batch(ctypes.Structure):
    _fields_ = [
        ("n_reads", ctypes.c_int64), ("n_haps", ctypes.c_int64), ("n_pairs", ctypes.c_int64),
        ("read_bases", ctypes.c_void_p), ("base_q", ctypes.c_void_p),
        ("ins_q", ctypes.c_void_p), ("del_q", ctypes.c_void_p),
        ("qual_dtype", ctypes.c_int32), ("alpha_mode", ctypes.c_int32),
        ("read_off", ctypes.c_void_p), ("hap_bases", ctypes.c_void_p),
        ("hap_off", ctypes.c_void_p), ("pair_read", ctypes.c_void_p),
        ("pair_hap", ctypes.c_void_p), ("gcp", ctypes.c_double),
        ("gcp_q", ctypes.c_void_p),
    ]


class Options(ctypes.Structure):
    _fields_ = [
        ("first_line", ctypes.c_int32), ("rescue", ctypes.c_int32),
        ("binning", ctypes.c_int32), ("lanes", ctypes.c_int32), ("rows", ctypes.c_int32),
        ("persistent", ctypes.c_int32), ("use_graph", ctypes.c_int32),
        ("warps_per_block", ctypes.c_int32),
        ("bin_rows", ctypes.c_int32 * (PHMM_MAX_READ_LEN // 4 + 1)),
        ("bin_table_valid", ctypes.c_int32), ("adjoint_rescue", ctypes.c_int32),
        ("bwd_rows", ctypes.c_int32 * (PHMM_MAX_READ_LEN // 4 + 1)),
        ("bwd_table_valid", ctypes.c_int32), ("bwd_warps_per_block", ctypes.c_int32),
    ]


def lib():
    """Load libphmm.so (build it first with __graft_entry__.build() or _build.build())."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(_LIB_PATH):
                raise ImportError(f"{os.path.basename(_LIB_PATH)} not built at {_LIB_PATH}; run "
                                  f"the package build")
            L = ctypes.CDLL(_LIB_PATH)
            vp, i64p = ctypes.c_void_p, ctypes.POINTER(ctypes.c_int64)
            L.phmm_options_default.argtypes = [ctypes.POINTER(Options)]
            L.phmm_options_default.restype = None
            L.phmm_plan_create.argtypes = [ctypes.POINTER(Batch), ctypes.POINTER(Options), vp,
                                           ctypes.POINTER(vp)]
            L.phmm_plan_create.restype = ctypes.c_int
            L.phmm_workspace_bytes.argtypes = [vp]
            L.phmm_workspace_bytes.restype = ctypes.c_size_t
            L.phmm_plan_info.argtypes = [vp, i64p, i64p, i64p]
            L.phmm_plan_info.restype = ctypes.c_int
            L.phmm_forward.argtypes = [vp, vp, ctypes.c_size_t, vp, vp, vp]
            L.phmm_forward.restype = ctypes.c_int
            L.phmm_backward.argtypes = [vp, vp, ctypes.c_size_t, vp, vp, vp, vp, vp, vp, vp]
            L.phmm_backward.restype = ctypes.c_int
            L.phmm_forward_partials.argtypes = [vp, vp, ctypes.c_size_t, vp, vp, vp]
            L.phmm_forward_partials.restype = ctypes.c_int
            L.phmm_backward_partials.argtypes = [vp, vp, ctypes.c_size_t, vp, vp, vp, vp, vp, vp,
                                                 vp]
            L.phmm_backward_partials.restype = ctypes.c_int
            L.phmm_plan_destroy.argtypes = [vp]
            L.phmm_plan_destroy.restype = None
            L.phmm_status_str.argtypes = [ctypes.c_int]
            L.phmm_status_str.restype = ctypes.c_char_p
            L.phmm_last_cuda_error.argtypes = []
            L.phmm_last_cuda_error.restype = ctypes.c_int
            L.phmm_plan_launch_count.argtypes = [vp, ctypes.c_int]
            L.phmm_plan_launch_count.restype = ctypes.c_int
            L.phmm_plan_wavefront_ms.argtypes = [vp, ctypes.POINTER(ctypes.c_float),
                                                 ctypes.POINTER(ctypes.c_float)]
            L.phmm_plan_wavefront_ms.restype = ctypes.c_int
            L.phmm_plan_backward_ms.argtypes = [vp, ctypes.POINTER(ctypes.c_float),
                                                ctypes.POINTER(ctypes.c_float)]
            L.phmm_plan_backward_ms.restype = ctypes.c_int
            L.phmm_plan_rescue_counts.argtypes = [vp, vp, vp, i64p]
            L.phmm_plan_rescue_counts.restype = ctypes.c_int
            L.phmm_autotune.argtypes = [ctypes.POINTER(Batch), ctypes.POINTER(Options),
                                        ctypes.c_int, ctypes.c_int64, vp]
            L.phmm_autotune.restype = ctypes.c_int
            L.phmm_score_host.argtypes = [ctypes.POINTER(Batch), ctypes.POINTER(Options),
                                          ctypes.c_int64, vp, vp]
            L.phmm_score_host.restype = ctypes.c_int
            L.phmm_grad_host.argtypes = [ctypes.POINTER(Batch), ctypes.POINTER(Options),
                                         ctypes.c_int64, vp, vp, vp, vp, vp, vp, vp, vp]
            L.phmm_grad_host.restype = ctypes.c_int
            L.phmm_score_host_release.argtypes = []
            L.phmm_score_host_release.restype = None
            L.phmm_probe_pipe.argtypes = [ctypes.c_int, ctypes.c_int,
                                          ctypes.POINTER(ctypes.c_double),
                                          ctypes.POINTER(ctypes.c_double)]
            L.phmm_probe_pipe.restype = ctypes.c_int
            _lib = L
    return _lib


def options(**kw) -> Options:
    """Library defaults (phmm_options_default) with keyword overrides; `bin_rows` / `bwd_rows`
    may be sequences of group ids per 4-row read-length bucket for the forward / adjoint
    (they set bin_table_valid / bwd_table_valid)."""
    o = Options()
    lib().phmm_options_default(ctypes.byref(o))
    for k, v in kw.items():
        if k in ("bin_rows", "bwd_rows"):
            arr = getattr(o, k)
            for i, x in enumerate(v):
                arr[i] = int(x)
            setattr(o, "bin_table_valid" if k == "bin_rows" else "bwd_table_valid", 1)
        else:
            setattr(o, k, int(v))
    return o


def _stream(stream=None):
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


class DeviceBatch:
    """A host batch (dict of numpy arrays, see synth.py) copied to device tensors."""

    def __init__(self, batch, device="cuda", non_blocking=False):
        import torch
        self.host = batch
        qd = np.asarray(batch["base_q"]).dtype
        self.qual_dtype = QUAL_F32 if qd == np.float32 else QUAL_U8
        qt = torch.float32 if self.qual_dtype == QUAL_F32 else torch.uint8

        def dev(a, dt):
            t = torch.from_numpy(np.ascontiguousarray(a))
            if non_blocking:
                t = t.pin_memory()
            return t.to(device=device, dtype=dt, non_blocking=non_blocking)

        self.read_bases = dev(batch["read_bases"], torch.uint8)
        self.base_q = dev(batch["base_q"], qt)
        self.ins_q = dev(batch["ins_q"], qt)
        self.del_q = dev(batch["del_q"], qt)
        self.read_off = dev(batch["read_off"], torch.int64)
        self.hap_bases = dev(batch["hap_bases"], torch.uint8)
        self.hap_off = dev(batch["hap_off"], torch.int64)
        self.pair_read = dev(batch["pair_read"], torch.int32)
        self.pair_hap = dev(batch["pair_hap"], torch.int32)
        self.gcp = float(batch["gcp"])
        self.alpha_mode = int(batch.get("alpha_mode", 0))
        gq = batch.get("gcp_q")
        self.gcp_q = dev(gq, qt) if gq is not None else None

    @classmethod
    def from_tensors(cls, read_bases, base_q, ins_q, del_q, read_off, hap_bases, hap_off,
                     pair_read, pair_hap, gcp, alpha_mode=0, gcp_q=None):
        """Wrap tensors already on the device (no copy).  The quals are uint8 or float32; the
        offsets int64, the pair lists int32, all contiguous.  gcp_q: an optional per-base
        gap-continuation track (the quals' dtype, one value per read base)."""
        import torch
        self = cls.__new__(cls)
        self.host = None
        if base_q.dtype == torch.float32:
            self.qual_dtype = QUAL_F32
        elif base_q.dtype == torch.uint8:
            self.qual_dtype = QUAL_U8
        else:
            raise TypeError(f"quals must be uint8 or float32, got {base_q.dtype}")
        want = {"read_bases": torch.uint8, "base_q": base_q.dtype, "ins_q": base_q.dtype,
                "del_q": base_q.dtype, "read_off": torch.int64, "hap_bases": torch.uint8,
                "hap_off": torch.int64, "pair_read": torch.int32, "pair_hap": torch.int32}
        loc = dict(read_bases=read_bases, base_q=base_q, ins_q=ins_q, del_q=del_q,
                   read_off=read_off, hap_bases=hap_bases, hap_off=hap_off,
                   pair_read=pair_read, pair_hap=pair_hap)
        for k, dt in want.items():
            t = loc[k]
            if t.dtype != dt or not t.is_contiguous() or t.device != read_bases.device:
                raise TypeError(f"{k}: need a contiguous {dt} tensor on {read_bases.device}")
            setattr(self, k, t)
        self.gcp = float(gcp)
        self.alpha_mode = int(alpha_mode)
        if gcp_q is not None and (gcp_q.dtype != base_q.dtype or not gcp_q.is_contiguous()
                                  or gcp_q.device != read_bases.device
                                  or gcp_q.numel() != base_q.numel()):
            raise TypeError("gcp_q: need a contiguous tensor like base_q")
        self.gcp_q = gcp_q
        return self

    @property
    def n_pairs(self):
        return int(self.pair_read.numel())

    def struct(self) -> Batch:
        b = Batch()
        b.n_reads = self.read_off.numel() - 1
        b.n_haps = self.hap_off.numel() - 1
        b.n_pairs = self.pair_read.numel()
        b.read_bases = self.read_bases.data_ptr()
        b.base_q = self.base_q.data_ptr()
        b.ins_q = self.ins_q.data_ptr()
        b.del_q = self.del_q.data_ptr()
        b.qual_dtype = self.qual_dtype
        b.alpha_mode = self.alpha_mode
        b.read_off = self.read_off.data_ptr()
        b.hap_bases = self.hap_bases.data_ptr()
        b.hap_off = self.hap_off.data_ptr()
        b.pair_read = self.pair_read.data_ptr() if b.n_pairs else None
        b.pair_hap = self.pair_hap.data_ptr() if b.n_pairs else None
        b.gcp = self.gcp
        b.gcp_q = self.gcp_q.data_ptr() if self.gcp_q is not None else None
        return b


class Plan:
    """phmm_plan_create + a torch-allocated workspace; forward/backward on torch tensors."""

    def __init__(self, dbatch: DeviceBatch, opts: Options | None = None, stream=None):
        import torch
        self.dbatch = dbatch
        self._b = dbatch.struct()
        self.opts = opts if opts is not None else options()
        h = ctypes.c_void_p()
        rc = lib().phmm_plan_create(ctypes.byref(self._b), ctypes.byref(self.opts),
                                    _stream(stream), ctypes.byref(h))
        if rc != PHMM_OK:
            raise PhmmError(rc, "phmm_plan_create")
        self.handle = h
        self.ws_bytes = int(lib().phmm_workspace_bytes(h))
        dev = dbatch.read_bases.device
        self.workspace = torch.empty(self.ws_bytes + 256, dtype=torch.uint8, device=dev)
        off = (-self.workspace.data_ptr()) % 256
        self._ws_ptr = self.workspace.data_ptr() + off
        sm, sn, c = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
        lib().phmm_plan_info(h, ctypes.byref(sm), ctypes.byref(sn), ctypes.byref(c))
        self.sum_m, self.sum_n, self.cells = sm.value, sn.value, c.value

    def forward(self, out=None, flags=None, stream=None):
        import torch
        P = self.dbatch.n_pairs
        dev = self.dbatch.read_bases.device
        if out is None:
            out = torch.empty(P, dtype=torch.float64, device=dev)
        if flags is None:
            flags = torch.empty(P, dtype=torch.uint8, device=dev)
        rc = lib().phmm_forward(self.handle, ctypes.c_void_p(self._ws_ptr), self.ws_bytes,
                                ctypes.c_void_p(out.data_ptr() if P else 0),
                                ctypes.c_void_p(flags.data_ptr() if P else 0), _stream(stream))
        if rc != PHMM_OK:
            raise PhmmError(rc, "phmm_forward")
        return out, flags

    def backward(self, dL, stream=None, out=None):
        """phmm_backward: d(loss)/d(quals) given dL = d(loss)/d(log10 L) (after forward):
        (d_base_q, d_ins_q, d_del_q, d_gcp), plus d_gcp_q for a batch with a per-base
        gap-continuation track.  `out`: optional tensors of that tuple to write into (the
        per-base ones of at least sum_m elements)."""
        return self._grad(lib().phmm_backward, "phmm_backward", dL, stream, out)

    def forward_partials(self, out=None, flags=None, stream=None):
        """phmm_forward_partials: log10 L and flags from the adjoint sweep's own forward pass,
        keeping every pair's d log10 L / d(quals) in the workspace for backward_partials."""
        import torch
        P = self.dbatch.n_pairs
        dev = self.dbatch.read_bases.device
        if out is None:
            out = torch.empty(P, dtype=torch.float64, device=dev)
        if flags is None:
            flags = torch.empty(P, dtype=torch.uint8, device=dev)
        rc = lib().phmm_forward_partials(self.handle, ctypes.c_void_p(self._ws_ptr),
                                         self.ws_bytes,
                                         ctypes.c_void_p(out.data_ptr() if P else 0),
                                         ctypes.c_void_p(flags.data_ptr() if P else 0),
                                         _stream(stream))
        if rc != PHMM_OK:
            raise PhmmError(rc, "phmm_forward_partials")
        return out, flags

    def backward_partials(self, dL, stream=None, out=None):
        """phmm_backward_partials: the partials of the latest forward_partials weighted by dL
        and reduced per read (same outputs and `out` as backward).  Calls that repeat the
        previous call's pointers (pass `out` and the same dL tensor) replay a captured CUDA
        graph on small batches."""
        return self._grad(lib().phmm_backward_partials, "phmm_backward_partials", dL, stream,
                          out)

    def _grad(self, fn, name, dL, stream, out=None):
        import torch
        dev = self.dbatch.read_bases.device
        tot = max(self.sum_m, 1)
        track = self.dbatch.gcp_q is not None
        if out is not None:
            dbq, diq, ddq, dgcp = out[:4]
            dgq = out[4] if track else None
        else:
            dbq = torch.empty(tot, dtype=torch.float32, device=dev)
            diq = torch.empty(tot, dtype=torch.float32, device=dev)
            ddq = torch.empty(tot, dtype=torch.float32, device=dev)
            dgq = torch.empty(tot, dtype=torch.float32, device=dev) if track else None
            dgcp = torch.empty(1, dtype=torch.float64, device=dev)
        if dL.device != dev or dL.dtype != torch.float64 or not dL.is_contiguous():
            dL = dL.to(device=dev, dtype=torch.float64).contiguous()
        rc = fn(self.handle, ctypes.c_void_p(self._ws_ptr), self.ws_bytes,
                ctypes.c_void_p(dL.data_ptr()), ctypes.c_void_p(dbq.data_ptr()),
                ctypes.c_void_p(diq.data_ptr()), ctypes.c_void_p(ddq.data_ptr()),
                ctypes.c_void_p(dgq.data_ptr() if track else 0),
                ctypes.c_void_p(dgcp.data_ptr()), _stream(stream))
        if rc != PHMM_OK:
            raise PhmmError(rc, name)
        out = (dbq[: self.sum_m], diq[: self.sum_m], ddq[: self.sum_m], dgcp)
        return out + (dgq[: self.sum_m],) if track else out

    def launch_count(self, which=0):
        return int(lib().phmm_plan_launch_count(self.handle, which))

    def wavefront_ms(self):
        a, r = ctypes.c_float(), ctypes.c_float()
        lib().phmm_plan_wavefront_ms(self.handle, ctypes.byref(a), ctypes.byref(r))
        return a.value, r.value

    def backward_ms(self):
        a, r = ctypes.c_float(), ctypes.c_float()
        lib().phmm_plan_backward_ms(self.handle, ctypes.byref(a), ctypes.byref(r))
        return a.value, r.value

    def rescue_counts(self, stream=None):
        """(forward FP64 rescues, of which extended, adjoint FP64 hand-offs, of which for the
        scale range, of which for non-finite partials, 0)."""
        c = (ctypes.c_int64 * 6)()
        rc = lib().phmm_plan_rescue_counts(self.handle, ctypes.c_void_p(self._ws_ptr),
                                           _stream(stream), c)
        if rc != PHMM_OK:
            raise PhmmError(rc, "phmm_plan_rescue_counts")
        return tuple(int(x) for x in c)

    def close(self):
        if getattr(self, "handle", None):
            lib().phmm_plan_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def forward(batch, opts: Options | None = None, device="cuda"):
    """log10 P(read | haplotype) and flags for every pair of a host or device batch."""
    db = batch if isinstance(batch, DeviceBatch) else DeviceBatch(batch, device)
    plan = Plan(db, opts)
    out, flags = plan.forward()
    return out, flags


def autotune(dbatch: DeviceBatch, opts: Options | None = None, which: int = 3,
             sample_pairs: int = 32768, stream=None) -> Options:
    """phmm_autotune: measured read-length -> group tables (forward: which & 1, adjoint:
    which & 2) for this batch, returned in a copy of `opts` (default options if None)."""
    o = Options.from_buffer_copy(opts if opts is not None else options())
    b = dbatch.struct()
    rc = lib().phmm_autotune(ctypes.byref(b), ctypes.byref(o), int(which), int(sample_pairs),
                             _stream(stream))
    if rc != PHMM_OK:
        raise PhmmError(rc, "phmm_autotune")
    return o


def host_batch_struct(batch, keep):
    """Batch struct over host numpy arrays (kept alive in `keep`)."""
    def arr(k, dt):
        a = np.ascontiguousarray(batch[k], dtype=dt)
        keep.append(a)
        return a.ctypes.data
    qd = np.asarray(batch["base_q"]).dtype
    qdt = np.float32 if qd == np.float32 else np.uint8
    b = Batch()
    b.n_reads = len(batch["read_off"]) - 1
    b.n_haps = len(batch["hap_off"]) - 1
    b.n_pairs = len(batch["pair_read"])
    b.read_bases = arr("read_bases", np.uint8)
    b.base_q = arr("base_q", qdt)
    b.ins_q = arr("ins_q", qdt)
    b.del_q = arr("del_q", qdt)
    b.qual_dtype = QUAL_F32 if qdt == np.float32 else QUAL_U8
    b.alpha_mode = int(batch.get("alpha_mode", 0))
    b.read_off = arr("read_off", np.int64)
    b.hap_bases = arr("hap_bases", np.uint8)
    b.hap_off = arr("hap_off", np.int64)
    b.pair_read = arr("pair_read", np.int32)
    b.pair_hap = arr("pair_hap", np.int32)
    b.gcp = float(batch["gcp"])
    b.gcp_q = arr("gcp_q", qdt) if batch.get("gcp_q") is not None else None
    return b


def score_host(batch, opts: Options | None = None, subset_cells: int = 1 << 33):
    """phmm_score_host: log10 L and flags (numpy) of a batch held in host memory, scored in
    pipelined subsets of about `subset_cells` cells."""
    keep = []
    b = host_batch_struct(batch, keep)
    P = b.n_pairs
    out = np.empty(P, dtype=np.float64)
    flags = np.empty(P, dtype=np.uint8)
    rc = lib().phmm_score_host(ctypes.byref(b), ctypes.byref(opts) if opts is not None else None,
                               int(subset_cells), out.ctypes.data, flags.ctypes.data)
    if rc != PHMM_OK:
        raise PhmmError(rc, "phmm_score_host")
    return out, flags


def grad_host(batch, dL, opts: Options | None = None, subset_cells: int = 1 << 38, out=None):
    """phmm_grad_host: log10 L, flags and d(loss)/d(base_q, ins_q, del_q, gcp) (numpy) of a
    batch held in host memory, given dL = d(loss)/d(log10 L) per pair (host), in pipelined
    subsets of about `subset_cells` cells.  `out`: optional preallocated
    (log10 [P] f64, flags [P] u8, dbq, diq, ddq [sum m] f32) arrays to write into.  A batch
    with a per-base gap-continuation track ("gcp_q") also returns d_gcp_q [sum m]."""
    keep = []
    b = host_batch_struct(batch, keep)
    P = b.n_pairs
    sm = int(np.asarray(batch["read_off"])[-1])
    if out is None:
        out = (np.empty(P, dtype=np.float64), np.empty(P, dtype=np.uint8),
               np.empty(sm, dtype=np.float32), np.empty(sm, dtype=np.float32),
               np.empty(sm, dtype=np.float32))
    y, flags, gb, gi, gd = out
    dL = np.ascontiguousarray(dL, dtype=np.float64)
    if dL.shape != (P,):
        raise ValueError("dL must hold one value per pair")
    track = batch.get("gcp_q") is not None
    gq = np.empty(sm, dtype=np.float32) if track else None
    gg = ctypes.c_double()
    rc = lib().phmm_grad_host(ctypes.byref(b), ctypes.byref(opts) if opts is not None else None,
                              int(subset_cells), dL.ctypes.data, y.ctypes.data, flags.ctypes.data,
                              gb.ctypes.data, gi.ctypes.data, gd.ctypes.data,
                              gq.ctypes.data if track else None, ctypes.byref(gg))
    if rc != PHMM_OK:
        raise PhmmError(rc, "phmm_grad_host")
    return (y, flags, gb, gi, gd, gg.value) + ((gq,) if track else ())


def probe_pipe(kind: int, iters: int = 4000):
    """Lane operations per second of FFMA (0), packed f32x2 FMA (1) or DFMA (2)."""
    r, ms = ctypes.c_double(), ctypes.c_double()
    rc = lib().phmm_probe_pipe(kind, iters, ctypes.byref(r), ctypes.byref(ms))
    if rc != PHMM_OK:
        raise PhmmError(rc, "phmm_probe_pipe")
    return r.value, ms.value
