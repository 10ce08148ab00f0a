"""FP64 CPU oracle for the batched Pair-HMM forward algorithm and its adjoint.

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` use it; the product package never imports it.  It shares no code with the CUDA
path.  ``phmm_oracle.c`` holds the arithmetic (Sec. II-A, Eq. 1-4, in FP64 with exact per-row
power-of-two renormalisation); ``brute.py`` enumerates alignment paths with exact rationals.

Python side: argument marshalling only (ctypes), plus building the shared object with gcc.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "phmm_oracle.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_OUT_DIR, "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (plain C, -O2, no vector intrinsics)."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-o", tmp, _SRC,
                               "-lm", "-lpthread"])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class _Batch(ctypes.Structure):
    _fields_ = [
        ("n_reads", ctypes.c_int64), ("n_haps", ctypes.c_int64), ("n_pairs", ctypes.c_int64),
        ("read_bases", ctypes.c_void_p), ("bq", ctypes.c_void_p), ("iq", ctypes.c_void_p),
        ("dq", ctypes.c_void_p), ("read_off", ctypes.c_void_p), ("hap_bases", ctypes.c_void_p),
        ("hap_off", ctypes.c_void_p), ("pair_read", ctypes.c_void_p),
        ("pair_hap", ctypes.c_void_p), ("gcp", ctypes.c_double), ("alpha_mode", ctypes.c_int32),
        ("gq", ctypes.c_void_p),
    ]


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = ctypes.CDLL(build())
            dp = ctypes.POINTER(ctypes.c_double)
            L.oracle_forward_pair.restype = ctypes.c_double
            L.oracle_forward_pair.argtypes = [ctypes.c_int, ctypes.c_char_p, dp, dp, dp,
                                              ctypes.c_int, ctypes.c_char_p, ctypes.c_double,
                                              ctypes.c_int, dp]
            L.oracle_backward_pair.restype = ctypes.c_double
            L.oracle_backward_pair.argtypes = [ctypes.c_int, ctypes.c_char_p, dp, dp, dp,
                                               ctypes.c_int, ctypes.c_char_p, ctypes.c_double,
                                               ctypes.c_int, dp, ctypes.c_double, dp, dp, dp, dp,
                                               dp]
            L.oracle_forward_batch.restype = ctypes.c_int
            L.oracle_forward_batch.argtypes = [ctypes.POINTER(_Batch), dp, ctypes.c_int]
            L.oracle_backward_batch.restype = ctypes.c_int
            L.oracle_backward_batch.argtypes = [ctypes.POINTER(_Batch), dp, dp, dp, dp, dp, dp,
                                                dp, ctypes.c_int]
            _lib = L
    return _lib


def _f64(x):
    return np.ascontiguousarray(np.asarray(x, dtype=np.float64))


def _dp(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _bytes(s) -> bytes:
    if isinstance(s, str):
        return s.encode("ascii")
    return bytes(np.asarray(s, dtype=np.uint8).tobytes())


def _gq_ptr(gcp_q, m):
    if gcp_q is None:
        return None, None
    g = _f64(gcp_q)
    assert g.shape == (m,)
    return g, _dp(g)


def forward_pair(read, bq, iq, dq, hap, gcp=10.0, alpha_mode=0, gcp_q=None) -> float:
    """log10 P(read | hap) for one pair; quals are Phred values (any real dtype).  gcp_q: an
    optional per-base gap-continuation track (Phred, length m) used instead of gcp."""
    r, h = _bytes(read), _bytes(hap)
    b, i, d = _f64(bq), _f64(iq), _f64(dq)
    g, gp = _gq_ptr(gcp_q, len(r))
    return lib().oracle_forward_pair(len(r), r, _dp(b), _dp(i), _dp(d), len(h), h, float(gcp),
                                     int(alpha_mode), gp)


def backward_pair(read, bq, iq, dq, hap, gcp=10.0, alpha_mode=0, dy=1.0, gcp_q=None):
    """(log10 L, d/dbq[m], d/diq[m], d/ddq[m], d/dgcp) of dy * log10 L for one pair.  With a
    per-base track gcp_q the last value is d/dgcp_q[m] (per position)."""
    r, h = _bytes(read), _bytes(hap)
    b, i, d = _f64(bq), _f64(iq), _f64(dq)
    m = len(r)
    g, gp = _gq_ptr(gcp_q, m)
    gb, gi, gd, gq, gg = np.zeros(m), np.zeros(m), np.zeros(m), np.zeros(m), np.zeros(1)
    y = lib().oracle_backward_pair(m, r, _dp(b), _dp(i), _dp(d), len(h), h, float(gcp),
                                   int(alpha_mode), gp, float(dy), _dp(gb), _dp(gi), _dp(gd),
                                   _dp(gq), _dp(gg))
    return y, gb, gi, gd, (gq if gcp_q is not None else float(gg[0]))


def _mk_batch(batch, keep):
    """Marshal a host batch dict (numpy arrays, see paper_2411_11547_gb300.synth) into ctypes."""
    a = {
        "read_bases": np.ascontiguousarray(batch["read_bases"], dtype=np.uint8),
        "bq": _f64(batch["base_q"]), "iq": _f64(batch["ins_q"]), "dq": _f64(batch["del_q"]),
        "read_off": np.ascontiguousarray(batch["read_off"], dtype=np.int64),
        "hap_bases": np.ascontiguousarray(batch["hap_bases"], dtype=np.uint8),
        "hap_off": np.ascontiguousarray(batch["hap_off"], dtype=np.int64),
        "pair_read": np.ascontiguousarray(batch["pair_read"], dtype=np.int32),
        "pair_hap": np.ascontiguousarray(batch["pair_hap"], dtype=np.int32),
    }
    keep.append(a)
    b = _Batch()
    b.n_reads = len(a["read_off"]) - 1
    b.n_haps = len(a["hap_off"]) - 1
    b.n_pairs = len(a["pair_read"])
    for k in ("read_bases", "bq", "iq", "dq", "read_off", "hap_bases", "hap_off", "pair_read",
              "pair_hap"):
        setattr(b, k, a[k].ctypes.data)
    b.gcp = float(batch["gcp"])
    b.alpha_mode = int(batch.get("alpha_mode", 0))
    if batch.get("gcp_q") is not None:
        a["gq"] = _f64(batch["gcp_q"])
        b.gq = a["gq"].ctypes.data
    else:
        b.gq = None
    return b


def default_threads() -> int:
    return len(os.sched_getaffinity(0))


def forward_batch(batch, nthreads=None) -> np.ndarray:
    """log10 L for every pair of a host batch, pairs spread over host threads."""
    keep = []
    b = _mk_batch(batch, keep)
    out = np.empty(b.n_pairs, dtype=np.float64)
    lib().oracle_forward_batch(ctypes.byref(b), _dp(out), int(nthreads or default_threads()))
    return out


def backward_batch(batch, dy, nthreads=None):
    """(log10 L[P], d/dbq[sum m], d/diq[sum m], d/ddq[sum m], d/dgcp) of sum_p dy_p log10 L_p.
    For a batch with a per-base gap-continuation track ("gcp_q", [sum m]) the last value is
    d/dgcp_q [sum m] instead of the scalar d/dgcp."""
    keep = []
    b = _mk_batch(batch, keep)
    dyv = _f64(dy)
    assert dyv.shape == (b.n_pairs,)
    out = np.empty(b.n_pairs)
    tot = int(keep[0]["read_off"][-1])
    gb, gi, gd, gq, gg = (np.zeros(tot), np.zeros(tot), np.zeros(tot), np.zeros(tot),
                          np.zeros(1))
    rc = lib().oracle_backward_batch(ctypes.byref(b), _dp(dyv), _dp(out), _dp(gb), _dp(gi),
                                     _dp(gd), _dp(gq), _dp(gg), int(nthreads or default_threads()))
    if rc != 0:
        raise MemoryError("oracle_backward_batch failed")
    return out, gb, gi, gd, (gq if batch.get("gcp_q") is not None else float(gg[0]))
