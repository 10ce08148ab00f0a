"""Host-side checks of the C ABI (no GPU): the library builds, loads and exports every entry
point include/phmm.h declares; argument checks that need no device answer correctly."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2411_11547_gb300 import _build, phmm
    _build.build()
    return phmm.lib()


def declared_functions():
    names = []
    for h in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if not h.endswith(".h"):
            continue
        src = open(os.path.join(ROOT, "include", h)).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        for m in re.finditer(r"^[A-Za-z_][\w\s\*]*?\b(phmm_\w+)\s*\(", src, flags=re.M):
            names.append(m.group(1))
    return sorted(set(names))


def test_header_declares_the_boundary():
    names = declared_functions()
    for must in ("phmm_plan_create", "phmm_forward", "phmm_backward", "phmm_workspace_bytes",
                 "phmm_forward_partials", "phmm_backward_partials", "phmm_plan_destroy",
                 "phmm_status_str"):
        assert must in names


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_status_strings(lib):
    for code in (0, -1, -2, -3, -4, -5):
        assert lib.phmm_status_str(code)
    assert lib.phmm_status_str(-99) == b"unknown status"


def test_options_default(lib):
    from paper_2411_11547_gb300 import phmm
    o = phmm.options()
    assert o.first_line == phmm.FIRST_EXT32 and o.rescue == 1 and o.binning == 1
    assert o.use_graph == 1 and o.persistent == 1 and o.bin_table_valid == 0


def test_plan_create_rejects_bad_arguments_on_host(lib):
    from paper_2411_11547_gb300 import phmm
    h = ctypes.c_void_p()
    assert lib.phmm_plan_create(None, None, None, ctypes.byref(h)) == phmm.PHMM_EINVAL
    b = phmm.Batch()  # n_reads = 0
    assert lib.phmm_plan_create(ctypes.byref(b), None, None, ctypes.byref(h)) == phmm.PHMM_EINVAL
    b.n_reads, b.n_haps, b.n_pairs = 1, 1, 1
    b.gcp = 10.0  # NULL data pointers
    assert lib.phmm_plan_create(ctypes.byref(b), None, None, ctypes.byref(h)) == phmm.PHMM_EINVAL
    assert not h.value


def test_forward_rejects_null_plan(lib):
    from paper_2411_11547_gb300 import phmm
    assert lib.phmm_forward(None, None, 0, None, None, None) == phmm.PHMM_EINVAL
    assert lib.phmm_backward(None, None, 0, None, None, None, None, None, None,
                             None) == phmm.PHMM_EINVAL
    assert lib.phmm_forward_partials(None, None, 0, None, None, None) == phmm.PHMM_EINVAL
    assert lib.phmm_backward_partials(None, None, 0, None, None, None, None, None,
                                      None, None) == phmm.PHMM_EINVAL
    assert lib.phmm_workspace_bytes(None) == 0


def test_autotune_rejects_bad_arguments_on_host(lib):
    from paper_2411_11547_gb300 import phmm
    o = phmm.options()
    b = phmm.Batch()
    assert lib.phmm_autotune(None, ctypes.byref(o), 3, 16, None) == phmm.PHMM_EINVAL
    assert lib.phmm_autotune(ctypes.byref(b), None, 3, 16, None) == phmm.PHMM_EINVAL
    assert lib.phmm_autotune(ctypes.byref(b), ctypes.byref(o), 0, 16, None) == phmm.PHMM_EINVAL
    assert lib.phmm_autotune(ctypes.byref(b), ctypes.byref(o), 3, 0, None) == phmm.PHMM_EINVAL
    assert lib.phmm_autotune(ctypes.byref(b), ctypes.byref(o), 3, 16, None) == phmm.PHMM_EINVAL
    assert o.bin_table_valid == 0 and o.bwd_table_valid == 0


def test_autograd_wrapper_checks_tensor_layout():
    import numpy as np
    import torch
    from paper_2411_11547_gb300 import phmm as ph, synth
    from paper_2411_11547_gb300.autograd import PairHMMLogLik, layout_from_host
    assert issubclass(PairHMMLogLik, torch.autograd.Function)
    b = synth.random_pairs(3, 4, (5, 10), (5, 10), qual_dtype=np.float32)
    layout, (bq, iq, dq) = layout_from_host(b, device="cpu")
    db = ph.DeviceBatch.from_tensors(layout["read_bases"], bq, iq, dq, layout["read_off"],
                                     layout["hap_bases"], layout["hap_off"],
                                     layout["pair_read"], layout["pair_hap"], b["gcp"])
    assert db.n_pairs == 4 and db.qual_dtype == ph.QUAL_F32
    with pytest.raises(TypeError):
        ph.DeviceBatch.from_tensors(layout["read_bases"], bq.double(), iq, dq,
                                    layout["read_off"], layout["hap_bases"], layout["hap_off"],
                                    layout["pair_read"], layout["pair_hap"], b["gcp"])
    with pytest.raises(TypeError):
        ph.DeviceBatch.from_tensors(layout["read_bases"], bq, iq, dq,
                                    layout["read_off"].int(), layout["hap_bases"],
                                    layout["hap_off"], layout["pair_read"], layout["pair_hap"],
                                    b["gcp"])


def test_score_host_rejects_bad_input_before_touching_the_gpu(lib):
    import numpy as np
    from paper_2411_11547_gb300 import phmm, synth
    b = synth.random_pairs(4, 6, (5, 10), (5, 10))
    keep = []
    s = phmm.host_batch_struct(b, keep)
    out = np.empty(6)
    fl = np.empty(6, dtype=np.uint8)
    assert lib.phmm_score_host(None, None, 10, out.ctypes.data, fl.ctypes.data) == phmm.PHMM_EINVAL
    assert lib.phmm_score_host(ctypes.byref(s), None, 0, out.ctypes.data,
                               fl.ctypes.data) == phmm.PHMM_EINVAL
    bad = dict(b, pair_hap=b["pair_hap"].copy())
    bad["pair_hap"][2] = 99
    s2 = phmm.host_batch_struct(bad, keep)
    assert lib.phmm_score_host(ctypes.byref(s2), None, 10, out.ctypes.data,
                               fl.ctypes.data) == phmm.PHMM_EINVAL


def test_grad_host_rejects_bad_input_before_touching_the_gpu(lib):
    import numpy as np
    from paper_2411_11547_gb300 import phmm, synth
    b = synth.random_pairs(4, 6, (5, 10), (5, 10))
    keep = []
    s = phmm.host_batch_struct(b, keep)
    sm = int(b["read_off"][-1])
    out, fl = np.empty(6), np.empty(6, dtype=np.uint8)
    g = [np.empty(sm, dtype=np.float32) for _ in range(3)]
    gg = ctypes.c_double()
    dL = np.ones(6)
    args = ([out.ctypes.data, fl.ctypes.data] + [x.ctypes.data for x in g] + [None]
            + [ctypes.byref(gg)])
    assert lib.phmm_grad_host(ctypes.byref(s), None, 10, None, *args) == phmm.PHMM_EINVAL
    no_grad = args[:2] + [None, None, None, None, ctypes.byref(gg)]
    assert lib.phmm_grad_host(ctypes.byref(s), None, 10, dL.ctypes.data,
                              *no_grad) == phmm.PHMM_EINVAL
    # a batch with a per-base gap-continuation track needs the d_gcp_q array
    tr = phmm.host_batch_struct(dict(b, gcp_q=np.full(sm, 10, np.uint8)), keep)
    assert lib.phmm_grad_host(ctypes.byref(tr), None, 10, dL.ctypes.data,
                              *args) == phmm.PHMM_EINVAL
    bad = dict(b, pair_hap=b["pair_hap"].copy())
    bad["pair_hap"][2] = 99
    s2 = phmm.host_batch_struct(bad, keep)
    assert lib.phmm_grad_host(ctypes.byref(s2), None, 10, dL.ctypes.data,
                              *args) == phmm.PHMM_EINVAL


def test_plan_create_rejects_bad_options_before_touching_the_gpu(lib):
    # option checks come before any device work, so host pointers (never read) serve here
    import numpy as np
    from paper_2411_11547_gb300 import phmm, synth
    b = synth.random_pairs(4, 6, (5, 10), (5, 10))
    keep = []
    s = phmm.host_batch_struct(b, keep)
    h = ctypes.c_void_p()
    for kw in ({"adjoint_rescue": 3}, {"adjoint_rescue": -1}, {"first_line": 7},
               {"warps_per_block": 8}):
        o = phmm.options(**kw)
        assert lib.phmm_plan_create(ctypes.byref(s), ctypes.byref(o), None,
                                    ctypes.byref(h)) == phmm.PHMM_EINVAL, kw
        assert not h.value
