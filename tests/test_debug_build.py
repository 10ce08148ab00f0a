"""The debug build (libphmm_debug.so, -DPHMM_DEBUG): guard regions after every workspace region,
checked after every call, and index checks in the kernels.

CPU: the debug library builds and exports every symbol include/phmm.h declares; the release
library answers the debug calls with PHMM_ESTATE.  GPU (in a child process that loads the
debug library): a forward and fused training step pass their checks and match the oracle; a
guard byte overwritten from the host is reported as PHMM_EGUARD, and the next call refills
the guards.
"""
import ctypes
import os
import re
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "phmm.h")).read()
    return sorted(set(re.findall(r"^(?:const )?\w[\w\s\*]*?\b(phmm_\w+)\(", src, re.M)))


def test_debug_library_builds_and_exports_the_abi():
    from paper_2411_11547_gb300 import _build
    path = _build.build(debug=True)
    lib = ctypes.CDLL(path)
    names = _declared()
    assert "phmm_debug_check" in names and "phmm_forward" in names
    for n in names:
        assert hasattr(lib, n), n
    lib.phmm_debug_guard_offset.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p]
    off = ctypes.c_size_t()
    assert lib.phmm_debug_guard_offset(None, 0, ctypes.byref(off)) == -1  # EINVAL: no plan


def test_release_library_has_no_debug_checks():
    from paper_2411_11547_gb300 import _build, phmm
    _build.build()
    L = ctypes.CDLL(_build.LIB)
    L.phmm_debug_guard_offset.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p]
    L.phmm_debug_check.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
    off = ctypes.c_size_t()
    assert L.phmm_debug_guard_offset(None, 0, ctypes.byref(off)) == phmm.PHMM_ESTATE
    assert L.phmm_debug_check(None, None, None) == phmm.PHMM_ESTATE


CHILD = r"""
import ctypes, sys
import numpy as np, torch
sys.path.insert(0, sys.argv[1])
import oracle
from paper_2411_11547_gb300 import _build, phmm, synth
_build.build(debug=True)
L = phmm.lib()
assert L._name.endswith("libphmm_debug.so"), L._name
L.phmm_debug_guard_offset.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p]
L.phmm_debug_check.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
b = synth.random_pairs(7, 80, (1, 600), (1, 700), alphabet=b"ACGTN", related=0.5,
                       qual_dtype=np.float32)
plan = phmm.Plan(phmm.DeviceBatch(b))
y, fl = plan.forward()                      # raises PhmmError(PHMM_EGUARD) on a failed check
torch.cuda.synchronize()
want = oracle.forward_batch(b)
assert np.max(np.abs(y.cpu().numpy() - want)) <= 1e-3
dy = np.random.default_rng(1).uniform(-1, 1, len(want))
y2, _ = plan.forward_partials()
gb, gi, gd, gg = plan.backward_partials(torch.as_tensor(dy, device="cuda"))
wy, wb, wi, wd, wg = oracle.backward_batch(b, dy)
assert np.max(np.abs(y2.cpu().numpy() - wy)) <= 1e-3
assert abs(float(gg.cpu()[0]) - wg) <= 1e-3 * abs(wg) + 1e-9
# every guard intact after the calls; then one byte of a guard overwritten from the host
n = 0
off = ctypes.c_size_t()
while L.phmm_debug_guard_offset(plan.handle, n, ctypes.byref(off)) == 0:
    n += 1
assert n >= 10, n
ws = ctypes.c_void_p(plan._ws_ptr)
assert L.phmm_debug_check(plan.handle, ws, None) == 0
L.phmm_debug_guard_offset(plan.handle, n // 2, ctypes.byref(off))
w = plan.workspace
base = plan._ws_ptr - w.data_ptr()
w[base + off.value + 17] = 0
assert L.phmm_debug_check(plan.handle, ws, None) == phmm.PHMM_EGUARD
plan.forward()                              # refills the guards: the call passes its checks
assert L.phmm_debug_check(plan.handle, ws, None) == 0
print("debug build ok", n, "guards")
"""


@pytest.mark.gpu
def test_debug_build_on_gpu():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    env = dict(os.environ, PHMM_DEBUG="1")
    r = subprocess.run([sys.executable, "-c", CHILD, ROOT], env=env, capture_output=True,
                       text=True, timeout=900)
    assert r.returncode == 0, r.stdout[-2000:] + r.stderr[-4000:]
    assert "debug build ok" in r.stdout
