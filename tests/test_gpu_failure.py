"""Failure detection without a GPU fault: the push's bounded waits, run against conditions
that never come true (a grid barrier short of one CTA; a queue position nobody fills while a
task is still counted), give up after their iteration limit, leave DAMF_ERR_TIMEOUT in the
device status for the host to read, and the device stays usable afterwards."""

import ctypes
import time

import numpy as np
import pytest

from tests.gpu_util import make_pair

pytestmark = pytest.mark.gpu

DAMF_ERR_TIMEOUT = 5


@pytest.mark.parametrize("which", [0, 1])
def test_bounded_waits_give_up_and_report(which):
    from paper_2306_08967_gb300 import _lib
    lib = _lib.load()
    st = ctypes.c_int32(-1)
    t0 = time.perf_counter()
    assert lib.damf_selftest_wait(which, 200_000, ctypes.byref(st), None) == 0
    assert st.value == DAMF_ERR_TIMEOUT
    assert time.perf_counter() - t0 < 10.0
    # the device and the library stay usable: a graph initialises, updates and pushes
    g, _, _ = make_pair(400, 6.0, 2.5, 16, 0.15, 1e-4, 0xDA3F0000 + 600 + which, oracle=False)
    g.apply_edges(np.array([1, 2], np.int32), np.array([5, 9], np.int32), np.array([1, 1], np.int8))
    g.ppr_refresh()
    g.check()
    g.close()


@pytest.mark.parametrize("after", [0, 1, 7, 30])
def test_allocation_failure_at_any_point_frees_everything(after):
    # fault injection on the host: the after-th device allocation of an initialisation fails;
    # the call reports DAMF_ERR_CAPACITY, frees what it had taken (device memory back to where
    # it was) and the next initialisation works
    import torch
    from paper_2306_08967_gb300 import DamfError, _lib
    lib = _lib.load()
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    lib.damf_debug_fail_allocations(after)
    try:
        with pytest.raises(DamfError) as ex:
            make_pair(500, 6.0, 2.5, 32, 0.15, 1e-4, 0xDA3F0000 + 610, oracle=False)
        assert ex.value.code == 2
    finally:
        lib.damf_debug_fail_allocations(-1)
    torch.cuda.synchronize()
    assert abs(torch.cuda.mem_get_info()[0] - free0) < (8 << 20)
    g, _, _ = make_pair(500, 6.0, 2.5, 32, 0.15, 1e-4, 0xDA3F0000 + 611, oracle=False)
    g.check()
    g.close()


def test_checked_build_runs_the_parity_cases_clean():
    # the DAMF_CHECK build (device bounds checks that set DAMF_ERR_BOUNDS and skip the access)
    # must pass the push-heavy parity cases: no check fires on correct work
    import os
    import subprocess
    import sys
    from tests.conftest import ROOT
    subprocess.run([sys.executable, "-c", "from paper_2306_08967_gb300 import build; build.build(check=True)"],
                   check=True, cwd=ROOT, timeout=900)
    env = dict(os.environ, DAMF_LIB_VARIANT="check")
    out = subprocess.run([sys.executable, "-m", "pytest", "tests/test_gpu_parity.py", "-q", "-x", "-p",
                          "no:cacheprovider", "-k", "ppr or hub or overflow or multi or deletion or bruteforce or captured"],
                         env=env, cwd=ROOT, capture_output=True, text=True, timeout=900)
    assert out.returncode == 0, out.stdout[-3000:]
    assert " passed" in out.stdout
