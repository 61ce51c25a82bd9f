"""CPU checks of the C ABI boundary: the library builds, loads and exports every symbol
include/*.h declares (no compute calls: there is no GPU here)."""

import ctypes
import glob
import os
import re

from tests.conftest import ROOT


def _declared():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        src = open(h).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        names |= set(re.findall(r"\b(damf_\w+)\s*\(", src))
    return names


def test_library_exports_every_declared_symbol():
    from paper_2306_08967_gb300 import build as b
    from paper_2306_08967_gb300 import _lib
    lib_path = b.build()
    lib = ctypes.CDLL(lib_path)
    declared = _declared()
    assert len(declared) >= 14
    missing = [n for n in sorted(declared) if not hasattr(lib, n)]
    assert not missing, missing
    # the binding declares a signature for each of them
    assert declared <= set(_lib.SIGNATURES), declared - set(_lib.SIGNATURES)


def test_host_side_config_checks():
    from paper_2306_08967_gb300 import _lib, make_config, bytes_required, rsvd_width
    _lib.load()
    cfg = make_config(1000, 16, 0.15, 1e-4, n_capacity=1100, nnz=10000)
    assert bytes_required(cfg) > 0
    assert rsvd_width(cfg) == 32
    bad = make_config(1000, 24, 0.15, 1e-4)          # d must be 16/32/64/128
    assert bytes_required(bad) == 0
    bad = make_config(1000, 16, 0.0, 1e-4)           # alpha in (0, 1]
    assert bytes_required(bad) == 0
    bad = make_config(1000, 16, 0.15, 1e-4)
    bad.threshold = 2                                # 0 absolute, 1 degree-scaled
    assert bytes_required(bad) == 0
    assert bytes_required(make_config(1000, 16, 0.15, 1e-4, threshold="degree")) > 0
    # the C2 workload fits easily in a GB300's HBM
    c2 = make_config(200_000, 128, 0.15, 1e-5, n_capacity=250_000, nnz=2_000_000)
    assert bytes_required(c2) < 2 << 30
    assert rsvd_width(c2) == 160


def test_init_rejects_bad_arguments_without_gpu_work():
    from paper_2306_08967_gb300 import _lib, make_config
    lib = _lib.load()
    cfg = make_config(10, 24, 0.15, 1e-4)
    h = ctypes.c_void_p()
    st = lib.damf_init_factorize(ctypes.byref(cfg), None, None, 0, None, None, ctypes.byref(h))
    assert st == 1 and not h.value                   # DAMF_ERR_INVALID, nothing created
    assert lib.damf_apply_edges(None, None, None, None, 0, 0, None) == 1
    assert lib.damf_ppr_refresh(None, None) == 1
    assert lib.damf_score_pairs(None, None, None, 0, 0, 0, None, None) == 1
    assert lib.damf_topk(None, None, 0, 1, 0, 0, None, None, None) == 1


def test_wait_selftest_rejects_bad_arguments_without_gpu_work():
    from paper_2306_08967_gb300 import _lib
    lib = _lib.load()
    st = ctypes.c_int32(-1)
    assert lib.damf_selftest_wait(2, 1000, ctypes.byref(st), None) == 1     # which: 0 or 1
    assert lib.damf_selftest_wait(0, 0, ctypes.byref(st), None) == 1        # limit >= 1
    assert lib.damf_selftest_wait(0, 1 << 40, ctypes.byref(st), None) == 1  # above the library's limit
    assert lib.damf_selftest_wait(0, 1000, None, None) == 1
    assert st.value == -1


def test_injected_allocation_failure_is_reported_and_cleaned_up_without_gpu_work():
    # fault injection on the host: the first device allocation of an init fails as cudaMalloc
    # out of memory does; init returns DAMF_ERR_CAPACITY, creates nothing, and the hook disarms
    from paper_2306_08967_gb300 import _lib, make_config
    lib = _lib.load()
    cfg = make_config(100, 16, 0.15, 1e-4, nnz=400)
    h = ctypes.c_void_p()
    lib.damf_debug_fail_allocations(0)
    st = lib.damf_init_factorize(ctypes.byref(cfg), ctypes.c_void_p(8), ctypes.c_void_p(8), 400, ctypes.c_void_p(8),
                                 None, ctypes.byref(h))
    assert st == 2 and not h.value                   # DAMF_ERR_CAPACITY, nothing created
    lib.damf_debug_fail_allocations(-1)


def test_checked_sources_compile():
    # the DAMF_CHECK variant (device bounds checks) of the kernels that carry checks compiles
    import subprocess
    import tempfile
    from paper_2306_08967_gb300 import build as b
    import concurrent.futures
    with tempfile.TemporaryDirectory() as td:
        def compile_one(src):
            cmd = [b.NVCC] + b.ARCH + b.FLAGS + ["-DDAMF_CHECK", "-c", os.path.join(b.CSRC, src), "-o",
                                                os.path.join(td, src + ".o")]
            subprocess.run(cmd, check=True, timeout=600)
        with concurrent.futures.ThreadPoolExecutor(2) as ex:
            list(ex.map(compile_one, ("ppr.cu", "update.cu")))
