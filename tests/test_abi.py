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


def test_every_entry_point_turns_away_null_handles_without_gpu_work():
    # each call given NULL handles / pointers and zero sizes returns its documented answer on
    # the host (no CUDA call is reached; there is no GPU here): DAMF_ERR_INVALID for a status,
    # 0 or -1 for a count, a message for an error text; an empty multi-graph call is a no-op
    import subprocess
    import sys
    code = r'''
import ctypes, json, sys
sys.path.insert(0, sys.argv[1])
from paper_2306_08967_gb300 import _lib
lib = _lib.load()
out = {}
for name, (res, args) in sorted(_lib.SIGNATURES.items()):
    if name == "damf_debug_fail_allocations":
        continue
    vals = [0 if a in (ctypes.c_int32, ctypes.c_int64, ctypes.c_size_t, ctypes.c_double) else None for a in args]
    r = getattr(lib, name)(*vals)
    out[name] = r.decode() if isinstance(r, bytes) else r
print(json.dumps(out))
'''
    # a separate process: a NULL dereference fails this test instead of ending the session
    p = subprocess.run([sys.executable, "-c", code, ROOT], capture_output=True, text=True, timeout=120)
    assert p.returncode == 0, p.stderr[-2000:]
    import json
    out = json.loads(p.stdout.strip().splitlines()[-1])
    from paper_2306_08967_gb300 import _lib
    assert set(out) == set(_lib.SIGNATURES) - {"damf_debug_fail_allocations"}
    counts = {"damf_bytes_required": 0, "damf_rsvd_width": 0, "damf_core_svd_workspace_size": 0,
              "damf_num_nodes": 0, "damf_fleet_launches": 0, "damf_plan_slots": -1}
    empty_ok = {"damf_apply_edges_multi", "damf_step_multi"}      # zero graphs: nothing to do
    for name, r in out.items():
        if name in counts:
            assert r == counts[name], name
        elif name in empty_ok:
            assert r == 0, name
        elif name in ("damf_destroy", "damf_fleet_destroy"):
            assert r is None, name
        elif name in ("damf_last_error", "damf_fleet_last_error"):
            assert isinstance(r, str) and r, name
        else:
            assert r == 1, (name, r)                              # DAMF_ERR_INVALID


def test_bytes_required_grows_with_every_size():
    # admission control counts the state (four n_cap x d tables), the adjacency (m_cap entries)
    # and the workspaces: more rows, entries or rank never need fewer bytes
    from paper_2306_08967_gb300 import _lib, bytes_required, make_config
    _lib.load()
    base = dict(n=50_000, d=64, alpha=0.15, eps=1e-5, n_capacity=60_000, m_capacity=2_000_000)
    b0 = bytes_required(make_config(**base))
    assert b0 > 4 * 60_000 * 64 * 4 + 2_000_000 * 4       # at least the state and the entries
    for key, more in (("n_capacity", 120_000), ("m_capacity", 8_000_000), ("d", 128)):
        assert bytes_required(make_config(**dict(base, **{key: more}))) > b0, key
    assert bytes_required(make_config(**dict(base, directed=True))) > b0   # the reverse adjacency too
    assert bytes_required(make_config(**dict(base, n_capacity=40_000))) == 0   # capacity below n
