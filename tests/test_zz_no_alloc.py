"""damf_core_svd_noalloc: the core SVD for callers that cannot allocate device memory.

Such callers (a plugin that only receives input and output pointers, code that must not
call cudaMalloc) get their scratch from a static device array inside the library.  This
file sorts last so that a run stopping at the first failure has run every other test.
It compares the no-allocation entry point with damf_core_svd (caller workspace) through
the C ABI, on two calls in a row with different inputs.  Both run the same deterministic
kernels on the same inputs, so their outputs must be equal bit for bit; the sizes include
the array's limit (d + r = 256) and a small d with the largest r.
"""

import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _core(rng, d, r):
    sigma = np.sort(rng.uniform(2.0, 40.0, d))[::-1].astype(np.float32)
    L = np.vstack([0.05 * rng.standard_normal((d, r)), np.triu(rng.standard_normal((r, r))) + np.eye(r)])
    R = np.vstack([0.05 * rng.standard_normal((d, r)), np.triu(rng.standard_normal((r, r))) + np.eye(r)])
    return sigma, L.astype(np.float32), R.astype(np.float32)


@pytest.mark.parametrize("d,r", [(128, 64), (128, 128), (16, 128)])
def test_noalloc_matches_workspace_entry_point_twice(d, r):
    import torch
    from paper_2306_08967_gb300 import _lib
    lib = _lib.load()
    rng = np.random.default_rng(2024 + d + r)
    m = d + r
    p = lambda t: ctypes.c_void_p(t.data_ptr())
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    nbytes = int(lib.damf_core_svd_workspace_size(d, r))
    ws = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
    for call in range(2):                    # the static scratch keeps the previous call's data
        sigma, L, R = (torch.from_numpy(a).cuda() for a in _core(rng, d, r))
        outs = []
        for noalloc in (False, True):
            E = torch.full((m, d), float("nan"), device="cuda")
            H = torch.full((m, d), float("nan"), device="cuda")
            th = torch.full((d,), float("nan"), device="cuda")
            status = torch.full((1,), -1, dtype=torch.int32, device="cuda")
            if noalloc:
                st = lib.damf_core_svd_noalloc(p(sigma), p(L), p(R), d, r, p(E), p(H), p(th), p(status), stream)
            else:
                st = lib.damf_core_svd(p(sigma), p(L), p(R), d, r, p(E), p(H), p(th), p(ws), nbytes, p(status),
                                       stream)
            assert st == 0
            torch.cuda.synchronize()
            assert int(status.item()) == 0, (noalloc, call, int(status.item()))
            outs.append((E, H, th))
        (E0, H0, t0), (E1, H1, t1) = outs
        assert torch.isfinite(E1).all() and torch.isfinite(H1).all() and torch.isfinite(t1).all()
        assert torch.equal(t1, t0) and torch.equal(E1, E0) and torch.equal(H1, H0), (d, r, call)


def test_noalloc_rejects_cores_beyond_its_scratch():
    from paper_2306_08967_gb300 import _lib
    lib = _lib.load()
    # r = 129 exceeds the static scratch (d + r <= 256): refused before any device work
    dummy = ctypes.c_void_p(16)
    assert lib.damf_core_svd_noalloc(dummy, dummy, dummy, 128, 129, dummy, dummy, dummy, None, None) == 2
    assert lib.damf_core_svd_noalloc(dummy, dummy, dummy, 24, 8, dummy, dummy, dummy, None, None) == 1
