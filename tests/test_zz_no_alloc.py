"""cc_collapse_multi_noalloc: the entry point for callers that cannot allocate device memory.

Some callers cannot call cudaMalloc at all: code under CUDA stream capture,
code whose device memory belongs to another framework's allocator, or loops
that cannot take the implicit synchronisation of an allocation. For them the
library offers a context-free variant whose scratch (spline table, counters)
lives in a fixed static device array. This file checks, through the C-ABI,
that two calls in a row give the same F_max/idx as the regular entry point
(cc_collapse_multi on a context) within the FP64 tolerance, and that the
counters start from zero on every call. It is collected last so that a failure
here stops a `-x` run only after every other test has run; it also passes
alone in a fresh process.
"""
import ctypes

import numpy as np
import pytest

import hessgen

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

REL_TOL = 1e-10  # the FP64 path's tolerance


@pytest.fixture(scope="module")
def lib():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    from paper_2510_02873_gb300 import _lib
    return _lib


def _noalloc(lib, cosmo, hess, sigma, F, idx, scale_idx0=0):
    R, _, n = hess.shape
    sig = (ctypes.c_double * R)(*[float(s) for s in sigma])
    st = lib.CcStats()
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    rc = lib.load().cc_collapse_multi_noalloc(ctypes.byref(cosmo), 0, hess.data_ptr(), 8, n, hess.stride(1),
                                              hess.stride(0), sig, R, F.data_ptr(), idx.data_ptr(),
                                              scale_idx0, ctypes.byref(st), stream)
    lib.check(rc, "cc_collapse_multi_noalloc")
    return st.as_dict()


def _regular(ctx, hess, sigma, scale_idx0=0):
    n = hess.shape[2]
    F = torch.empty(n, dtype=torch.float64, device="cuda")
    idx = torch.empty(n, dtype=torch.int32, device="cuda")
    ctx.reset_max(F, idx)
    ctx.collapse_multi(hess, sigma, F, idx, scale_idx0=scale_idx0)
    torch.cuda.synchronize()
    return F.cpu().numpy(), idx.cpu().numpy()


def _check(F_got, idx_got, F_ref, idx_ref):
    F_got, idx_got = F_got.cpu().numpy(), idx_got.cpu().numpy()
    err = np.abs(F_got - F_ref) / np.where(F_ref > 0, F_ref, 1.0)
    assert err.max() <= REL_TOL
    assert np.array_equal(idx_got, idx_ref)


def test_noalloc_matches_regular_entry_on_two_calls(lib):
    import paper_2510_02873_gb300 as cc
    n, R = 70001, 6
    cosmos = [(0.3, 0.7, 512, 1e-3, 1.0), (0.25, 0.75, 700, 2e-3, 1.0)]
    for call, (om, ol, nk, amin, amax) in enumerate(cosmos):
        sig = hessgen.sigma_schedule(R, 0.5 + call, 5.0)
        stack = hessgen.hessian_stack(900 + call, 0, sig, n + 1)  # plane stride n + 1 (even)
        hess = torch.from_numpy(stack).cuda()[:, :, :n]
        with cc.Context(om, ol, nk, amin, amax) as ctx:
            F_ref, idx_ref = _regular(ctx, hess, sig)
        F = torch.zeros(n, dtype=torch.float64, device="cuda")
        idx = torch.full((n,), -1, dtype=torch.int32, device="cuda")
        cosmo = lib.CcCosmology(om, ol, nk, amin, amax)
        stats = _noalloc(lib, cosmo, hess, sig, F, idx)
        _check(F, idx, F_ref, idx_ref)
        assert stats["evaluations"] == n * R  # counters cleared at the start of the call
        assert stats["error_flags"] == 0
        # the same cosmology again: table already resident, counters cleared again
        F.zero_()
        idx.fill_(-1)
        stats = _noalloc(lib, cosmo, hess, sig, F, idx)
        _check(F, idx, F_ref, idx_ref)
        assert stats["evaluations"] == n * R


def test_noalloc_rejects_tables_beyond_its_static_size(lib):
    n = 64
    hess = torch.zeros((1, 6, n), dtype=torch.float64, device="cuda")
    F = torch.zeros(n, dtype=torch.float64, device="cuda")
    idx = torch.full((n,), -1, dtype=torch.int32, device="cuda")
    cosmo = lib.CcCosmology(0.3, 0.7, 1025, 1e-3, 1.0)
    sig = (ctypes.c_double * 1)(1.0)
    rc = lib.load().cc_collapse_multi_noalloc(ctypes.byref(cosmo), 0, hess.data_ptr(), 8, n, n, 6 * n, sig, 1,
                                              F.data_ptr(), idx.data_ptr(), 0, None, None)
    assert rc == lib.CC_EINVAL
    assert b"1024" in lib.load().cc_last_error_message()
