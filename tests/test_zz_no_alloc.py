"""cc_collapse_multi_noalloc: the entry point for callers that cannot allocate device memory.

Some callers cannot call cudaMalloc: code whose device memory belongs to
another framework's caching allocator, or loops that cannot take the implicit
device synchronisation of an allocation. For them the library offers a
context-free variant whose scratch (spline table, counters) lives in a fixed
static device array. This file checks, through the C-ABI:
  - two calls in a row give F_max/idx bit for bit equal to the regular entry
    point (cc_collapse_multi on a context, same launch code and same table),
    and within the FP64 tolerance of the oracle;
  - the counters start from zero on every call;
  - tables up to the documented maximum of 1024 knots work, 1025 is rejected;
  - no call changes the device's free memory (after a first call has loaded the
    library's kernels);
  - FP32 planes give the regular entry point's result as well.
It is collected last so that a failure here stops a `-x` run only after every
other test has run; it also passes alone in a fresh process.
"""
import ctypes

import numpy as np
import pytest

import hessgen
import oracle
from parity import compare_max, oracle_per_radius

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def lib():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    from paper_2510_02873_gb300 import _lib
    return _lib


def _noalloc(lib, cosmo, hess, sigma, F, idx, scale_idx0=0, stats=True):
    R, _, n = hess.shape
    sig = (ctypes.c_double * R)(*[float(s) for s in sigma])
    st = lib.CcStats()
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    dtype = 8 if hess.dtype == torch.float64 else 4
    rc = lib.load().cc_collapse_multi_noalloc(ctypes.byref(cosmo), 0, hess.data_ptr(), dtype, n, hess.stride(1),
                                              hess.stride(0), sig, R, F.data_ptr(), idx.data_ptr(),
                                              scale_idx0, ctypes.byref(st) if stats else None, stream)
    lib.check(rc, "cc_collapse_multi_noalloc")
    return st.as_dict() if stats else None


def _regular(ctx, hess, sigma, scale_idx0=0):
    n = hess.shape[2]
    F = torch.empty(n, dtype=torch.float64, device="cuda")
    idx = torch.empty(n, dtype=torch.int32, device="cuda")
    ctx.reset_max(F, idx)
    ctx.collapse_multi(hess, sigma, F, idx, scale_idx0=scale_idx0)
    torch.cuda.synchronize()
    return F.cpu().numpy(), idx.cpu().numpy()


def _fresh_outputs(n):
    return (torch.zeros(n, dtype=torch.float64, device="cuda"), torch.full((n,), -1, dtype=torch.int32, device="cuda"))


COSMOS = [(0.3, 0.7, 512, 1e-3, 1.0), (0.25, 0.75, 700, 2e-3, 1.0), (0.3, 0.7, 1024, 1e-3, 1.0)]


def test_noalloc_matches_regular_entry_and_oracle_on_two_calls(lib):
    import paper_2510_02873_gb300 as cc
    n, R = 70001, 6
    for call, (om, ol, nk, amin, amax) in enumerate(COSMOS):
        sig = hessgen.sigma_schedule(R, 0.5 + call, 5.0)
        stack = hessgen.hessian_stack(900 + call, 0, sig, n + 1)  # plane stride n + 1 (even)
        hess = torch.from_numpy(stack).cuda()[:, :, :n]
        with cc.Context(om, ol, nk, amin, amax) as ctx:
            F_ref, idx_ref = _regular(ctx, hess, sig)
        cosmo = lib.CcCosmology(om, ol, nk, amin, amax)
        for repeat in range(2):  # the second call finds this cosmology's table resident
            F, idx = _fresh_outputs(n)
            stats = _noalloc(lib, cosmo, hess, sig, F, idx)
            torch.cuda.synchronize()
            assert np.array_equal(F.cpu().numpy(), F_ref), (nk, repeat)
            assert np.array_equal(idx.cpu().numpy(), idx_ref), (nk, repeat)
            assert stats["evaluations"] == n * R  # counters cleared at the start of every call
            assert stats["error_flags"] == 0
        # and against the oracle on a sample of points, for this cosmology's own tables
        t = oracle.Tables(om, ol, nk, amin, amax)
        pts = np.random.default_rng(call).choice(n, 3000, replace=False)
        F_all, fl = oracle_per_radius(t, np.ascontiguousarray(stack[:, :, pts]))
        compare_max(F.cpu().numpy()[pts], idx.cpu().numpy()[pts], F_all, fl)


def test_noalloc_allocates_no_device_memory(lib):
    n, R = 40000, 4
    sig = hessgen.sigma_schedule(R, 0.5, 4.0)
    hess = torch.from_numpy(hessgen.hessian_stack(77, 0, sig, n)).cuda()
    F, idx = _fresh_outputs(n)
    _noalloc(lib, lib.CcCosmology(*COSMOS[0]), hess, sig, F, idx)  # loads the kernels, looks up the array
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    for cos in (COSMOS[1], COSMOS[2], COSMOS[0]):  # every call uploads a new table into the static array
        _noalloc(lib, lib.CcCosmology(*cos), hess, sig, F, idx, stats=False)
        _noalloc(lib, lib.CcCosmology(*cos), hess, sig, F, idx)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0


def test_noalloc_fp32_planes(lib):
    import paper_2510_02873_gb300 as cc
    n, R = 30001, 3
    sig = hessgen.sigma_schedule(R, 0.5, 4.0)
    stack = hessgen.hessian_stack(4321, 0, sig, n + 3, dtype=np.float32)  # plane stride n + 3 (16-byte planes)
    hess = torch.from_numpy(stack).cuda()[:, :, :n]
    with cc.Context(*COSMOS[0]) as ctx:
        F_ref, idx_ref = _regular(ctx, hess, sig)
    for _ in range(2):
        F, idx = _fresh_outputs(n)
        _noalloc(lib, lib.CcCosmology(*COSMOS[0]), hess, sig, F, idx)
        torch.cuda.synchronize()
        assert np.array_equal(F.cpu().numpy(), F_ref) and np.array_equal(idx.cpu().numpy(), idx_ref)


def test_noalloc_rejects_tables_beyond_its_static_size(lib):
    n = 64
    hess = torch.zeros((1, 6, n), dtype=torch.float64, device="cuda")
    F, idx = _fresh_outputs(n)
    cosmo = lib.CcCosmology(0.3, 0.7, 1025, 1e-3, 1.0)
    sig = (ctypes.c_double * 1)(1.0)
    rc = lib.load().cc_collapse_multi_noalloc(ctypes.byref(cosmo), 0, hess.data_ptr(), 8, n, n, 6 * n, sig, 1,
                                              F.data_ptr(), idx.data_ptr(), 0, None, None)
    assert rc == lib.CC_EINVAL
    assert b"1024" in lib.load().cc_last_error_message()
