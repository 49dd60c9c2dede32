"""GPU parity of the FP64-accurate collapse paths (C-ABI through the binding) against the
oracle: CC_MODE_FP64 (FP64 unit) and CC_MODE_F32X2 (the same steps in float-float
arithmetic), both held to 1e-10 relative."""
import ctypes

import numpy as np
import pytest

import hessgen
import oracle
from parity import REL_TOL_FP64, compare_max, near_pair_corner_planes, oracle_per_radius, rel_err, running_max

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    import paper_2510_02873_gb300 as cc
    c = cc.Context(0.3, 0.7, 512, 1e-3, 1.0, device=0)
    yield c
    c.close()


@pytest.fixture(scope="module")
def tables():
    return oracle.Tables(0.3, 0.7, 512, 1e-3, 1.0)


def gpu_multi(ctx, stack: np.ndarray, sigma, plane_stride=None, scale_idx0=0, mode="fp64"):
    """Upload (R, 6, n) planes (optionally padded planes) and run one fused launch."""
    R, _, n = stack.shape
    ps = n if plane_stride is None else plane_stride
    dt = torch.float64 if stack.dtype == np.float64 else torch.float32
    buf = torch.zeros((R, 6, ps), dtype=dt, device="cuda")
    buf[:, :, :n] = torch.from_numpy(stack).cuda()
    view = buf[:, :, :n]
    F = torch.empty(n, dtype=torch.float64, device="cuda")
    idx = torch.empty(n, dtype=torch.int32, device="cuda")
    ctx.reset_max(F, idx)
    ctx.collapse_multi(view, sigma, F, idx, scale_idx0=scale_idx0, mode=mode)
    torch.cuda.synchronize()
    return F.cpu().numpy(), idx.cpu().numpy()


MODES = ["fp64", "f32x2"]


@pytest.mark.parametrize("mode", MODES)
def test_config1_fused_over_radii(ctx, tables, mode):
    """32^3 grid x 8 radii, s log-spaced 0.3 -> 4.0: every point, every radius."""
    n, R = 32 ** 3, 8
    sig = hessgen.sigma_schedule(R, 0.3, 4.0)
    stack = hessgen.hessian_stack(2511, 0, sig, n)
    F_all, fl = oracle_per_radius(tables, stack)
    F, idx = gpu_multi(ctx, stack, sig, mode=mode)
    s = compare_max(F, idx, F_all, fl)
    assert (idx >= 0).mean() > 0.3
    print("config1", mode, s)


def test_scale_by_scale_equals_fused(ctx):
    """R calls of cc_collapse_scale give exactly the fused launch's result."""
    n, R = 5000, 6
    sig = hessgen.sigma_schedule(R, 0.3, 4.0)
    stack = hessgen.hessian_stack(77, 1, sig, n)
    F_f, idx_f = gpu_multi(ctx, stack, sig)
    d = torch.from_numpy(stack).cuda()
    F = torch.empty(n, dtype=torch.float64, device="cuda")
    idx = torch.empty(n, dtype=torch.int32, device="cuda")
    ctx.reset_max(F, idx)
    for r in range(R):
        ctx.collapse_scale(d[r], sig[r], F, idx, r)
    torch.cuda.synchronize()
    assert np.array_equal(F.cpu().numpy(), F_f)
    assert np.array_equal(idx.cpu().numpy(), idx_f)


@pytest.mark.parametrize("mode", MODES)
@pytest.mark.parametrize("n", [1, 2, 31, 32, 33, 255, 257, 1023, 4097, 70001])
def test_ragged_sizes_and_padded_planes(ctx, tables, n, mode):
    R = 3
    sig = hessgen.sigma_schedule(R, 1.0, 5.0)
    stack = hessgen.hessian_stack(1000 + n, 0, sig, n)
    ps = n + (n % 2) + 2  # padded plane stride, 16-byte aligned planes
    F_all, fl = oracle_per_radius(tables, stack)
    F, idx = gpu_multi(ctx, stack, sig, plane_stride=ps, scale_idx0=5, mode=mode)
    compare_max(F, idx, F_all, fl, scale_idx0=5)


@pytest.mark.parametrize("mode", MODES)
def test_fp32_planes_in_fp64_mode(ctx, tables, mode):
    n, R = 20000, 4
    sig = hessgen.sigma_schedule(R, 0.5, 4.0)
    stack = hessgen.hessian_stack(31337, 2, sig, n, dtype=np.float32)
    F_all, fl = oracle_per_radius(tables, stack)
    F, idx = gpu_multi(ctx, stack, sig, mode=mode)
    compare_max(F, idx, F_all, fl)


def _planes_from_matrices(Ms):
    return np.stack([Ms[:, 0, 0], Ms[:, 1, 1], Ms[:, 2, 2], Ms[:, 0, 1], Ms[:, 0, 2], Ms[:, 1, 2]])


def _rotated(spectra, rng):
    Ms = []
    for lam in spectra:
        Q, _ = np.linalg.qr(rng.normal(size=(3, 3)))
        Ms.append(Q @ np.diag(lam) @ Q.T)
    return np.array(Ms)


@pytest.mark.parametrize("mode", MODES)
def test_degenerate_and_special_spectra(ctx, tables, mode):
    """Exact and near-exact degeneracies (the deflation branch), spherical,
    plane-wave, voids, collapse before the first knot (EdS branch), and axis-aligned."""
    rng = np.random.default_rng(5)
    spectra = []
    for s in (0.5, 2.0, 8.0):
        spectra += [[s, s, s], [s, 0, 0], [s, s, -s], [s, s, 0.3 * s], [s, -s, -s], [-s, -s, -s],
                    [s, 0.5 * s, 0.5 * s], [0.0, 0.0, 0.0]]
        for eps in (1e-4, 1e-6, 1e-8, 1e-10, 1e-12, 1e-14):
            spectra += [[s, s * (1 - eps), -0.4 * s], [s, 0.2 * s, 0.2 * s * (1 - eps)],
                        [s * (1 + eps), s, s * (1 - eps)]]
    spectra += [[900.0, 10.0, -5.0], [3000.0, 1.0, 1.0], [1.2, 0.1, 0.05], [1.0 + 1e-9, 0.0, 0.0]]
    Ms = _rotated(spectra, rng)
    Ms = np.concatenate([Ms, np.array([np.diag(l) for l in spectra])])
    planes = _planes_from_matrices(Ms)
    stack = planes[None]
    F_all, fl = oracle_per_radius(tables, stack)
    F, idx = gpu_multi(ctx, stack, [1.0], mode=mode)
    compare_max(F, idx, F_all, fl)


@pytest.mark.parametrize("mode", MODES)
def test_near_pair_threshold_corner(ctx, tables, mode):
    """Spectra just above the deflation threshold with small l1 against a
    large negative l3 (the FP64 eigenvalue stage's weakest case); most collapse."""
    stack = near_pair_corner_planes(3000, 23)
    F_all, fl = oracle_per_radius(tables, stack)
    F, idx = gpu_multi(ctx, stack, [1.0], mode=mode)
    s = compare_max(F, idx, F_all, fl)
    assert (F > 0).sum() > 1500
    print("near-pair corner", mode, s)


@pytest.mark.parametrize("mode", MODES)
def test_supported_eigenvalue_range_ends(ctx, tables, mode):
    """The header's supported range, eigenvalue magnitudes up to 1e6: random
    and structured spectra scaled to 1e-6 .. 1e6 (collapse from ~0.7 up, deep
    in the EdS segment at the top end; nothing collapses at the bottom end),
    in random frames and on the diagonal."""
    rng = np.random.default_rng(17)
    spectra = []
    for scale in (1e-6, 1e-3, 0.7, 30.0, 1e3, 1e5, 1e6):
        base = [[1.0, 0.3, -0.2], [1.0, 1.0, 1.0], [1.0, 0.0, 0.0], [0.6, -0.5, -1.0], [1.0, 1.0 - 1e-9, -0.4],
                [0.01, -0.9, -1.0]]
        base += list(-np.sort(-rng.normal(size=(40, 3)), axis=1))
        spectra += [list(np.asarray(b) * scale) for b in base]
    Ms = np.concatenate([_rotated(spectra, rng), np.array([np.diag(l) for l in spectra])])
    stack = _planes_from_matrices(Ms)[None]
    F_all, fl = oracle_per_radius(tables, stack)
    F, idx = gpu_multi(ctx, stack, [1.0], mode=mode)
    s = compare_max(F, idx, F_all, fl)
    m = len(spectra) // 7
    top = np.concatenate([np.arange(6 * m, 7 * m), len(spectra) + np.arange(6 * m, 7 * m)])
    bottom = np.concatenate([np.arange(m), len(spectra) + np.arange(m)])
    assert (F[top] > 1e4).sum() > m and np.all(F[bottom] == 0)
    print("eigenvalue range", mode, s)


@pytest.mark.parametrize("mode", MODES)
def test_non_finite_inputs_give_no_collapse(ctx, mode):
    n = 64
    stack = np.zeros((1, 6, n))
    stack[0, 0, :] = 2.0
    stack[0, :, ::4] = np.nan
    stack[0, 0, 1::4] = np.inf
    F, idx = gpu_multi(ctx, stack, [1.0], mode=mode)
    assert np.all(F[::4] == 0) and np.all(idx[::4] == -1)
    assert np.all(np.isfinite(F))


def test_stats_counters(ctx, tables):
    n, R = 9000, 3
    sig = hessgen.sigma_schedule(R, 0.5, 4.0)
    stack = hessgen.hessian_stack(4242, 0, sig, n)
    ctx.reset_stats()
    gpu_multi(ctx, stack, sig)
    st = ctx.stats()
    F_all, fl = oracle_per_radius(tables, stack)
    assert st["evaluations"] == n * R
    amb = int(((fl & oracle.FLAGS_AMBIGUOUS) != 0).sum())
    assert abs(st["collapsed"] - int((F_all > 0).sum())) <= amb
    assert st["eds_branch"] == int(((fl & oracle.FLAG_EDS) != 0).sum())
    assert st["error_flags"] == 0
    ctx.reset_stats()
    assert ctx.stats()["evaluations"] == 0


def test_invalid_arguments_are_rejected(ctx):
    import paper_2510_02873_gb300 as cc
    from paper_2510_02873_gb300 import _lib
    L = _lib.load()
    n = 64
    buf = torch.zeros(6 * n + 8, dtype=torch.float64, device="cuda")
    F = torch.zeros(n, dtype=torch.float64, device="cuda")
    idx = torch.zeros(n, dtype=torch.int32, device="cuda")
    h = ctx.handle
    p = buf.data_ptr()
    s = None
    # misaligned base, odd plane stride (8-byte planes), stride < n, bad dtype, bad sigma, bad R
    assert L.cc_collapse_scale(h, 0, p + 8, 8, n, n, 1.0, F.data_ptr(), idx.data_ptr(), 0, s) == _lib.CC_EINVAL
    assert L.cc_collapse_scale(h, 0, p, 8, n, n + 1, 1.0, F.data_ptr(), idx.data_ptr(), 0, s) == _lib.CC_EINVAL
    assert L.cc_collapse_scale(h, 0, p, 8, n, n - 1, 1.0, F.data_ptr(), idx.data_ptr(), 0, s) == _lib.CC_EINVAL
    assert L.cc_collapse_scale(h, 0, p, 2, n, n, 1.0, F.data_ptr(), idx.data_ptr(), 0, s) == _lib.CC_EINVAL
    assert L.cc_collapse_scale(h, 0, p, 8, n, n, 0.0, F.data_ptr(), idx.data_ptr(), 0, s) == _lib.CC_EINVAL
    assert L.cc_collapse_scale(h, 0, p, 8, n, n, 1.0, F.data_ptr(), idx.data_ptr(), -1, s) == _lib.CC_EINVAL
    assert L.cc_collapse_scale(h, 7, p, 8, n, n, 1.0, F.data_ptr(), idx.data_ptr(), 0, s) == _lib.CC_EINVAL
    assert L.cc_collapse_scale(h, 0, p, 8, n, n, 1.0, None, idx.data_ptr(), 0, s) == _lib.CC_EINVAL
    # empty input is a no-op in every mode, and an unknown mode is rejected even then
    for mode in range(6):
        assert L.cc_collapse_scale(h, mode, None, 8, 0, 0, 1.0, None, None, 0, s) == _lib.CC_OK
        sig2 = (ctypes.c_double * 2)(1.0, 2.0)
        assert L.cc_collapse_multi(h, mode, None, 4, 0, 0, 0, sig2, 2, None, None, 0, s) == _lib.CC_OK
    assert L.cc_collapse_scale(h, 7, None, 8, 0, 0, 1.0, None, None, 0, s) == _lib.CC_EINVAL
    with pytest.raises(cc.CollapseError):  # 8-byte plane stride
        ctx.collapse_scale(buf[:6 * (n + 1)].view(6, n + 1)[:, :n], 1.0, F, idx, 0)


@pytest.mark.parametrize("mode", MODES)
def test_host_buffer_entry_matches_device_path(ctx, mode):
    """cc_collapse_multi_host (pinned and pageable host planes) == cc_collapse_multi, bit for bit."""
    n, R = 100003, 5
    sig = hessgen.sigma_schedule(R, 0.4, 5.0)
    stack = hessgen.hessian_stack(555, 0, sig, n)
    F_d, idx_d = gpu_multi(ctx, np.ascontiguousarray(stack), sig, plane_stride=n + 3, mode=mode)
    for pinned in (True, False):
        host = torch.zeros((R, 6, n + 2), dtype=torch.float64, pin_memory=pinned)  # odd plane stride
        host[:, :, :n] = torch.from_numpy(stack)
        Fh = torch.zeros(n, dtype=torch.float64, pin_memory=pinned)
        ih = torch.full((n,), -1, dtype=torch.int32, pin_memory=pinned)
        import paper_2510_02873_gb300 as cc
        with pytest.raises(cc.CollapseError):
            ctx.collapse_multi_host(host[:, :, :n], sig, Fh, ih, mode=mode)  # 8-byte plane stride
        host2 = torch.zeros((R, 6, n + 3), dtype=torch.float64, pin_memory=pinned)
        host2[:, :, :n] = torch.from_numpy(stack)
        ctx.collapse_multi_host(host2[:, :, :n], sig, Fh, ih, mode=mode)
        assert np.array_equal(Fh.numpy(), F_d) and np.array_equal(ih.numpy(), idx_d)
        # a second call continues the running maximum (scale indices shifted)
        ctx.collapse_multi_host(host2[:, :, :n], sig, Fh, ih, scale_idx0=R, mode=mode)
        assert np.array_equal(Fh.numpy(), F_d) and np.array_equal(ih.numpy(), idx_d)


@pytest.mark.parametrize("mode", MODES)
def test_config2_full_size_sampled(ctx, tables, mode):
    """256^3 grid x 25 radii (FP64 planes, 20 GB resident), one fused launch as
    the bench times it; sampled points checked against the oracle one by one,
    and properties that hold at any size checked on every point."""
    import hessgen.device as hdev
    n, R = 256 ** 3, 25
    sig = hessgen.sigma_schedule(R, 0.2, 6.0)
    seed = 2510 + 2
    hess = torch.empty((R, 6, n), dtype=torch.float64, device="cuda")
    for r in range(R):
        hdev.fill(hess[r], seed, 0, r, sig[r])
    F = torch.empty(n, dtype=torch.float64, device="cuda")
    idx = torch.empty(n, dtype=torch.int32, device="cuda")
    ctx.reset_max(F, idx)
    ctx.reset_stats()
    ctx.collapse_multi(hess, sig, F, idx, mode=mode)
    torch.cuda.synchronize()
    st = ctx.stats()
    assert st["evaluations"] == n * R and st["error_flags"] == 0
    rng = np.random.default_rng(99)
    pts = np.unique(np.concatenate([rng.integers(0, n, 20000), [0, 1, n - 2, n - 1]]))
    pts_t = torch.from_numpy(pts).cuda()
    dev_planes = hess[:, :, pts_t].cpu().numpy()  # (R, 6, m) as generated on the device
    host_planes = np.stack([hessgen.hessian_points(seed, 0, r, sig[r], pts) for r in range(R)])
    # the two generators agree to a few ulps (Box-Muller transcendentals differ)
    scale = np.asarray(sig)[:, None, None]
    assert np.all(np.abs(dev_planes - host_planes) <= 1e-14 * scale)
    F_all, fl = oracle_per_radius(tables, host_planes)
    Fs = F.cpu().numpy()
    ids = idx.cpu().numpy()
    s = compare_max(Fs[pts], ids[pts], F_all, fl)
    # whole-grid properties
    assert np.all(np.isfinite(Fs)) and np.all(Fs >= 0)
    assert np.all((Fs == 0) == (ids == -1)) and ids.min() >= -1 and ids.max() < R
    assert (ids >= 0).mean() > 0.5
    print("config2 sampled", mode, s, st)
    del hess
    torch.cuda.empty_cache()


@pytest.mark.parametrize("mode", MODES)
def test_eds_segment_below_first_knot(ctx, tables, mode):
    """Fields strong enough that D_c falls below the first knot D_0 at some
    radii (a_c = a_0 D_c / D_0, taken through the spline's Horner scheme with
    that segment's coefficients): parity, and the same count of EdS-branch
    evaluations as the oracle."""
    D0 = tables.D[0]
    sig = [0.5 / D0, 1.5 / D0, 4.0 / D0]
    n = 4096
    stack = hessgen.hessian_stack(2600, 0, sig, n)
    F_all, fl = oracle_per_radius(tables, stack)
    n_eds = int(((fl & oracle.FLAG_EDS) != 0).sum())
    assert n_eds > 1000
    ctx.reset_stats()
    F, idx = gpu_multi(ctx, stack, sig, mode=mode)
    st = ctx.stats()
    s = compare_max(F, idx, F_all, fl)
    assert st["eds_branch"] == n_eds
    print("EdS segment", mode, s, "eds evaluations", n_eds)
