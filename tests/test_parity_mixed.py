"""GPU parity of the mixed-precision path (CC_MODE_MIXED) against the FP64 oracle.

Mixed mode computes in FP32 and keeps FP64 for the (nearly) degenerate
eigenvalues, the collapse-root polish and the a(D) spline; its bound is 3e-5
relative on F (the paper's ~0.003 % interpolation residual). The oracle runs
on the same FP32 values widened to FP64.
"""
import numpy as np
import pytest

import hessgen
import oracle
from parity import oracle_per_radius, rel_err, running_max

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

REL_TOL_MIXED = 3e-5


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


def run_mixed(ctx, stack, sigma, plane_stride=None):
    R, _, n = stack.shape
    ps = n if plane_stride is None else plane_stride
    dt = torch.float32 if stack.dtype == np.float32 else torch.float64
    buf = torch.zeros((R, 6, ps), dtype=dt, device="cuda")
    buf[:, :, :n] = torch.from_numpy(stack).cuda()
    F = torch.empty(n, dtype=torch.float64, device="cuda")
    idx = torch.empty(n, dtype=torch.int32, device="cuda")
    ctx.reset_max(F, idx)
    ctx.reset_stats()
    ctx.collapse_multi(buf[:, :, :n], sigma, F, idx, mode="mixed")
    torch.cuda.synchronize()
    return F.cpu().numpy(), idx.cpu().numpy(), ctx.stats()


def compare_mixed(F, idx, F_all, flags_all, tol=REL_TOL_MIXED):
    F_ref, idx_ref = running_max(F_all)
    amb = (flags_all & oracle.FLAGS_AMBIGUOUS).any(axis=0)
    srt = np.sort(F_all, axis=0)
    tie = np.zeros_like(amb)
    if F_all.shape[0] > 1:
        tie = (srt[-1] > 0) & (srt[-1] - srt[-2] <= 2 * tol * srt[-1])
    # points whose best radius sits within the tolerance of the a_max edge may
    # legitimately flip between F ~ 1 and no collapse
    edge = ((F_ref > 0) & (F_ref < 1.0 + 4 * tol)) | ((F > 0) & (F < 1.0 + 4 * tol))
    ok = ~amb & ~edge
    err = rel_err(F, F_ref)
    worst = float(err[ok].max())
    assert worst <= tol, f"max relative F error {worst:.3e} > {tol:.1e}"
    mism = int((idx[ok & ~tie] != idx_ref[ok & ~tie]).sum())
    assert mism == 0, f"{mism} argmax mismatches outside ties"
    assert np.all(np.isfinite(F)) and np.all(F >= 0)
    return {"max_rel_err": worst, "rms_rel_err": float(np.sqrt(np.mean(err[ok] ** 2))),
            "ambiguous": int(amb.sum()), "edge": int(edge.sum()), "ties": int(tie.sum())}


def test_mixed_one_launch_per_radius_matches_fused(ctx):
    """One cc_collapse_scale launch per radius (F_max/idx updated in HBM each
    time) stores the same F as the fused launch, bit for bit; idx may differ
    only where two radii give the same FP32 reciprocal F (the per-radius
    pattern keeps the first of them, the fused launch the one with the
    smaller FP64 a): both radii then reach the stored F on their own."""
    n, R = 100000, 8  # 16-byte FP32 planes
    sig = hessgen.sigma_schedule(R, 0.2, 6.0)
    stack = hessgen.hessian_stack(2541, 0, sig, n, dtype=np.float32)
    buf = torch.from_numpy(stack).cuda()
    F1 = torch.empty(n, dtype=torch.float64, device="cuda")
    i1 = torch.empty(n, dtype=torch.int32, device="cuda")
    ctx.reset_max(F1, i1)
    for r in range(R):
        ctx.collapse_scale(buf[r], sig[r], F1, i1, r, mode="mixed")
    F2 = torch.empty_like(F1)
    i2 = torch.empty_like(i1)
    ctx.reset_max(F2, i2)
    ctx.collapse_multi(buf, sig, F2, i2, mode="mixed")
    Fr = np.empty((R, n))
    Fo, io = torch.empty_like(F1), torch.empty_like(i1)
    for r in range(R):
        ctx.reset_max(Fo, io)
        ctx.collapse_scale(buf[r], sig[r], Fo, io, r, mode="mixed")
        torch.cuda.synchronize()
        Fr[r] = Fo.cpu().numpy()
    F1, i1, F2, i2 = (t.cpu().numpy() for t in (F1, i1, F2, i2))
    assert np.array_equal(F1, F2)
    d = np.nonzero(i1 != i2)[0]
    assert np.all(i1[d] < i2[d])
    assert np.array_equal(Fr[i1[d], d], F1[d]) and np.array_equal(Fr[i2[d], d], F1[d])
    print("mixed per-radius vs fused: idx differs on", len(d), "FP32 ties of", n)


def test_mixed_fp32_planes_32cube_x8(ctx, tables):
    n, R = 32 ** 3, 8
    sig = hessgen.sigma_schedule(R, 0.2, 6.0)
    stack = hessgen.hessian_stack(2513, 0, sig, n, dtype=np.float32)
    F_all, fl = oracle_per_radius(tables, stack)
    F, idx, st = run_mixed(ctx, stack, sig)
    s = compare_mixed(F, idx, F_all, fl)
    assert st["evaluations"] == n * R
    assert st["fp64_branch"] < 0.03 * n * R
    print("mixed 32^3 x 8", s, "fp64 fraction", st["fp64_branch"] / (n * R))


@pytest.mark.parametrize("s", [0.5, 2.0, 6.0, 12.0])
def test_mixed_single_radius_many_points(ctx, tables, s):
    n = 200003
    stack = hessgen.hessian_stack(77 + int(s * 10), 1, [s], n, dtype=np.float32)
    F_all, fl = oracle_per_radius(tables, stack)
    F, idx, st = run_mixed(ctx, stack, [s], plane_stride=n + 1)
    compare_mixed(F, idx, F_all, fl)


def test_mixed_fp64_planes(ctx, tables):
    """FP64 planes in mixed mode are rounded to FP32 at load; still within 3e-5
    of the oracle on the FP64 values."""
    n, R = 50000, 4
    sig = hessgen.sigma_schedule(R, 0.5, 5.0)
    stack = hessgen.hessian_stack(4040, 0, sig, n)
    F_all, fl = oracle_per_radius(tables, stack)
    F, idx, st = run_mixed(ctx, stack, sig)
    compare_mixed(F, idx, F_all, fl)


def test_mixed_degenerate_spectra(ctx, tables):
    rng = np.random.default_rng(11)
    spectra = []
    for s in (0.5, 2.0, 8.0):
        spectra += [[s, s, s], [s, 0, 0], [s, s, -s], [s, -s, -s], [0.05 * s, 0.04 * s, -2 * s]]
        for eps in (1e-2, 1e-3, 1e-4, 1e-5, 1e-6, 1e-7):
            spectra += [[s, s * (1 - eps), -0.4 * s], [s, 0.2 * s, 0.2 * s * (1 - eps)],
                        [s * (1 + eps), s, s * (1 - eps)], [0.03 * s, 0.03 * s * (1 - eps), -3 * s]]
    Ms = []
    for lam in spectra:
        Q, _ = np.linalg.qr(rng.normal(size=(3, 3)))
        Ms.append(Q @ np.diag(lam) @ Q.T)
    Ms = np.array(Ms)
    planes = np.stack([Ms[:, 0, 0], Ms[:, 1, 1], Ms[:, 2, 2], Ms[:, 0, 1], Ms[:, 0, 2], Ms[:, 1, 2]])
    stack = planes[None].astype(np.float32)
    F_all, fl = oracle_per_radius(tables, stack)
    n = stack.shape[2]
    F, idx, st = run_mixed(ctx, stack, [1.0], plane_stride=(n + 3) // 4 * 4)
    compare_mixed(F, idx, F_all, fl)


def test_mixed_config3_full_size_sampled(ctx, tables):
    """512^3 x 30 radii, FP32 planes (96.6 GB resident), one fused launch;
    sampled points against the oracle one by one."""
    import hessgen.device as hdev
    n, R = 512 ** 3, 30
    sig = hessgen.sigma_schedule(R, 0.2, 6.0)
    seed = 2510 + 3
    hess = torch.empty((R, 6, n), dtype=torch.float32, device="cuda")
    for r in range(R):
        hdev.fill(hess[r], seed, 0, r, sig[r])
    F = torch.empty(n, dtype=torch.float64, device="cuda")
    idx = torch.empty(n, dtype=torch.int32, device="cuda")
    ctx.reset_max(F, idx)
    ctx.reset_stats()
    ctx.collapse_multi(hess, sig, F, idx, mode="mixed")
    torch.cuda.synchronize()
    st = ctx.stats()
    assert st["evaluations"] == n * R and st["error_flags"] == 0
    rng = np.random.default_rng(5)
    pts = np.unique(np.concatenate([rng.integers(0, n, 12000), [0, n - 1]]))
    pts_t = torch.from_numpy(pts).cuda()
    dev_planes = hess[:, :, pts_t].cpu().numpy()
    host_planes = np.stack([hessgen.hessian_points(seed, 0, r, sig[r], pts, dtype=np.float32) for r in range(R)])
    diff = np.abs(dev_planes.astype(np.float64) - host_planes.astype(np.float64))
    assert np.all(diff <= np.spacing(np.abs(host_planes)).astype(np.float64) * 1.0001)
    F_all, fl = oracle_per_radius(tables, host_planes)
    s = compare_mixed(F.cpu().numpy()[pts], idx.cpu().numpy()[pts], F_all, fl)
    Fs = F.cpu().numpy()
    assert np.all(np.isfinite(Fs)) and np.all(Fs >= 0)
    print("config3 sampled", s, st, "fp64 fraction", st["fp64_branch"] / (n * R))
    del hess
    torch.cuda.empty_cache()


def _degenerate_matrices(rng, scales=(0.5, 2.0, 8.0)):
    spectra = []
    for s in scales:
        spectra += [[s, s, s], [s, 0, 0], [s, s, -s], [s, -s, -s], [0.05 * s, 0.04 * s, -2 * s]]
        for eps in (1e-2, 1e-3, 1e-4, 1e-5, 1e-6, 1e-7):
            spectra += [[s, s * (1 - eps), -0.4 * s], [s, 0.2 * s, 0.2 * s * (1 - eps)],
                        [s * (1 + eps), s, s * (1 - eps)], [0.03 * s, 0.03 * s * (1 - eps), -3 * s]]
    Ms = []
    for lam in spectra:
        Q, _ = np.linalg.qr(rng.normal(size=(3, 3)))
        Ms.append(Q @ np.diag(lam) @ Q.T)
    Ms = np.array(Ms)
    return np.stack([Ms[:, 0, 0], Ms[:, 1, 1], Ms[:, 2, 2], Ms[:, 0, 1], Ms[:, 0, 2], Ms[:, 1, 2]])


def test_mixed_deferred_queue_overflow_and_ties(ctx, tables):
    """Points that are mostly 'hard' (FP64 refinement or the whole FP64 path)
    at every radius, so nearly every point leaves the main kernel as a record,
    and the same matrices at every radius make every collapsing point an exact
    tie, which the earliest radius must win."""
    rng = np.random.default_rng(23)
    hard = _degenerate_matrices(rng)                      # 6 x 87
    easy = hessgen.hessian_stack(31, 0, [1.0], 100)[0]    # 6 x 100 (FP64)
    planes = np.concatenate([hard] * 3 + [easy] + [hard] * 3, axis=1)
    perm = rng.permutation(planes.shape[1])
    planes = planes[:, perm].astype(np.float32)
    R = 12
    stack = np.repeat(planes[None], R, axis=0)
    F_all, fl = oracle_per_radius(tables, stack[:1])
    F, idx, st = run_mixed(ctx, stack, [1.0] * R, plane_stride=(planes.shape[1] + 3) // 4 * 4)
    F_ref = F_all[0]
    amb = (fl[0] & oracle.FLAGS_AMBIGUOUS) != 0
    edge = ((F_ref > 0) & (F_ref < 1.0 + 4 * REL_TOL_MIXED)) | ((F > 0) & (F < 1.0 + 4 * REL_TOL_MIXED))
    ok = ~amb & ~edge
    assert float(rel_err(F, F_ref)[ok].max()) <= REL_TOL_MIXED
    assert np.all(idx[F > 0] == 0), "exact ties must keep the earliest radius"
    assert np.all(idx[F == 0] == -1)
    assert st["evaluations"] == planes.shape[1] * R
    # the hard share is large: most points carry hard radii
    assert st["fp64_branch"] > 0.15 * planes.shape[1] * R


def test_mixed_deferred_mixed_radii(ctx, tables):
    """Hard matrices scattered over random (point, radius) cells of a random
    field: a point's hard radii (second kernel) and its other radii (main
    kernel) meet in the running maximum out of radius order."""
    rng = np.random.default_rng(29)
    n, R = 3000, 9
    sig = hessgen.sigma_schedule(R, 0.3, 5.0)
    stack = hessgen.hessian_stack(2529, 0, sig, n, dtype=np.float32)
    hard = _degenerate_matrices(rng).astype(np.float32)
    cells = rng.integers(0, n * R, 2500)
    for c, j in zip(cells, rng.integers(0, hard.shape[1], cells.size)):
        r, p = divmod(int(c), n)
        stack[r, :, p] = hard[:, j] * np.float32(sig[r])
    F_all, fl = oracle_per_radius(tables, stack)
    F, idx, st = run_mixed(ctx, stack, sig, plane_stride=n + 4)
    s = compare_mixed(F, idx, F_all, fl)
    print("mixed, scattered hard cells", s, "fp64 fraction", st["fp64_branch"] / (n * R))


def _batch_mixed(ctx, stack, sig, ps):
    """The same planes through the batched kernel: F_max, idx and the counters."""
    import paper_2510_02873_gb300 as cc
    R, _, n = stack.shape
    buf = torch.zeros((R, 6, ps), dtype=torch.float32, device="cuda")
    buf[:, :, :n] = torch.from_numpy(stack).cuda()
    F = torch.zeros(n, dtype=torch.float64, device="cuda")
    idx = torch.full((n,), -1, dtype=torch.int32, device="cuda")
    b = cc.Batch(ctx, [(buf[:, :, :n], sig, F, idx, 0)], mode="mixed")
    ctx.reset_stats()
    b.run()
    torch.cuda.synchronize()
    st = ctx.stats()
    b.close()
    return F.cpu().numpy(), idx.cpu().numpy(), st


def _mostly_hard(rng, n, sig, easy_share, seed):
    hard = _degenerate_matrices(rng)
    R = len(sig)
    cols = rng.integers(0, hard.shape[1], (R, n))
    stack = np.stack([hard[:, cols[r]] * sig[r] for r in range(R)]).astype(np.float32)
    easy = hessgen.hessian_stack(seed, 0, sig, n, dtype=np.float32)
    mix = rng.random((R, n)) < easy_share
    return np.where(mix[:, None, :], easy, stack).astype(np.float32)


def test_mixed_hard_record_overflow(ctx, tables):
    """A point's result does not depend on how its hard radii were finished.
    512 points alone all fit in the record buffer; the same 512 points after
    30,000 points that nearly all have hard radii (capacity n (0.006 R + 0.02)
    + 1024 = 2,732 at R = 6) mostly overflow and are recomputed in radius
    order: bit-identical either way. The long run also matches the batched
    kernel bit for bit, with the same counters, and the oracle within 3e-5."""
    rng = np.random.default_rng(37)
    sig = [0.6, 1.0, 1.4, 2.0, 2.8, 4.0]
    R = len(sig)
    a = _mostly_hard(rng, 512, sig, 0.4, 41)
    b = _mostly_hard(rng, 30000, sig, 0.05, 42)
    F1, i1, _ = run_mixed(ctx, a, sig, plane_stride=512)
    both = np.concatenate([b, a], axis=2)
    n = both.shape[2]
    F2, i2, st = run_mixed(ctx, both, sig, plane_stride=n)
    assert np.array_equal(F2[-512:], F1) and np.array_equal(i2[-512:], i1)
    Fb, ib, stb = _batch_mixed(ctx, both, sig, n)
    assert np.array_equal(F2, Fb) and np.array_equal(i2, ib)
    for k in ("evaluations", "collapsed", "eds_branch", "refined", "fp64_branch"):
        assert st[k] == stb[k], (k, st[k], stb[k])
    assert st["fp64_branch"] > 0.1 * n * R  # most points carry hard radii: far beyond the capacity
    F_all, fl = oracle_per_radius(tables, both)
    s = compare_mixed(F2, i2, F_all, fl)
    print("mixed, record overflow", s, st)


def test_mixed_hard_radii_above_32(ctx, tables):
    """40 radii with hard matrices on both sides of radius 32: radii below 32
    travel as bits of the record, the others are found again by the second
    and third kernels. Bit-identical to the batched kernel (its own main
    kernel and records), same counters, and within 3e-5 of the oracle."""
    rng = np.random.default_rng(43)
    n, R = 2500, 40
    sig = hessgen.sigma_schedule(R, 0.3, 5.0)
    stack = hessgen.hessian_stack(2543, 0, sig, n, dtype=np.float32)
    hard = _degenerate_matrices(rng).astype(np.float32)
    for _ in range(3000):
        p = int(rng.integers(0, n))
        r = int(rng.integers(24, R))
        stack[r, :, p] = hard[:, int(rng.integers(0, hard.shape[1]))] * np.float32(sig[r])
    ps = n + 4
    F, idx, st = run_mixed(ctx, stack, sig, plane_stride=ps)
    Fb, ib, stb = _batch_mixed(ctx, stack, sig, ps)
    assert np.array_equal(F, Fb) and np.array_equal(idx, ib)
    for k in ("evaluations", "collapsed", "eds_branch", "refined", "fp64_branch"):
        assert st[k] == stb[k], (k, st[k], stb[k])
    F_all, fl = oracle_per_radius(tables, stack)
    s = compare_mixed(F, idx, F_all, fl)
    assert (idx >= 32).sum() > 100
    print("mixed, hard radii above 32", s, st)


def test_mixed_eds_segment_below_first_knot(ctx, tables):
    """The mixed path's spline (FP32 tail, FP64 head) on the EdS segment below
    the first knot."""
    D0 = tables.D[0]
    sig = [0.5 / D0, 1.5 / D0, 4.0 / D0]
    n = 4096
    stack = hessgen.hessian_stack(2600, 0, sig, n, dtype=np.float32)
    F_all, fl = oracle_per_radius(tables, stack)
    n_eds = int(((fl & oracle.FLAG_EDS) != 0).sum())
    assert n_eds > 1000
    F, idx, st = run_mixed(ctx, stack, sig)
    s = compare_mixed(F, idx, F_all, fl)
    # a point within the tolerance of D_0 may land on either side
    assert abs(st["eds_branch"] - n_eds) <= 2
    print("mixed EdS segment", s, st["eds_branch"], n_eds)


def test_mixed_non_finite_inputs_give_no_collapse(ctx, tables):
    """NaN planes give no collapse and infinite ones a finite F (the FP32 ->
    FP64 widenings of the mixed finish skip the special cases); the clean
    points of the same warps keep their oracle values."""
    n = 256
    stack = np.zeros((1, 6, n), dtype=np.float32)
    stack[0, 0, :] = 2.0  # plane wave: l1 = 2, D_c = 1/2
    stack[0, :, ::4] = np.nan
    stack[0, 0, 1::4] = np.inf
    stack[0, 1, 3::8] = -np.inf
    F, idx, st = run_mixed(ctx, stack, [1.0])
    assert st["error_flags"] == 0
    assert np.all(np.isfinite(F)) and np.all(F >= 0)
    assert np.all(F[::4] == 0) and np.all(idx[::4] == -1)
    clean = np.arange(2, n, 4)
    F_all, fl = oracle_per_radius(tables, stack[:, :, clean].astype(np.float64))
    assert np.all(F_all[0] > 0)
    assert np.max(rel_err(F[clean], F_all[0])) <= REL_TOL_MIXED
