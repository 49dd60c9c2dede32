"""The learned surrogate: GPU training kernels vs the oracle's FP64 MLP, training
convergence, CC_MODE_SURROGATE parity, and what the network gains over the
method without it (the mixed path, whose closed-form cubic it replaces)."""
import time

import numpy as np
import pytest

import hessgen
import oracle
from parity import compare_reduced, oracle_per_radius, rel_err, running_max

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

REL_TOL = 3e-5


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


def init_like(rng):
    p = np.zeros(oracle.MLP_NPARAM)
    p[0:192] = rng.uniform(-1, 1, 192) * np.sqrt(3 / 3)
    p[256:4352] = rng.uniform(-1, 1, 4096) * np.sqrt(3 / 64)
    p[4416:8512] = rng.uniform(-1, 1, 4096) * np.sqrt(3 / 64)
    p[8576:8640] = rng.uniform(-1, 1, 64) * np.sqrt(3 / 64)
    p[192:256] = rng.normal(size=64) * 0.1
    p[4352:4416] = rng.normal(size=64) * 0.1
    p[8512:8576] = rng.normal(size=64) * 0.1
    p[8640] = 0.3
    return p.astype(np.float32)


def sample_inputs(rng, m):
    lam = np.sort(rng.normal(size=(m, 3)) * 1.2, axis=1)[:, ::-1]
    return np.ascontiguousarray(lam, dtype=np.float32)


def test_gpu_gradient_matches_oracle(ctx):
    """One minibatch through the BF16 tensor-core training kernel against the
    FP64 reference gradient of the same loss and parameters."""
    rng = np.random.default_rng(1)
    params = init_like(rng)
    ctx.load_surrogate(params, [-10, -10, -10, 10, 10, 10])
    z = sample_inputs(rng, 256)
    t = rng.normal(size=256).astype(np.float32)
    loss_g, grad_g = ctx.surrogate_grad(z, t)
    loss_o, grad_o = oracle.mlp_loss_grad(params.astype(np.float64), z.astype(np.float64), t.astype(np.float64))
    assert abs(loss_g - loss_o) <= 2e-2 * loss_o
    groups = {"W1": (0, 192), "b1": (192, 256), "W2": (256, 4352), "b2": (4352, 4416), "W3": (4416, 8512),
              "b3": (8512, 8576), "W4": (8576, 8640), "b4": (8640, 8641)}
    for name, (a, b) in groups.items():
        g, o = grad_g[a:b].astype(np.float64), grad_o[a:b]
        rel = np.linalg.norm(g - o) / np.linalg.norm(o)
        assert rel < 5e-2, (name, rel)
        if b - a > 1:
            cos = g @ o / (np.linalg.norm(g) * np.linalg.norm(o))
            assert cos > 0.998, (name, cos)


def test_gpu_forward_matches_oracle(ctx):
    rng = np.random.default_rng(2)
    params = init_like(rng)
    ctx.load_surrogate(params, [-10, -10, -10, 10, 10, 10])
    z = sample_inputs(rng, 1000 + 7)
    out = torch.empty(len(z), dtype=torch.float32, device="cuda")
    ctx.surrogate_eval(torch.from_numpy(z).cuda(), out)
    torch.cuda.synchronize()
    ref = oracle.mlp_forward(params.astype(np.float64), z.astype(np.float64))
    got = out.cpu().numpy()
    assert np.all(np.abs(got - ref) <= 3e-2 * (1 + np.abs(ref)))
    params2, hull = ctx.surrogate_params()
    np.testing.assert_array_equal(params2, params)


@pytest.fixture(scope="module")
def trained(ctx):
    """Train on 4M points of the isotropic field at s = 1 (about 2M collapsing samples)."""
    import hessgen.device as hdev
    n = 4 * 1024 * 1024
    h = torch.empty((6, n), dtype=torch.float32, device="cuda")
    hdev.fill(h, 777, 9, 0, 1.0)
    t0 = time.perf_counter()
    rep = ctx.surrogate_train(h, 1.0, steps=1500, batch=16384, lr=3e-3, seed=5)
    rep["seconds"] = time.perf_counter() - t0
    print("training", rep)
    del h
    torch.cuda.empty_cache()
    return rep


def test_training_converges(trained):
    rep = trained
    assert rep["samples"] > 1_000_000
    assert rep["loss_last"] < rep["loss_first"] / 20
    assert rep["val_rms"] < 5e-2
    lo, hi = np.array(rep["hull_lo"]), np.array(rep["hull_hi"])
    assert np.all(lo < hi) and lo[0] > 0


def compare(F, idx, F_all, fl, tol=REL_TOL):
    F_ref, idx_ref = running_max(F_all)
    amb = (fl & oracle.FLAGS_AMBIGUOUS).any(axis=0)
    edge = ((F_ref > 0) & (F_ref < 1.0 + 4 * tol)) | ((F > 0) & (F < 1.0 + 4 * tol))
    srt = np.sort(F_all, axis=0)
    tie = (srt[-1] > 0) & (srt[-1] - srt[-2] <= 2 * tol * srt[-1]) if F_all.shape[0] > 1 else np.zeros_like(amb)
    ok = ~amb & ~edge
    err = rel_err(F, F_ref)
    assert err[ok].max() <= tol
    assert np.array_equal(idx[ok & ~tie], idx_ref[ok & ~tie])
    return float(err[ok].max())


def run(ctx, stack, sig, mode):
    R, _, n = stack.shape
    d = torch.from_numpy(stack).cuda()
    F = torch.empty(n, dtype=torch.float64, device="cuda")
    idx = torch.empty(n, dtype=torch.int32, device="cuda")
    ctx.reset_max(F, idx)
    ctx.reset_stats()
    ctx.collapse_multi(d, sig, F, idx, mode=mode)
    torch.cuda.synchronize()
    return F.cpu().numpy(), idx.cpu().numpy(), ctx.stats()


@pytest.mark.parametrize("engine", ["mma_sync", "tcgen05"])
def test_surrogate_mode_parity(ctx, tables, trained, engine):
    n, R = 32 ** 3 + 76, 8  # a ragged last tile of 128 points (16-byte plane stride)
    sig = hessgen.sigma_schedule(R, 0.3, 6.0)
    stack = hessgen.hessian_stack(2516, 0, sig, n, dtype=np.float32)
    F_all, fl = oracle_per_radius(tables, stack)
    ctx.set_surrogate_engine(engine)
    try:
        F, idx, st = run(ctx, stack, sig, "surrogate")
    finally:
        ctx.set_surrogate_engine("tcgen05")
    worst = compare(F, idx, F_all, fl)
    frac = st["fallback"] / st["evaluations"]
    print("surrogate parity", engine, worst, "fallback fraction", frac, st)
    assert frac < 0.2
    assert st["error_flags"] == 0 and st["evaluations"] == n * R


def test_surrogate_engines_agree(ctx, trained):
    """Both kernels evaluate the same network (BF16 operands, FP32 sums in a
    different order): the seeds differ by a few BF16 roundings, the refined
    roots agree to the mixed tolerance and the same points collapse."""
    import hessgen.device as hdev
    n, R = 100004, 5  # ragged last tile, 16-byte plane stride
    sig = hessgen.sigma_schedule(R, 0.3, 6.0)
    h = torch.empty((R, 6, n), dtype=torch.float32, device="cuda")
    for r in range(R):
        hdev.fill(h[r], 919, 0, r, sig[r])
    out = {}
    for engine in ("mma_sync", "tcgen05"):
        ctx.set_surrogate_engine(engine)
        F = torch.empty(n, dtype=torch.float64, device="cuda")
        idx = torch.empty(n, dtype=torch.int32, device="cuda")
        ctx.reset_max(F, idx)
        ctx.reset_stats()
        ctx.collapse_multi(h, sig, F, idx, mode="surrogate")
        torch.cuda.synchronize()
        out[engine] = (F.cpu().numpy(), idx.cpu().numpy(), ctx.stats())
    ctx.set_surrogate_engine("tcgen05")
    (Fa, ia, sa), (Fb, ib, sb) = out["mma_sync"], out["tcgen05"]
    assert sa["error_flags"] == 0 and sb["error_flags"] == 0
    # away from the a_max edge (F ~ 1) the same points collapse
    edge = ((Fa > 0) & (Fa < 1.0 + 1.2e-4)) | ((Fb > 0) & (Fb < 1.0 + 1.2e-4))
    assert np.array_equal((Fa > 0)[~edge], (Fb > 0)[~edge])
    both = (Fa > 0) & (Fb > 0)
    assert np.all(np.abs(Fa[both] - Fb[both]) <= 3e-5 * Fa[both])
    print("engines: max rel diff", float(np.max(np.abs(Fa[both] - Fb[both]) / Fa[both])),
          "fallbacks", sa["fallback"], sb["fallback"])


def test_surrogate_gain_over_the_method_without_it(ctx, trained):
    """The network replaces the closed-form FP32 cubic of the mixed path as the
    Newton seed. Same planes through both: results agree to the mixed tolerance;
    the printed ratio is what the network gains (below 1 means it costs time)."""
    import hessgen.device as hdev
    n, R = 128 ** 3, 8
    sig = hessgen.sigma_schedule(R, 0.3, 6.0)
    h = torch.empty((R, 6, n), dtype=torch.float32, device="cuda")
    for r in range(R):
        hdev.fill(h[r], 818, 0, r, sig[r])
    times, outs = {}, {}
    for mode in ("mixed", "surrogate", "mixed", "surrogate"):
        F = torch.empty(n, dtype=torch.float64, device="cuda")
        idx = torch.empty(n, dtype=torch.int32, device="cuda")
        ctx.reset_max(F, idx)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        ctx.collapse_multi(h, sig, F, idx, mode=mode)
        e1.record()
        torch.cuda.synchronize()
        times[mode] = e0.elapsed_time(e1)
        outs[mode] = F.cpu().numpy()
    a, b = outs["mixed"], outs["surrogate"]
    both = (a > 1.0 + 1.2e-4) & (b > 1.0 + 1.2e-4)
    assert np.max(np.abs(a[both] - b[both]) / a[both]) <= 2 * REL_TOL
    gain = times["mixed"] / times["surrogate"]
    print(f"surrogate gain over the closed-form seed: {gain:.3f}x "
          f"(mixed {times['mixed']:.2f} ms, surrogate {times['surrogate']:.2f} ms)")
    assert gain > 0


@pytest.mark.parametrize("engine", ["mma_sync", "tcgen05"])
def test_surrogate_config5_full_size_sampled(ctx, tables, trained, engine):
    """768^3 grid x 40 radii of FP32 planes, streamed one radius at a time
    (10.9 GB each) through collapse_scale as the bench times them; sampled
    points against the oracle."""
    import hessgen.device as hdev
    n, R, seed = 768 ** 3, 40, 2518
    sig = hessgen.sigma_schedule(R, 0.2, 6.0)
    planes = torch.empty((6, n), dtype=torch.float32, device="cuda")
    F = torch.zeros(n, dtype=torch.float64, device="cuda")
    idx = torch.full((n,), -1, dtype=torch.int32, device="cuda")
    rng = np.random.default_rng(8)
    pts = np.unique(np.concatenate([rng.integers(0, n, 6000), [0, n - 1]]))
    pts_t = torch.from_numpy(pts).cuda()
    host = np.empty((R, 6, len(pts)), dtype=np.float32)
    ctx.set_surrogate_engine(engine)
    ctx.reset_stats()
    try:
        for r in range(R):
            hdev.fill(planes, seed, 0, r, sig[r])
            ctx.collapse_scale(planes, sig[r], F, idx, r, mode="surrogate")
            host[r] = hessgen.hessian_points(seed, 0, r, sig[r], pts, dtype=np.float32)
            dev = planes[:, pts_t].cpu().numpy()
            assert np.all(np.abs(dev.astype(np.float64) - host[r]) <=
                          np.spacing(np.abs(host[r])).astype(np.float64) * 1.0001)
        torch.cuda.synchronize()
    finally:
        ctx.set_surrogate_engine("tcgen05")
    st = ctx.stats()
    assert st["evaluations"] == n * R and st["error_flags"] == 0
    assert st["fallback"] < 0.01 * n * R
    F_all, fl = oracle_per_radius(tables, host)
    s = compare_reduced(F.cpu().numpy()[pts], idx.cpu().numpy()[pts], F_all, fl)
    print("config 5 full size, sampled", engine, s, "fallback fraction", st["fallback"] / (n * R))
    del planes
    torch.cuda.empty_cache()


@pytest.mark.parametrize("engine", ["mma_sync", "tcgen05"])
@pytest.mark.parametrize("n", [1, 100, 300])
def test_surrogate_small_and_fp64_planes(ctx, tables, trained, engine, n):
    """Fewer points than one tile (or one warp), FP64 planes (rounded to FP32
    at load, as the mixed path does), both engines."""
    R = 3
    sig = hessgen.sigma_schedule(R, 0.5, 4.0)
    stack = hessgen.hessian_stack(2560 + n, 0, sig, n)
    F_all, fl = oracle_per_radius(tables, stack.astype(np.float32))
    ps = (n + 1) // 2 * 2  # 16-byte plane stride for FP64
    buf = torch.zeros((R, 6, ps), dtype=torch.float64, device="cuda")
    buf[:, :, :n] = torch.from_numpy(stack).cuda()
    F = torch.empty(n, dtype=torch.float64, device="cuda")
    idx = torch.empty(n, dtype=torch.int32, device="cuda")
    ctx.reset_max(F, idx)
    ctx.reset_stats()
    ctx.set_surrogate_engine(engine)
    try:
        ctx.collapse_multi(buf[:, :, :n], sig, F, idx, mode="surrogate")
        torch.cuda.synchronize()
    finally:
        ctx.set_surrogate_engine("tcgen05")
    st = ctx.stats()
    assert st["evaluations"] == n * R and st["error_flags"] == 0
    compare_reduced(F.cpu().numpy(), idx.cpu().numpy(), F_all, fl)


@pytest.mark.parametrize("engine", ["mma_sync", "tcgen05"])
def test_surrogate_non_finite_inputs_give_no_collapse(ctx, tables, trained, engine):
    """NaN planes give no collapse, infinite ones a finite F, and the clean
    points of the same tile keep their oracle values, with either engine."""
    n = 256
    stack = np.zeros((1, 6, n), dtype=np.float32)
    stack[0, 0, :] = 2.0
    stack[0, 1, :] = -0.5
    stack[0, :, ::4] = np.nan
    stack[0, 0, 1::4] = np.inf
    h = torch.from_numpy(stack).cuda()
    F = torch.empty(n, dtype=torch.float64, device="cuda")
    idx = torch.empty(n, dtype=torch.int32, device="cuda")
    ctx.reset_max(F, idx)
    ctx.reset_stats()
    ctx.set_surrogate_engine(engine)
    try:
        ctx.collapse_multi(h, [1.0], F, idx, mode="surrogate")
        torch.cuda.synchronize()
    finally:
        ctx.set_surrogate_engine("tcgen05")
    assert ctx.stats()["error_flags"] == 0
    F, idx = F.cpu().numpy(), idx.cpu().numpy()
    assert np.all(np.isfinite(F)) and np.all(F >= 0)
    assert np.all(F[::4] == 0) and np.all(idx[::4] == -1)
    clean = np.concatenate([np.arange(2, n, 4), np.arange(3, n, 4)])
    F_all, fl = oracle_per_radius(tables, stack[:, :, clean].astype(np.float64))
    assert np.all(F_all[0] > 0)
    assert np.max(rel_err(F[clean], F_all[0])) <= REL_TOL


def test_surrogate_invalid_arguments_are_rejected(ctx):
    """Each surrogate entry point refuses what its header rules out: a fresh
    context has no network for CC_MODE_SURROGATE, eval, grad or params; the
    engine must be one of the two; loaded parameters must be finite and the
    hull ordered; training needs enough points and a valid configuration."""
    import paper_2510_02873_gb300 as cc
    from paper_2510_02873_gb300 import _lib
    L = _lib.load()
    fresh = cc.Context(0.3, 0.7, 512, 1e-3, 1.0, device=0)
    try:
        n = 64
        h = torch.zeros((1, 6, n), dtype=torch.float32, device="cuda")
        F = torch.empty(n, dtype=torch.float64, device="cuda")
        idx = torch.empty(n, dtype=torch.int32, device="cuda")
        fresh.reset_max(F, idx)
        with pytest.raises(cc.CollapseError):
            fresh.collapse_multi(h, [1.0], F, idx, mode="surrogate")
        z = torch.zeros((n, 3), dtype=torch.float32, device="cuda")
        out = torch.empty(n, dtype=torch.float32, device="cuda")
        with pytest.raises(cc.CollapseError):
            fresh.surrogate_eval(z, out)
        with pytest.raises(cc.CollapseError):
            fresh.surrogate_grad(np.zeros((n, 3)), np.zeros(n))
        with pytest.raises(cc.CollapseError):
            fresh.surrogate_params()
        assert L.cc_set_surrogate_engine(fresh.handle, 2) == _lib.CC_EINVAL
        assert L.cc_set_surrogate_engine(fresh.handle, -1) == _lib.CC_EINVAL
        with pytest.raises(ValueError):
            fresh.set_surrogate_engine("wmma")
        p = np.zeros(cc.Context.MLP_NPARAM, dtype=np.float32)
        with pytest.raises(cc.CollapseError):
            fresh.load_surrogate(np.full_like(p, np.nan), [0, 0, 0, 1, 1, 1])
        with pytest.raises(cc.CollapseError):
            fresh.load_surrogate(p, [0, 0, 2, 1, 1, 1])
        small = torch.zeros((6, 512), dtype=torch.float32, device="cuda")
        with pytest.raises(cc.CollapseError):
            fresh.surrogate_train(small, 1.0, steps=1, batch=64)
        big = torch.zeros((6, 4096), dtype=torch.float32, device="cuda")
        with pytest.raises(cc.CollapseError):
            fresh.surrogate_train(big, 1.0, steps=1, batch=100)  # not a multiple of 64
        # after a valid load the calls work
        fresh.load_surrogate(p, [0, -1, -1, 1, 1, 1])
        fresh.surrogate_eval(z, out)
        torch.cuda.synchronize()
        assert torch.all(torch.isfinite(out))
    finally:
        fresh.close()


def test_checkpoint_restore_and_resume(ctx):
    """Training state round trip and resumption: a checkpoint restored into a
    fresh context reproduces the blob byte for byte and the network's outputs
    exactly; training resumed from it continues the loss curve (its first
    minibatch loss is near the last one before the checkpoint, far below a
    fresh start's) and ends at least as well as the uninterrupted run; a
    blob of another size, version or magic is refused."""
    import ctypes

    import hessgen.device as hdev
    import paper_2510_02873_gb300 as cc
    from paper_2510_02873_gb300 import _lib

    h = torch.empty((6, 2 * 1024 * 1024), dtype=torch.float32, device="cuda")
    hdev.fill(h, 777, 5, 0, 1.0)
    rep1 = ctx.surrogate_train(h, 1.0, steps=200, batch=8192, lr=3e-3, seed=5)
    blob = ctx.surrogate_checkpoint()
    z = torch.from_numpy(sample_inputs(np.random.default_rng(8), 4096)).cuda()
    f_a = torch.empty(4096, dtype=torch.float32, device="cuda")
    ctx.surrogate_eval(z, f_a)
    with cc.Context(0.3, 0.7, 512, 1e-3, 1.0, device=0) as c2:
        c2.surrogate_restore(blob)
        assert c2.surrogate_checkpoint() == blob
        f_b = torch.empty_like(f_a)
        c2.surrogate_eval(z, f_b)
        torch.cuda.synchronize()
        assert torch.equal(f_a, f_b)
        rep2 = c2.surrogate_train_resume(h, 1.0, steps=100, schedule_steps=300)
        # a continuation, not a restart
        assert rep2["loss_first"] < 3.0 * rep1["loss_last"] + 1e-4
        assert rep2["loss_first"] < 0.1 * rep1["loss_first"]
        assert rep2["val_rms"] <= 1.2 * rep1["val_rms"]
        assert len(c2.surrogate_checkpoint()) == len(blob)
        # refused blobs
        L = _lib.load()
        bad = bytearray(blob)
        bad[0] = ord("X")
        for b, code in ((bytes(bad), _lib.CC_EINVAL), (blob[:-4], _lib.CC_EINVAL)):
            buf = ctypes.create_string_buffer(b, len(b))
            assert L.cc_surrogate_restore(c2.handle, buf, len(b)) == code
        ver = bytearray(blob)
        ver[8] = 99  # version field
        buf = ctypes.create_string_buffer(bytes(ver), len(ver))
        assert L.cc_surrogate_restore(c2.handle, buf, len(ver)) == _lib.CC_ENOTSUP
    # loading bare parameters leaves nothing to resume
    params, hull = ctx.surrogate_params()
    ctx.load_surrogate(params, hull)
    with pytest.raises(cc.CollapseError):
        ctx.surrogate_checkpoint()
    with pytest.raises(cc.CollapseError):
        ctx.surrogate_train_resume(h, 1.0, steps=10)
    print("checkpoint", len(blob), "bytes; loss", rep1["loss_first"], rep1["loss_last"], "-> resumed",
          rep2["loss_first"], rep2["loss_last"], "val rms", rep1["val_rms"], rep2["val_rms"])
