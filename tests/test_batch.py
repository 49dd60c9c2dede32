"""Batched persistent launch (cc_batch_*): many realizations of uneven size in one kernel."""
import numpy as np
import pytest

import hessgen
import oracle
from parity import compare_max, compare_reduced, oracle_per_radius

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def cc():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    import paper_2510_02873_gb300 as cc
    return cc


@pytest.fixture(scope="module")
def ctx(cc):
    c = cc.Context(0.3, 0.7, 512, 1e-3, 1.0, device=0)
    yield c
    c.close()


SIZES = [(17 ** 3, 3), (20 ** 3, 9), (1, 4), (31 ** 3, 5), (5, 2), (32 ** 3, 8), (24 ** 3, 6), (40 ** 3, 7),
         (48 ** 3, 3)]


def make_items(dtype=torch.float32, seed=31, fp64_item=True):
    items = []
    for k, (n, R) in enumerate(SIZES):
        sig = hessgen.sigma_schedule(R, 0.3 + 0.1 * k, 5.0)
        dt = torch.float64 if (fp64_item and k == 3) else dtype
        np_dt = np.float64 if dt == torch.float64 else np.float32
        ps = (n + 3) // 4 * 4  # 16-byte aligned planes for both dtypes
        buf = torch.zeros((R, 6, ps), dtype=dt, device="cuda")
        buf[:, :, :n] = torch.from_numpy(hessgen.hessian_stack(seed + k, k, sig, n, dtype=np_dt)).cuda()
        F = torch.zeros(n, dtype=torch.float64, device="cuda")
        idx = torch.full((n,), -1, dtype=torch.int32, device="cuda")
        items.append((buf[:, :, :n], sig, F, idx, 10 * k))
    return items


def reference(ctx, items, mode):
    out = []
    for hess, sig, F, idx, s0 in items:
        F2 = torch.zeros_like(F)
        i2 = torch.full_like(idx, -1)
        ctx.collapse_multi(hess, sig, F2, i2, scale_idx0=s0, mode=mode)
        out.append((F2, i2))
    torch.cuda.synchronize()
    return out


def reset(items):
    for _, _, F, idx, _ in items:
        F.zero_()
        idx.fill_(-1)


@pytest.mark.parametrize("mode", ["fp64", "mixed"])
def test_batch_equals_per_realization_launches(cc, ctx, mode):
    items = make_items()
    ref = reference(ctx, items, mode)
    b = cc.Batch(ctx, items, mode=mode)
    ctx.reset_stats()
    b.run()
    torch.cuda.synchronize()
    st = ctx.stats()
    assert st["evaluations"] == sum(n * R for n, R in SIZES)
    for (hess, sig, F, idx, s0), (F2, i2) in zip(items, ref):
        assert torch.equal(F, F2) and torch.equal(idx, i2)
    # graph capture on first use, replay afterwards: same results every time
    stream = torch.cuda.Stream()
    for _ in range(3):
        reset(items)
        with torch.cuda.stream(stream):
            b.run_graph(stream)
        stream.synchronize()
        for (hess, sig, F, idx, s0), (F2, i2) in zip(items, ref):
            assert torch.equal(F, F2) and torch.equal(idx, i2)
    b.close()


def test_batch_against_oracle(cc, ctx):
    items = make_items(dtype=torch.float64, seed=77, fp64_item=False)[:4]
    b = cc.Batch(ctx, items, mode="fp64")
    b.run()
    torch.cuda.synchronize()
    t = oracle.Tables(0.3, 0.7, 512, 1e-3, 1.0)
    for hess, sig, F, idx, s0 in items:
        stack = hess.cpu().numpy()
        F_all, fl = oracle_per_radius(t, stack)
        compare_max(F.cpu().numpy(), idx.cpu().numpy(), F_all, fl, scale_idx0=s0)
    b.close()


def test_autotune_and_cache(cc, ctx, tmp_path):
    items = make_items(seed=5)
    b = cc.Batch(ctx, items, mode="mixed")
    cache = str(tmp_path / "tune.txt")
    b.autotune(cache)
    blk, tiles = b.config()
    assert blk in (128, 256)
    assert all(t in (256, 512, 1024, 2048, 4096, 8192) and t >= blk for t in tiles)
    lines = open(cache).read().split("\n")
    assert any(" -1 " in line for line in lines)
    # a second plan takes the cached shapes and still computes the same values
    reset(items)
    b2 = cc.Batch(ctx, items, mode="mixed")
    b2.autotune(cache)
    assert b2.config() == (blk, tiles)
    ref = reference(ctx, items, "mixed")
    b2.run()
    torch.cuda.synchronize()
    for (hess, sig, F, idx, s0), (F2, i2) in zip(items, ref):
        assert torch.equal(F, F2) and torch.equal(idx, i2)
    b.close()
    b2.close()


def test_batch_rejects_bad_items(cc, ctx):
    items = make_items()[:2]
    hess, sig, F, idx, s0 = items[0]
    with pytest.raises(cc.CollapseError):
        cc.Batch(ctx, [(hess, [-1.0] * hess.shape[0], F, idx)], mode="mixed")
    with pytest.raises(cc.CollapseError):
        cc.Batch(ctx, items, mode="surrogate")


def test_batch_config4_full_size_sampled(cc, ctx):
    """The 48-realization workload as the bench times it: grids drawn from
    {64..384}^3 and 8..40 radii (seed 2514), FP32 planes (240 GB resident),
    mixed precision, autotuned tiles, one persistent launch replayed from a
    CUDA graph; sampled points of every realization against the oracle."""
    import hessgen.device as hdev
    rng = np.random.default_rng(2514)
    grids = rng.choice((64, 96, 128, 192, 256, 384), 48)
    radii = rng.integers(8, 41, 48)
    items = []
    for k, (g, R) in enumerate(zip(grids, radii)):
        n, R = int(g) ** 3, int(R)
        sig = hessgen.sigma_schedule(R, 0.2, 6.0)
        hess = torch.empty((R, 6, n), dtype=torch.float32, device="cuda")
        for r in range(R):
            hdev.fill(hess[r], 2514, k, r, sig[r])
        items.append((hess, sig, torch.zeros(n, dtype=torch.float64, device="cuda"),
                      torch.full((n,), -1, dtype=torch.int32, device="cuda")))
    b = cc.Batch(ctx, items, mode="mixed")
    stream = torch.cuda.Stream()
    b.autotune(None, stream)
    for _, _, F, idx in items:
        F.zero_()
        idx.fill_(-1)
    torch.cuda.synchronize()
    ctx.reset_stats()
    with torch.cuda.stream(stream):
        b.run_graph(stream)
    stream.synchronize()
    st = ctx.stats()
    assert st["evaluations"] == sum(int(g) ** 3 * int(R) for g, R in zip(grids, radii))
    assert st["error_flags"] == 0
    t = oracle.Tables(0.3, 0.7, 512, 1e-3, 1.0)
    pick = np.random.default_rng(6)
    worst = 0.0
    for k, (hess, sig, F, idx) in enumerate(items):
        n = hess.shape[2]
        pts = np.unique(np.concatenate([pick.integers(0, n, 150), [0, n - 1]]))
        host = np.stack([hessgen.hessian_points(2514, k, r, sig[r], pts, dtype=np.float32)
                         for r in range(len(sig))])
        dev = hess[:, :, torch.from_numpy(pts).cuda()].cpu().numpy()
        # the device and host generators agree to the last FP32 place
        assert np.all(np.abs(dev.astype(np.float64) - host) <= np.spacing(np.abs(host)).astype(np.float64) * 1.0001)
        F_all, fl = oracle_per_radius(t, host)
        s = compare_reduced(F.cpu().numpy()[pts], idx.cpu().numpy()[pts], F_all, fl)
        worst = max(worst, s["max_rel_err"])
    print("config 4 full size, sampled: max rel err", worst, st)
    b.close()
    del items
    torch.cuda.empty_cache()
