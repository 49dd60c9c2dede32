"""CC_MODE_EXACT_GROWTH (the collapse condition with the background's own
second- and third-order growth factors) against the oracle's exact-ratio
collapse, and its EdS limit against the FP64 path."""
import numpy as np
import pytest

import hessgen
import oracle
from parity import compare_max, near_pair_corner_planes

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def make_ctx(om, ol):
    import __graft_entry__
    __graft_entry__.build()
    import paper_2510_02873_gb300 as cc
    return cc.Context(om, ol, 512, 1e-3, 1.0, device=0)


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    c = make_ctx(0.3, 0.7)
    yield c
    c.close()


@pytest.fixture(scope="module")
def rtables():
    return oracle.RatioTables(0.3, 0.7, 512, 1e-3, 1.0)


def oracle_exact_per_radius(rt, stack):
    Fs, fl = [], []
    for r in range(stack.shape[0]):
        F, f = rt.F_points(stack[r])
        Fs.append(F)
        fl.append(f)
    return np.stack(Fs), np.stack(fl)


def gpu_multi(ctx, stack, sig, mode="exact_growth"):
    R, _, n = stack.shape
    buf = torch.zeros((R, 6, n + (n % 2)), dtype=torch.float64, device="cuda")  # 16-byte plane stride
    buf[:, :, :n] = torch.from_numpy(np.ascontiguousarray(stack)).cuda()
    F = torch.empty(n, dtype=torch.float64, device="cuda")
    idx = torch.empty(n, dtype=torch.int32, device="cuda")
    ctx.reset_max(F, idx)
    ctx.collapse_multi(buf[:, :, :n], sig, F, idx, mode=mode)
    torch.cuda.synchronize()
    return F.cpu().numpy(), idx.cpu().numpy()


def test_exact_growth_32cube_x8(ctx, rtables):
    n, R = 32 ** 3, 8
    sig = hessgen.sigma_schedule(R, 0.3, 4.0)
    stack = hessgen.hessian_stack(2521, 0, sig, n)
    F_all, fl = oracle_exact_per_radius(rtables, stack)
    F, idx = gpu_multi(ctx, stack, sig)
    s = compare_max(F, idx, F_all, fl)
    # the exact ratios move the result away from the EdS-ratio path
    F64, _ = gpu_multi(ctx, stack, sig, mode="fp64")
    both = (F > 0) & (F64 > 0)
    shift = np.abs(F[both] / F64[both] - 1.0)
    print("exact growth 32^3 x 8", s, "max shift vs EdS ratios", float(shift.max()))
    assert shift.max() > 1e-6


@pytest.mark.parametrize("n", [1, 33, 4097])
def test_exact_growth_ragged(ctx, rtables, n):
    R = 3
    sig = hessgen.sigma_schedule(R, 1.0, 5.0)
    stack = hessgen.hessian_stack(3000 + n, 0, sig, n)
    F_all, fl = oracle_exact_per_radius(rtables, stack)
    F, idx = gpu_multi(ctx, stack, sig)
    compare_max(F, idx, F_all, fl)


def test_exact_growth_special_spectra(ctx, rtables):
    rng = np.random.default_rng(6)
    spectra = []
    for s in (0.5, 2.0, 8.0):
        spectra += [[s, s, s], [s, 0, 0], [s, s, -s], [s, -s, -s], [-s, -s, -s], [0.0, 0.0, 0.0]]
        for eps in (1e-4, 1e-8, 1e-12):
            spectra += [[s, s * (1 - eps), -0.4 * s], [s * (1 + eps), s, s * (1 - eps)]]
    Ms = []
    for lam in spectra:
        Q, _ = np.linalg.qr(rng.normal(size=(3, 3)))
        Ms.append(Q @ np.diag(lam) @ Q.T)
    Ms = np.array(Ms)
    planes = np.stack([Ms[:, 0, 0], Ms[:, 1, 1], Ms[:, 2, 2], Ms[:, 0, 1], Ms[:, 0, 2], Ms[:, 1, 2]])[None]
    F_all, fl = oracle_exact_per_radius(rtables, planes)
    F, idx = gpu_multi(ctx, planes, [1.0])
    compare_max(F, idx, F_all, fl)


def test_exact_growth_near_pair_threshold_corner(ctx, rtables):
    """Spectra just above the deflation threshold with small l1 against a
    large negative l3 (the FP64 eigenvalue stage's weakest case)."""
    planes = near_pair_corner_planes(2000, 29)
    F_all, fl = oracle_exact_per_radius(rtables, planes)
    F, idx = gpu_multi(ctx, planes, [1.0])
    compare_max(F, idx, F_all, fl)
    assert (F > 0).sum() > 1000


def test_exact_growth_in_eds_is_the_rlpt_path():
    c = make_ctx(1.0, 0.0)
    n, R = 20000, 4
    sig = hessgen.sigma_schedule(R, 0.5, 4.0)
    stack = hessgen.hessian_stack(77, 3, sig, n)
    Fe, ie = gpu_multi(c, stack, sig)
    F6, i6 = gpu_multi(c, stack, sig, mode="fp64")
    c.close()
    nz = F6 > 0
    assert np.array_equal(Fe > 0, nz)
    assert np.abs(Fe[nz] / F6[nz] - 1.0).max() < 1e-12
    assert (ie != i6).sum() <= 2
