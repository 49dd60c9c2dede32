"""GPU parity of the tabulated mode and of the interpolation routines against the oracle."""
import numpy as np
import pytest

import hessgen
import oracle
from parity import REL_TOL_FP64, compare_max, near_pair_corner_planes, rel_err, running_max

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def table_axes(nd=128, nxy=64, d_max=40.0, xy_max=40.0):
    """Non-uniform axes, denser near zero (the paper samples delta non-uniformly)."""
    t = np.linspace(-1.0, 1.0, nd)
    dg = d_max * np.sinh(2.5 * t) / np.sinh(2.5)
    s = np.linspace(0.0, 1.0, nxy)
    xg = xy_max * (0.3 * s + 0.7 * s ** 2)
    return dg, xg, xg.copy()


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


@pytest.fixture(scope="module")
def table(ctx):
    dg, xg, yg = table_axes()
    val = oracle.tab_node_values(dg, xg, yg)
    ctx.set_table(dg, xg, yg, val)
    return oracle.Tab(dg, xg, yg, val), (dg, xg, yg, val)


def oracle_tab_per_radius(tables, tab, stack):
    Fs, fl = [], []
    for r in range(stack.shape[0]):
        F, f = tab.F_points(tables, stack[r].astype(np.float64))
        Fs.append(F)
        fl.append(f)
    return np.stack(Fs), np.stack(fl)


def run_tab(ctx, stack, sig, plane_stride=None):
    R, _, n = stack.shape
    ps = n if plane_stride is None else plane_stride
    buf = torch.zeros((R, 6, ps), dtype=torch.float64, device="cuda")
    buf[:, :, :n] = torch.from_numpy(stack).cuda()
    F = torch.empty(n, dtype=torch.float64, device="cuda")
    idx = torch.empty(n, dtype=torch.int32, device="cuda")
    ctx.reset_max(F, idx)
    ctx.reset_stats()
    ctx.collapse_multi(buf[:, :, :n], sig, F, idx, mode="tabulated")
    torch.cuda.synchronize()
    return F.cpu().numpy(), idx.cpu().numpy(), ctx.stats()


def test_tabulated_near_pair_threshold_corner(ctx, tables, table):
    """Spectra just above the deflation threshold with small l1 against a
    large negative l3: inside the table and, beyond it, the R-LPT fallback."""
    tab, _ = table
    stack = near_pair_corner_planes(2000, 31)
    F_all, fl = oracle_tab_per_radius(tables, tab, stack)
    F, idx, st = run_tab(ctx, stack, [1.0])
    compare_max(F, idx, F_all, fl)
    assert (F > 0).sum() > 1000


def test_tabulated_32cube_x8(ctx, tables, table):
    tab, _ = table
    n, R = 32 ** 3, 8
    sig = hessgen.sigma_schedule(R, 0.3, 16.0)  # the largest radii leave the +-40 table
    stack = hessgen.hessian_stack(2515, 0, sig, n)
    F_all, fl = oracle_tab_per_radius(tables, tab, stack)
    F, idx, st = run_tab(ctx, stack, sig)
    s = compare_max(F, idx, F_all, fl)
    outside = int(((fl & oracle.FLAG_HULL_OUT) != 0).sum())
    assert outside > 0  # the fallback is exercised
    print("tabulated 32^3 x 8", s, "outside", outside, st)


@pytest.mark.parametrize("n", [1, 33, 4097, 200003])
def test_tabulated_ragged(ctx, tables, table, n):
    tab, _ = table
    stack = hessgen.hessian_stack(4000 + n, 0, [3.0], n)
    F_all, fl = oracle_tab_per_radius(tables, tab, stack)
    F, idx, _ = run_tab(ctx, stack, [3.0], plane_stride=n + (n % 2))
    compare_max(F, idx, F_all, fl)


def test_tabulated_degenerate_spectra(ctx, tables, table):
    tab, _ = table
    rng = np.random.default_rng(21)
    spectra = []
    for s in (0.5, 3.0):
        spectra += [[s, s, s], [s, 0, 0], [s, 0.2 * s, 0.2 * s], [s, -s, -s], [0.05 * s, -s, -s]]
        for eps in (1e-3, 1e-6, 1e-9, 1e-12):
            spectra += [[s, s * (1 - eps), -0.4 * s], [s, 0.2 * s, 0.2 * s * (1 - eps)]]
    # a small l2 - l3 on a large trace (l2 + l3 >> l2 - l3): the cell
    # coordinates come from the traceless part, so nothing cancels against it
    spectra += [[10.5, 10.2, 10.0], [13.1, 13.0, 12.95], [13.0, 12.9, 12.9 - 1e-7]]
    Ms = np.array([(lambda Q: Q @ np.diag(l) @ Q.T)(np.linalg.qr(rng.normal(size=(3, 3)))[0]) for l in spectra])
    planes = np.stack([Ms[:, 0, 0], Ms[:, 1, 1], Ms[:, 2, 2], Ms[:, 0, 1], Ms[:, 0, 2], Ms[:, 1, 2]])
    stack = planes[None]
    F_all, fl = oracle_tab_per_radius(tables, tab, stack)
    n = stack.shape[2]
    F, idx, _ = run_tab(ctx, stack, [1.0], plane_stride=n + (n % 2))
    compare_max(F, idx, F_all, fl)


def test_tabulated_close_to_classic(ctx, table):
    """Same planes through the table and through the R-LPT root: they differ by
    interpolation error only."""
    n = 100000
    stack = hessgen.hessian_stack(99, 0, [2.0], n)
    F_t, _, st = run_tab(ctx, stack, [2.0])
    d = torch.from_numpy(stack).cuda()
    F = torch.empty(n, dtype=torch.float64, device="cuda")
    idx = torch.empty(n, dtype=torch.int32, device="cuda")
    ctx.reset_max(F, idx)
    ctx.collapse_multi(d, [2.0], F, idx, mode="fp64")
    F_c = F.cpu().numpy()
    both = (F_t > 0) & (F_c > 0)
    rel = np.abs(F_t - F_c)[both] / F_c[both]
    # interpolation error of a 128 x 64 x 64 table spanning +-40: ~2e-4 typical
    assert np.median(rel) < 1e-3 and np.quantile(rel, 0.99) < 2e-2


def test_device_table_nodes_match_oracle(ctx, table):
    """Node values u = 1/D_c, the largest root of P(u) = u^3 - l1 u^2 + c2 u + c3.
    Where that root is simple (relative condition number
    kappa = sum |terms of P| / |u P'(u)| below 1e4), GPU and oracle agree to
    1e-10 relative. Near a double or triple root (nodes with l1 <= 0, where u
    carries only the no-collapse sign, and the spherical corner) no method
    resolves the root beyond sqrt(eps) or cbrt(eps); there the GPU value must
    be a root to rounding: |P(u_gpu)| <= 1e-13 sum |terms of P(u_gpu)|."""
    _, (dg, xg, yg, val) = table
    got = ctx.table_nodes_rlpt(dg, xg, yg)
    d = dg[None, None, :]
    x = xg[:, None, None]
    y = yg[None, :, None]
    l2 = (d - x + y) / 3.0
    l1, l3 = l2 + x, l2 - y
    c1, c2 = -l1, -3.0 / 7.0 * l2 * l3
    c3 = l1 * l2 * l3 / 9.0 - 5.0 / 21.0 * l1 * (l2 ** 2 + l3 ** 2)

    def terms(u):
        return np.abs(u) ** 3 + np.abs(c1 * u * u) + np.abs(c2 * u) + np.abs(c3)

    dP = 3 * val ** 2 + 2 * c1 * val + c2
    kappa = terms(val) / np.maximum(np.abs(val * dP), 1e-300)
    # a root at 0 (l1 = 0 with l2 l3 = 0: P(u) = u^3) has no relative accuracy: not simple
    u_scale = np.abs(c1) + np.sqrt(np.abs(c2)) + np.cbrt(np.abs(c3)) + np.abs(l1) + np.abs(l2) + np.abs(l3)
    simple = (kappa < 1e4) & (np.abs(val) > 1e-12 * u_scale)
    err = np.abs(got - val) / np.maximum(np.abs(val), 1e-300)
    assert simple.mean() > 0.99
    assert err[simple].max() <= 1e-10, err[simple].max()
    P = ((got + c1) * got + c2) * got + c3
    assert np.all(np.abs(P[~simple]) <= 1e-13 * terms(got)[~simple])


def test_tabulated_hull_with_axes_above_zero(tables):
    """x and y axes starting at 0.3: points with x or y below 0.3 lie outside
    the table and take the R-LPT root, as in the oracle; points just above it
    are interpolated. Eigenvalue spectra are placed on both sides of the faces
    x = 0.3 and y = 0.3, plus isotropic Gaussian Hessians."""
    import paper_2510_02873_gb300 as cc
    dg, xg0, _ = table_axes()
    xg = 0.3 + xg0 * (39.7 / 40.0)
    yg = xg.copy()
    val = oracle.tab_node_values(dg, xg, yg)
    tab = oracle.Tab(dg, xg, yg, val)
    rng = np.random.default_rng(31)
    spectra = []
    for l1 in (0.6, 1.5, 4.0):
        for xv in (0.0, 0.1, 0.25, 0.299, 0.301, 0.35, 0.8):
            for yv in (0.0, 0.2, 0.299, 0.301, 0.5, 2.0):
                spectra.append([l1, l1 - xv, l1 - xv - yv])
    Ms = np.array([(lambda Q: Q @ np.diag(l) @ Q.T)(np.linalg.qr(rng.normal(size=(3, 3)))[0]) for l in spectra])
    planes = np.stack([Ms[:, 0, 0], Ms[:, 1, 1], Ms[:, 2, 2], Ms[:, 0, 1], Ms[:, 0, 2], Ms[:, 1, 2]])
    n_sp = planes.shape[1]
    gauss = hessgen.hessian_planes(3131, 0, 0, 2.0, 60000)
    stack = np.concatenate([planes, gauss], axis=1)[None]
    F_all, fl = oracle_tab_per_radius(tables, tab, stack)
    with cc.Context(0.3, 0.7, 512, 1e-3, 1.0, device=0) as c:
        c.set_table(dg, xg, yg, val)
        F, idx, st = run_tab(c, stack, [2.0], plane_stride=stack.shape[2] + (stack.shape[2] % 2))
    s = compare_max(F, idx, F_all, fl)
    out = (fl[0] & oracle.FLAG_HULL_OUT) != 0
    # both sides of the lower faces are exercised, among the designed spectra and the Gaussian ones
    assert out[:n_sp].sum() > 40 and (~out[:n_sp]).sum() >= 27  # 3 x 3 inside per l1
    assert out[n_sp:].sum() > 1000 and (~out[n_sp:]).sum() > 1000
    # the kernel counts every point it sends to the R-LPT root (l1 <= 0 included)
    assert st["fp64_branch"] >= int(out.sum())
    print("tabulated hull x, y >= 0.3", s, "outside", int(out.sum()))


def test_tabulated_delta_hull_at_signed_zero(tables):
    """A delta axis that starts at 0: a point whose trace is exactly -0.0 (all
    three diagonal entries -0.0) is treated as one with trace +0.0 and the
    same off-diagonal entries (inside the table, as the FP64 comparison with
    the axis end has it; the oracle, whose trace comes from its eigenvalues,
    flags both as on the hull's edge), and points with a trace of -1e-3 lie
    outside (R-LPT root)."""
    import paper_2510_02873_gb300 as cc
    _, xg, yg = table_axes()
    dg = np.linspace(0.0, 40.0, 64)
    val = oracle.tab_node_values(dg, xg, yg)
    tab = oracle.Tab(dg, xg, yg, val)
    rng = np.random.default_rng(47)
    m = 1000
    off = rng.normal(size=(3, m)) * 0.8
    neg0 = np.concatenate([np.full((3, m), -0.0), off])
    pos0 = np.concatenate([np.zeros((3, m)), off])
    shifted = pos0.copy()
    shifted[0] = -1e-3
    planes = np.concatenate([neg0, pos0, shifted], axis=1)
    assert np.all(np.signbit((planes[0] + planes[1] + planes[2])[:m]))  # the trace is -0.0 there
    stack = planes[None]
    F_all, fl = oracle_tab_per_radius(tables, tab, stack)
    assert np.all((fl[0, 2 * m:] & oracle.FLAG_HULL_OUT) != 0)
    with cc.Context(0.3, 0.7, 512, 1e-3, 1.0, device=0) as c:
        c.set_table(dg, xg, yg, val)
        F, idx, st = run_tab(c, stack, [1.0])
    assert np.array_equal(F[:m], F[m:2 * m]) and np.array_equal(idx[:m], idx[m:2 * m])
    assert (F[:m] > 0).sum() > m // 2
    compare_max(F, idx, F_all, fl)


def test_table_query_toy(ctx, table):
    """The spline x bilinear routine on its own (the paper's 64 x 64 grid with a
    128-knot spline per node), against the oracle's query."""
    tab, (dg, xg, yg, val) = table
    rng = np.random.default_rng(3)
    m = 20000
    q = [rng.uniform(dg[0], dg[-1], m), rng.uniform(0, xg[-1], m), rng.uniform(0, yg[-1], m)]
    qd = [torch.from_numpy(a).cuda() for a in q]
    out = torch.empty(m, dtype=torch.float64, device="cuda")
    ctx.table_query(*qd, out)
    torch.cuda.synchronize()
    ref = tab.query(*q)
    assert np.all(rel_err(out.cpu().numpy(), ref) <= 1e-12 * np.maximum(1.0, 1.0 / np.maximum(np.abs(ref), 1e-300)))


def test_spline_toy_x_squared(ctx):
    """The paper's spline toy: y = x^2 on 512 random knots, random queries;
    GPU vs the oracle's natural spline to rounding, and the residual vs x^2."""
    rng = np.random.default_rng(4)
    xk = np.sort(rng.uniform(0.0, 1.0, 512))
    yk = xk ** 2
    m = 100000
    q = rng.uniform(xk[0], xk[-1], m)
    qd = torch.from_numpy(q).cuda()
    out = torch.empty(m, dtype=torch.float64, device="cuda")
    ctx.spline_eval(xk, yk, qd, out)
    torch.cuda.synchronize()
    got = out.cpu().numpy()
    M = oracle.spline_build(xk, yk)
    sample = rng.choice(m, 3000, replace=False)
    ref = oracle.spline_eval(xk, yk, M, q[sample])
    assert np.all(np.abs(got[sample] - ref) <= 1e-14 * np.maximum(1.0, np.abs(ref)) + 1e-15)
    resid = np.abs(got - q ** 2) / q ** 2
    assert np.median(resid) < 1e-6


def test_tabulated_needs_a_table():
    import paper_2510_02873_gb300 as cc
    with cc.Context() as c:
        n = 64
        d = torch.zeros((1, 6, n), dtype=torch.float64, device="cuda")
        F = torch.zeros(n, dtype=torch.float64, device="cuda")
        idx = torch.full((n,), -1, dtype=torch.int32, device="cuda")
        with pytest.raises(cc.CollapseError):
            c.collapse_multi(d, [1.0], F, idx, mode="tabulated")
        with pytest.raises(cc.CollapseError):  # bad axes
            c.set_table([0, 1, 1, 2], [0, 1], [0, 1], np.zeros((2, 2, 4)))


def test_bilinear_toy_paper_definition():
    """The paper's 2D interpolation toy (Sec. 4.3): z = x^2 + y^2 tabulated on
    a random 64 x 64 grid whose nodes each carry a 128-knot spline (random
    knots along delta), 1e6 random queries through cc_table_query: GPU vs the
    oracle's query to rounding, and the residual against the analytic function
    within the bilinear bound (hx^2 + hy^2) / 4 (the function is constant
    along delta, so the splines reproduce the node values)."""
    import paper_2510_02873_gb300 as cc
    rng = np.random.default_rng(41)
    dg = np.sort(rng.uniform(-1.0, 1.0, 128))
    xg = np.sort(rng.uniform(0.0, 1.0, 64))
    yg = np.sort(rng.uniform(0.0, 1.0, 64))
    val = np.repeat((xg[:, None] ** 2 + yg[None, :] ** 2)[:, :, None], 128, axis=2)
    m = 1000000
    q = [rng.uniform(dg[0], dg[-1], m), rng.uniform(xg[0], xg[-1], m), rng.uniform(yg[0], yg[-1], m)]
    with cc.Context(device=0) as c:
        c.set_table(dg, xg, yg, val)
        qd = [torch.from_numpy(a).cuda() for a in q]
        out = torch.empty(m, dtype=torch.float64, device="cuda")
        c.table_query(*qd, out)
        torch.cuda.synchronize()
        got = out.cpu().numpy()
    ref = oracle.Tab(dg, xg, yg, val).query_many(*q)
    assert np.all(np.abs(got - ref) <= 1e-13 * np.maximum(1.0, np.abs(ref)))
    ix = np.searchsorted(xg, q[1], side="right") - 1
    iy = np.searchsorted(yg, q[2], side="right") - 1
    hx, hy = xg[ix + 1] - xg[ix], yg[iy + 1] - yg[iy]
    err = got - (q[1] ** 2 + q[2] ** 2)
    assert np.all(err >= -1e-13) and np.all(err <= (hx ** 2 + hy ** 2) / 4 + 1e-13)
    print("2D toy: mean relative residual vs x^2 + y^2", float(np.mean(np.abs(err) / (q[1] ** 2 + q[2] ** 2))))
