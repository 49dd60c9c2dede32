"""The checking build of the library (compiled with CC_DEBUG): every table
index of the collapse kernels is tested against its range; an index outside
sets bit 2 of cc_stats.error_flags and is clamped, so the kernel never reads
outside a table. Small cases of every mode run through that build in a child
process (the binding loads it with CC_LIBCOLLAPSE_DEBUG=1) and must raise no
flag and give exactly the release build's F_max/idx."""
import json
import os
import subprocess
import sys

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = r"""
import json, sys
import numpy as np
import torch
sys.path.insert(0, ROOT)
import hessgen
import hessgen.device as hdev
import paper_2510_02873_gb300 as cc

out = {}
with cc.Context(0.3, 0.7, 512, 1e-3, 1.0, device=0) as ctx:
    n = 9000
    for mode, dt in (("fp64", np.float64), ("f32x2", np.float64), ("exact_growth", np.float64),
                     ("mixed", np.float32), ("tabulated", np.float64)):
        sig = hessgen.sigma_schedule(5, 0.3, 8.0)
        stack = hessgen.hessian_stack(61, 0, sig, n, dtype=dt)
        if mode == "tabulated":
            t = np.linspace(-1.0, 1.0, 64)
            dg = 30.0 * np.sinh(2.5 * t) / np.sinh(2.5)
            xg = np.linspace(0.0, 20.0, 32) ** 1.0
            ctx.set_table(dg, xg, xg.copy(), ctx.table_nodes_rlpt(dg, xg, xg.copy()))
        h = torch.from_numpy(stack).cuda()
        F = torch.empty(n, dtype=torch.float64, device="cuda")
        idx = torch.empty(n, dtype=torch.int32, device="cuda")
        ctx.reset_max(F, idx)
        ctx.reset_stats()
        ctx.collapse_multi(h, sig, F, idx, mode=mode)
        st = ctx.stats()
        out[mode] = {"F": F.cpu().numpy().tolist(), "idx": idx.cpu().numpy().tolist(), "flags": st["error_flags"]}
    # surrogate (both engines), the network trained once by the parent
    net = np.load(NET)
    ctx.load_surrogate(net["params"], net["hull"])
    sig = hessgen.sigma_schedule(3, 0.5, 4.0)
    h = torch.from_numpy(hessgen.hessian_stack(62, 0, sig, n, dtype=np.float32)).cuda()
    for eng in ("tcgen05", "mma_sync"):
        ctx.set_surrogate_engine(eng)
        F = torch.empty(n, dtype=torch.float64, device="cuda")
        idx = torch.empty(n, dtype=torch.int32, device="cuda")
        ctx.reset_max(F, idx)
        ctx.reset_stats()
        ctx.collapse_multi(h, sig, F, idx, mode="surrogate")
        st = ctx.stats()
        out["surrogate_" + eng] = {"F": F.cpu().numpy().tolist(), "idx": idx.cpu().numpy().tolist(),
                                   "flags": st["error_flags"]}
    # batched persistent kernel
    items = []
    for k, g in enumerate((20, 32)):
        sg = hessgen.sigma_schedule(4 + k, 0.3, 4.0)
        hh = torch.from_numpy(hessgen.hessian_stack(70 + k, 0, sg, g ** 3, dtype=np.float32)).cuda()
        items.append((hh, sg, torch.zeros(g ** 3, dtype=torch.float64, device="cuda"),
                      torch.full((g ** 3,), -1, dtype=torch.int32, device="cuda")))
    ctx.reset_stats()
    b = cc.Batch(ctx, items, mode="mixed")
    b.run()
    torch.cuda.synchronize()
    st = ctx.stats()
    out["batched"] = {"F": torch.cat([it[2] for it in items]).cpu().numpy().tolist(),
                      "idx": torch.cat([it[3] for it in items]).cpu().numpy().tolist(), "flags": st["error_flags"]}
    b.close()
print("RESULT " + json.dumps(out))
"""


def _run(debug: bool, net: str) -> dict:
    env = dict(os.environ)
    env["CC_LIBCOLLAPSE_DEBUG"] = "1" if debug else "0"
    code = CHILD.replace("ROOT", repr(ROOT)).replace("NET", repr(net))
    res = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True, timeout=900)
    assert res.returncode == 0, res.stderr[-3000:]
    line = [l for l in res.stdout.splitlines() if l.startswith("RESULT ")][-1]
    return json.loads(line[len("RESULT "):])


def test_debug_build_raises_no_flag_and_matches_release(tmp_path):
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    from paper_2510_02873_gb300 import buildlib
    import __graft_entry__
    __graft_entry__.build()
    buildlib.build(debug=True)
    # one network for both children (training order depends on atomics, so
    # two trainings differ at rounding level)
    import hessgen.device as hdev
    import paper_2510_02873_gb300 as cc
    with cc.Context(0.3, 0.7, 512, 1e-3, 1.0, device=0) as ctx:
        tr = torch.empty((6, 1 << 20), dtype=torch.float32, device="cuda")
        hdev.fill(tr, 5, 1, 0, 1.0)
        ctx.surrogate_train(tr, 1.0, steps=60, batch=8192, lr=3e-3, seed=2)
        params, hull = ctx.surrogate_params()
    net = str(tmp_path / "net.npz")
    np.savez(net, params=params, hull=hull)
    rel = _run(False, net)
    dbg = _run(True, net)
    assert set(rel) == set(dbg)
    for mode in rel:
        assert dbg[mode]["flags"] == 0, (mode, dbg[mode]["flags"])
        assert rel[mode]["flags"] == 0, mode
        assert np.array_equal(np.asarray(dbg[mode]["F"]), np.asarray(rel[mode]["F"])), mode
        assert np.array_equal(np.asarray(dbg[mode]["idx"]), np.asarray(rel[mode]["idx"])), mode
