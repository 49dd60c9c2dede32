"""The C-ABI library loads and exports every declared symbol; host-only calls (no GPU)."""
import ctypes
import os
import re

import numpy as np
import pytest

import oracle
import paper_2510_02873_gb300 as cc
from paper_2510_02873_gb300 import _lib, buildlib as pkg_build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared(header: str) -> list[str]:
    text = open(os.path.join(ROOT, "include", header)).read()
    return re.findall(r"^CC_API\s+[\w\s\*]+?\b(cc_\w+)\s*\(", text, flags=re.M)


@pytest.fixture(scope="module")
def lib():
    pkg_build.build()
    return _lib.load()


def test_every_declared_symbol_is_exported(lib):
    names = _declared("collapse.h")
    assert len(names) >= 12
    for name in names:
        assert hasattr(lib, name), f"{name} declared in include/collapse.h but not exported"
    assert set(names) == set(_lib.EXPORTS)


def test_only_api_symbols_are_exported():
    import subprocess
    out = subprocess.run(["nm", "-D", "--defined-only", pkg_build.LIB_PATH], capture_output=True,
                         text=True, check=True).stdout
    text_syms = {line.split()[-1] for line in out.splitlines() if " T " in line}
    assert text_syms == set(_declared("collapse.h"))


def test_strerror_and_version(lib):
    assert lib.cc_strerror(0) == b"CC_OK"
    assert lib.cc_strerror(1).startswith(b"CC_EINVAL")
    assert lib.cc_strerror(999) == b"unknown status code"
    assert lib.cc_version() >= 100


def test_host_growth_table_matches_oracle():
    """The library's growth ODE (RK4 in ln a) and the oracle's (RK4 in a) are
    independent discretisations; both must converge to the same D(a_k)."""
    a_o, D_o = oracle.growth_table(0.3, 0.7, 512, 1e-3, 1.0)
    a_l, D_l = cc.cc_build_growth_table(0.3, 0.7, 512, 1e-3, 1.0)
    np.testing.assert_allclose(a_l, a_o, rtol=1e-15, atol=0)
    np.testing.assert_allclose(D_l, D_o, rtol=1e-12, atol=0)
    a_e, D_e = cc.cc_build_growth_table(1.0, 0.0, 64, 1e-3, 1.0)
    np.testing.assert_allclose(D_e, a_e, rtol=1e-12, atol=0)


@pytest.mark.parametrize("bad", [
    dict(n_knots=1), dict(n_knots=5000), dict(a_min=1e-6), dict(a_min=0.5, a_max=0.4),
    dict(omega_m=0.0), dict(omega_m=float("nan")),
])
def test_host_growth_table_rejects_bad_cosmology(bad):
    args = dict(omega_m=0.3, omega_l=0.7, n_knots=64, a_min=1e-3, a_max=1.0)
    args.update(bad)
    n = max(args["n_knots"], 1)
    a = np.empty(n)
    D = np.empty(n)
    cosmo = _lib.CcCosmology(args["omega_m"], args["omega_l"], args["n_knots"], args["a_min"], args["a_max"])
    rc = _lib.load().cc_build_growth_table(ctypes.byref(cosmo), a.ctypes.data, D.ctypes.data)
    assert rc == _lib.CC_EINVAL
    assert _lib.load().cc_last_error_message()


def test_null_arguments_rejected_without_device(lib):
    assert lib.cc_create(None, None, 0) == _lib.CC_EINVAL
    assert lib.cc_collapse_scale(None, 0, None, 8, 0, 0, 1.0, None, None, 0, None) == _lib.CC_EINVAL
    assert lib.cc_reset_max(None, None, None, 0, None) == _lib.CC_EINVAL
    lib.cc_destroy(None)  # no-op


def test_mode_names_match_the_header():
    text = open(os.path.join(ROOT, "include", "collapse.h")).read()
    enum = {m.group(1).lower(): int(m.group(2)) for m in re.finditer(r"CC_MODE_(\w+)\s*=\s*(\d+)", text)}
    assert enum == {"fp64": 0, "mixed": 1, "surrogate": 2, "tabulated": 3, "f32x2": 4, "exact_growth": 5}
    assert enum == _lib.MODES


def test_surrogate_engine_names_match_the_header(lib):
    import paper_2510_02873_gb300 as cc
    text = open(os.path.join(ROOT, "include", "collapse.h")).read()
    enum = {m.group(1).lower(): int(m.group(2)) for m in re.finditer(r"CC_SURROGATE_(\w+)\s*=\s*(\d+)", text)}
    assert enum == cc.Context.SURROGATE_ENGINES == {"mma_sync": 0, "tcgen05": 1}
    assert lib.cc_set_surrogate_engine(None, 0) == _lib.CC_EINVAL
