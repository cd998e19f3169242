"""The C-ABI library loads and exports every entry point include/tvcs.h declares;
argument validation happens on the host before any device work."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "tvcs.h")


@pytest.fixture(scope="module")
def tv():
    import importlib.util
    spec = importlib.util.spec_from_file_location(
        "tvcs_build", os.path.join(ROOT, "paper_1001_1774_gb300", "build.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    mod.build()
    import paper_1001_1774_gb300 as tv
    return tv


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(tvcs_[a-z_]+)\s*\(", text)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ["tvcs_create", "tvcs_solve", "tvcs_solve_batched", "tvcs_destroy",
                     "tvcs_last_error"]:
        assert required in names


def test_library_exports_every_declared_symbol(tv):
    lib = ctypes.CDLL(tv.LIB_PATH)
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing
    assert sorted(tv.EXPORTED) == declared_functions()


def test_default_options(tv):
    o = tv.tvcs_default_options()
    assert o.algo == tv.TVCS_ALGO_IADM and o.max_iter == 500 and o.tau == 0.0
    assert o.precision == tv.TVCS_PREC_FP32 and o.power_iters == 100


@pytest.mark.parametrize("kwargs,frag", [
    (dict(m=0), "m = 0"),
    (dict(n=20), "n = 20"),
    (dict(n=8), "n = 8"),
    (dict(mu=0.0), "mu"),
    (dict(beta=-1.0), "beta"),
    (dict(tol=-1e-3), "tol"),
])
def test_create_rejects_invalid_arguments_on_host(tv, kwargs, frag):
    args = dict(m=10, n=32, mu=1.0, beta=1.0, tol=0.0)
    args.update(kwargs)
    with pytest.raises(tv.TvcsError) as ei:
        tv.tvcs_create(None, 0, args["m"], args["n"], args["mu"], args["beta"], args["tol"])
    assert ei.value.status == tv.TVCS_ERR_INVALID_ARG
    assert frag in str(ei.value)


def test_unknown_options_rejected(tv):
    o = tv.tvcs_default_options()
    o.algo = 7
    with pytest.raises(tv.TvcsError) as ei:
        tv.tvcs_create(None, 0, 10, 32, 1.0, 1.0, 0.0, o)
    assert ei.value.status == tv.TVCS_ERR_INVALID_ARG


def test_null_handle_and_batch_arguments(tv):
    lib = tv._lib
    assert lib.tvcs_solve(None, None, None, None) == tv.TVCS_ERR_INVALID_ARG
    assert "null handle" in tv.tvcs_last_error()
    assert lib.tvcs_solve_batched(None, -1, None, None, None, None) == tv.TVCS_ERR_INVALID_ARG
    assert lib.tvcs_solve_batched(None, 0, None, None, None, None) == tv.TVCS_OK
    # per-problem mu overrides are checked before any handle is touched
    buf = (ctypes.c_float * 4)()
    hs = (ctypes.c_void_p * 1)(ctypes.addressof(buf))
    fs = (ctypes.c_void_p * 1)(ctypes.addressof(buf))
    for bad in (0.0, -1.0, float("nan"), float("inf")):
        mus = (ctypes.c_double * 1)(bad)
        assert lib.tvcs_solve_batched(hs, 1, fs, fs, mus, None) == tv.TVCS_ERR_INVALID_ARG
        assert "mu[0]" in tv.tvcs_last_error()
    assert lib.tvcs_destroy(None) == tv.TVCS_OK
