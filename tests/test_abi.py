"""The C ABI without a GPU: the library loads, exports what include/culgt.h
declares, and rejects bad arguments on the host before any device work."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__
    __graft_entry__.build_library()
    from paper_1412_3655_gb300 import culgt
    return culgt


def declared_functions():
    names = []
    for h in os.listdir(os.path.join(ROOT, "include")):
        if h.endswith(".h"):
            text = open(os.path.join(ROOT, "include", h)).read()
            text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
            names += re.findall(r"\b(culgt_\w+)\s*\(", text)
    return sorted(set(names))


def test_every_declared_symbol_is_exported(lib):
    names = declared_functions()
    assert len(names) >= 15
    so = ctypes.CDLL(lib.LIBRARY_PATH)
    missing = [n for n in names if not hasattr(so, n)]
    assert not missing


def test_status_strings(lib):
    for s in range(-7, 2):
        assert lib.culgt_status_string(s).startswith("CULGT_")
    assert "unknown" in lib.culgt_status_string(42)


def test_defaults_validate(lib):
    p = lib.culgt_default_params(3, (8, 4, 4, 6))
    assert p.omega == 1.7 and p.theta_target == 1e-12 and p.switch_theta == 1e-8
    assert lib.culgt_validate(p) == lib.OK


@pytest.mark.parametrize("change,code", [
    ({"dims": (4, 3, 4, 4)}, -2),
    ({"dims": (0, 4, 4, 4)}, -2),
    ({"dims": (1024, 1024, 1024, 2)}, -2),
    ({"nc": 4}, -3),
    ({"storage_reals": 12, "nc": 2}, -3),
    ({"storage_reals": 10}, -3),
    ({"omega": 2.0}, -1),
    ({"omega": 0.9}, -1),
    ({"omega": float("nan")}, -1),
    ({"check_every": 0}, -1),
    ({"max_sweeps": -1}, -1),
    ({"precision": 5}, -1),
    ({"precision": 2, "switch_theta": float("nan")}, -1),
    ({"precision": 2, "switch_theta": -1e-8}, -1),
    ({"precision": 3, "switch_theta": -1.0}, -1),
    ({"theta_target": float("inf")}, -1),
    ({"dtype_in": 2}, -1),
    ({"or_variant": 2}, -1),
    ({"threads_per_site": 3}, -1),
    ({"block_size": 96}, -1),
    ({"min_blocks_per_sm": 2}, -1),
])
def test_validate_rejects(lib, change, code):
    p = lib.Params.defaults(3, (4, 4, 4, 4))
    for k, v in change.items():
        setattr(p, k, v)
    assert lib.culgt_validate(p) == code
    # the one-call entry points check before touching the device
    so = lib.library()
    assert so.culgt_landau_fix(ctypes.c_void_p(16), ctypes.byref(p._c()), None, None) == code


@pytest.mark.parametrize("precision", [2, 3])
def test_automatic_switch_validates(lib, precision):
    """switch_theta = 0 selects the automatic switch of the mixed schedules."""
    p = lib.Params.defaults(3, (4, 4, 4, 4), precision=precision, switch_theta=0.0)
    assert lib.culgt_validate(p) == lib.OK


@pytest.mark.parametrize("precision", [0, 1, 2, 3, 4])
@pytest.mark.parametrize("nc", [2, 3])
def test_every_precision_validates(lib, precision, nc):
    p = lib.Params.defaults(nc, (4, 2, 4, 6), precision=precision)
    assert lib.culgt_validate(p) == lib.OK
    assert lib.culgt_workspace_bytes(p) > 0


def test_null_pointers_rejected(lib):
    p = lib.Params.defaults(3, (4, 4, 4, 4))
    so = lib.library()
    assert so.culgt_landau_fix(None, ctypes.byref(p._c()), None, None) == lib.ERR_ARG
    assert so.culgt_landau_fix(ctypes.c_void_p(16), None, None, None) == lib.ERR_ARG
    assert so.culgt_sweep(ctypes.c_void_p(16), ctypes.byref(p._c()), -1, None) == lib.ERR_ARG
    assert so.culgt_create(ctypes.byref(p._c()), None, None) == lib.ERR_ARG


def test_workspace_bytes(lib):
    p = lib.Params.defaults(3, (32, 32, 32, 32))
    # FP64, 18 reals: 4V links x 144 B plus reduction scratch
    b = lib.culgt_workspace_bytes(p)
    V = 32 ** 4
    assert 4 * V * 144 <= b < 4 * V * 144 * 1.01
    p.precision = lib.MIXED
    b2 = lib.culgt_workspace_bytes(p)
    # mixed: FP32 12-real and FP64 18-real links plus the FP32 gauge accumulator
    assert b2 == pytest.approx(4 * V * (144 + 48) + V * 48, rel=0.01)


def test_anneal_defaults_validate(lib):
    a = lib.culgt_default_anneal_params()
    assert (a.t_start, a.t_end, a.steps, a.micro_sweeps, a.seed) == (0.6, 0.01, 500, 3, 0)
    assert lib.culgt_validate_anneal(a) == lib.OK
    assert lib.culgt_validate_anneal(lib.AnnealParams(seed=2 ** 64 - 1, steps=0)) == lib.OK


@pytest.mark.parametrize("change", [
    {"t_start": 0.0}, {"t_end": -1.0}, {"t_start": float("inf")}, {"t_end": float("nan")},
    {"steps": -1}, {"micro_sweeps": -2},
])
def test_anneal_validate_rejects(lib, change):
    a = lib.AnnealParams(**change)
    assert lib.culgt_validate_anneal(a) == lib.ERR_ARG
    # the annealing entry points check before touching the device
    so = lib.library()
    p = lib.Params.defaults(3, (4, 4, 4, 4))
    assert so.culgt_landau_fix_anneal(ctypes.c_void_p(16), ctypes.byref(p._c()), ctypes.byref(a._c()), None,
                                      None) == lib.ERR_ARG
    probs = (lib._Problem * 1)()
    probs[0].d_links = 16
    probs[0].dims = (ctypes.c_int * 4)(4, 4, 4, 4)
    assert so.culgt_fix_batched_anneal(probs, 1, ctypes.byref(p._c()), ctypes.byref(a._c()), None,
                                       None) == lib.ERR_ARG


def test_anneal_null_arguments_rejected(lib):
    so = lib.library()
    p = lib.Params.defaults(3, (4, 4, 4, 4))
    a = lib.AnnealParams()
    assert so.culgt_landau_fix_anneal(ctypes.c_void_p(16), ctypes.byref(p._c()), None, None, None) == lib.ERR_ARG
    assert so.culgt_landau_fix_anneal(None, ctypes.byref(p._c()), ctypes.byref(a._c()), None, None) == lib.ERR_ARG
    assert so.culgt_handle_anneal(None, ctypes.byref(a._c())) == lib.ERR_ARG
    assert so.culgt_handle_heatbath(None, 1.0, 0, 0) == lib.ERR_ARG
    assert so.culgt_default_anneal_params(None) == lib.ERR_ARG


def test_gauge_field_validates(lib):
    p = lib.Params.defaults(3, (4, 4, 4, 4), gauge=lib.MAG)
    assert lib.culgt_validate(p) == lib.OK
    p.gauge = 2
    assert lib.culgt_validate(p) == lib.ERR_ARG
    # Landau-only entry points refuse a MAG parameter block before any device work
    so = lib.library()
    q = lib.Params.defaults(3, (4, 4, 4, 4), gauge=lib.MAG)
    assert so.culgt_landau_fix(ctypes.c_void_p(16), ctypes.byref(q._c()), None, None) == lib.ERR_ARG
    assert so.culgt_landau_fix_host(ctypes.c_void_p(16), ctypes.byref(q._c()), None, None) == lib.ERR_ARG
    assert so.culgt_coulomb_fix(ctypes.c_void_p(16), ctypes.byref(q._c()), None, None, None) == lib.ERR_ARG
    a = lib.AnnealParams()
    assert so.culgt_landau_fix_anneal(ctypes.c_void_p(16), ctypes.byref(q._c()), ctypes.byref(a._c()), None,
                                      None) == lib.ERR_ARG
    assert so.culgt_mag_fix(None, ctypes.byref(q._c()), None, None) == lib.ERR_ARG
    # the gauge-returning fixes: Landau refuses a MAG block, both refuse null buffers
    assert so.culgt_landau_fix_gauge(ctypes.c_void_p(16), ctypes.byref(q._c()), None, None,
                                     ctypes.c_void_p(16)) == lib.ERR_ARG
    assert so.culgt_mag_fix_gauge(None, ctypes.byref(q._c()), None, None, ctypes.c_void_p(16)) == lib.ERR_ARG
    assert so.culgt_mag_fix_gauge(ctypes.c_void_p(16), ctypes.byref(q._c()), None, None, None) == lib.ERR_ARG
    bad = lib.Params.defaults(3, (4, 4, 4, 4), gauge=lib.MAG)
    bad.omega = 2.5
    assert so.culgt_mag_fix_gauge(ctypes.c_void_p(16), ctypes.byref(bad._c()), None, None,
                                  ctypes.c_void_p(16)) != lib.OK


def test_coulomb_anneal_rejects_before_device_work(lib):
    so = lib.library()
    p = lib.Params.defaults(3, (4, 4, 4, 4))
    bad = lib.AnnealParams(steps=-1)
    assert so.culgt_coulomb_fix_anneal(ctypes.c_void_p(16), ctypes.byref(p._c()), ctypes.byref(bad._c()), None,
                                       None, None) == lib.ERR_ARG
    assert so.culgt_coulomb_fix_anneal(ctypes.c_void_p(16), ctypes.byref(p._c()), None, None, None,
                                       None) == lib.ERR_ARG


def test_batched_empty_and_bad_problems_rejected(lib):
    """An empty batch, a NULL problem table or links pointer, and a problem
    with odd dims are refused before any device work."""
    so = lib.library()
    p = lib.Params.defaults(3, (4, 4, 4, 4))
    probs = (lib._Problem * 2)()
    probs[0].d_links = 16
    probs[0].dims = (ctypes.c_int * 4)(4, 4, 4, 4)
    probs[1].d_links = 16
    probs[1].dims = (ctypes.c_int * 4)(4, 3, 4, 4)
    assert so.culgt_fix_batched(probs, 0, ctypes.byref(p._c()), None, None) == lib.ERR_ARG
    assert so.culgt_fix_batched(None, 1, ctypes.byref(p._c()), None, None) == lib.ERR_ARG
    assert so.culgt_fix_batched(probs, 2, ctypes.byref(p._c()), None, None) == lib.ERR_DIMS
    probs[1].dims = (ctypes.c_int * 4)(4, 4, 4, 4)
    probs[1].d_links = None
    assert so.culgt_fix_batched(probs, 2, ctypes.byref(p._c()), None, None) == lib.ERR_ARG


def test_header_enums_match_the_binding(lib):
    """The constants of culgt.py are the values include/culgt.h declares."""
    text = open(os.path.join(ROOT, "include", "culgt.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    vals = {k: int(v) for k, v in re.findall(r"\b(CULGT_[A-Z0-9_]+)\s*=\s*(-?\d+)", text)}
    for name in ("OK", "NOT_CONVERGED", "ERR_ARG", "ERR_DIMS", "ERR_NC", "ERR_CUDA", "ERR_OOM", "ERR_NONFINITE",
                 "ERR_TIMEOUT", "ERR_TOO_LARGE", "FP64", "FP32", "MIXED", "MIXED_DF", "DF", "LANDAU", "MAG"):
        assert vals["CULGT_" + name] == getattr(lib, name), name


def test_struct_layouts_match_the_header(lib):
    """Field order of the ctypes mirrors equals the C structs' (names in order)."""
    text = open(os.path.join(ROOT, "include", "culgt.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    for cname, py in (("culgt_params", lib._Params), ("culgt_result", lib._Result),
                      ("culgt_anneal_params", lib._AnnealParams), ("culgt_problem", lib._Problem)):
        body = re.search(r"typedef struct \{([^{}]*)\}\s*" + cname + r";", text).group(1)
        names = re.findall(r"(\w+)(?:\[\d+\])?\s*;", body)
        assert names == [f[0] for f in py._fields_], cname
