"""CPU checks of the C ABI boundary: the library builds, loads, exports every symbol include/enufft.h
declares, fills the documented defaults, and rejects bad arguments synchronously (no GPU needed)."""
import ctypes
import os
import re
import subprocess

import pytest

import paper_2606_21278_b300 as enufft
from paper_2606_21278_b300 import build as enufft_build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "enufft.h")


@pytest.fixture(scope="module")
def lib():
    enufft_build.build()
    return enufft.load_library()


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(enufft_[a-z0-9_]+)\s*\(", src)))


def test_header_declares_the_boundary_calls():
    names = declared_functions()
    for required in ("enufft_plan_create", "enufft_type1", "enufft_ems", "enufft_type1_backward",
                     "enufft_plan_destroy", "enufft_type1_ems", "enufft_ems_backward"):
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    names = declared_functions()
    out = subprocess.run(["nm", "-D", "--defined-only", enufft.LIB_PATH], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\bT (enufft_[a-z0-9_]+)", out))
    missing = [n for n in names if n not in exported]
    assert not missing, missing
    for n in names:
        assert hasattr(lib, n)


def test_build_targets_sm_103a_only():
    assert enufft_build.ARCH == ["-gencode", "arch=compute_103a,code=sm_103a"]


def test_defaults(lib):
    o = enufft._Opts()
    lib.enufft_default_opts(ctypes.byref(o))
    assert (o.modes, o.oversamp, o.kernel_width, o.prec, o.mask, o.eta, o.tc_max_points, o.kernel, o.frame,
            o.autotune, o.tune_cache, o.deterministic) == (64, 2.0, 7, 2, 0, 1.5, 0, 0, 0, 0, None, 1)
    e = enufft._Ems()
    lib.enufft_default_ems(ctypes.byref(e))
    assert (e.k_min, e.k_max, e.alpha_min, e.alpha_max, e.delta, e.w1, e.w2, e.sum_over, e.include_dc) == \
        (1, 12, 0.0, 0.7, 0.02, 0.5, 0.5, 0, 0)


@pytest.mark.parametrize("field,value", [("modes", 7), ("modes", 0), ("modes", 256), ("oversamp", 1.5),
                                         ("kernel_width", 1), ("kernel_width", 17), ("prec", 9), ("mask", 5),
                                         ("eta", 0.0), ("tol", -1.0), ("tc_max_points", -1), ("kernel", 2),
                                         ("kernel", -1), ("frame", 2), ("frame", -1), ("autotune", 2),
                                         ("deterministic", 2), ("deterministic", -1)])
def test_plan_create_rejects_bad_options(lib, field, value):
    o = enufft._Opts()
    lib.enufft_default_opts(ctypes.byref(o))
    setattr(o, field, value)
    h = ctypes.c_void_p(123)
    st = lib.enufft_plan_create(ctypes.byref(h), ctypes.byref(o), 0, None, None, None, None)
    assert st == 1 and h.value is None
    assert lib.enufft_last_error(None).decode().startswith("plan_create")


def test_null_arguments_are_errors(lib):
    h = ctypes.c_void_p()
    assert lib.enufft_plan_create(ctypes.byref(h), None, 0, None, None, None, None) == 1
    assert lib.enufft_plan_create(None, None, 0, None, None, None, None) == 1
    o = enufft._Opts()
    lib.enufft_default_opts(ctypes.byref(o))
    assert lib.enufft_plan_create(ctypes.byref(h), ctypes.byref(o), 4, None, None, None, None) == 1
    assert lib.enufft_plan_create(ctypes.byref(h), ctypes.byref(o), -1, None, None, None, None) == 1
    for call, n in (("enufft_type1", 6), ("enufft_type1_backward", 8), ("enufft_sync_status", 1),
                    ("enufft_set_stream", 2), ("enufft_get_plan_info", 2)):
        assert getattr(lib, call)(*([None] * n)) == 1
    e = enufft._Ems()
    lib.enufft_default_ems(ctypes.byref(e))
    assert lib.enufft_ems(None, None, None, 0, ctypes.byref(e), None, None, None) == 1
    assert lib.enufft_selftest_wait_timeout(None, 8) == 1
    assert lib.enufft_reconstruct(None, None, None, None, 12, None, None, None, None, None, None) == 1
    assert lib.enufft_voronoi_weights(None, None, None, 64, None) == 1
    assert lib.enufft_plan_destroy(None) == 0


def test_binding_option_maps_match_the_header():
    """The binding's option names map to the enum values that include/enufft.h declares."""
    hdr = open(os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include", "enufft.h")).read()
    values = {name: int(v) for name, v in re.findall(r"\b(ENUFFT_[A-Z0-9_]+)\s*=\s*(\d+)", hdr)}
    expect = [
        (enufft._PREC, {"fp64": "ENUFFT_FP64", "fp32": "ENUFFT_FP32", "mixed": "ENUFFT_MIXED"}),
        (enufft._MASK, {"cell": "ENUFFT_MASK_CELL", "square": "ENUFFT_MASK_SQUARE", "circle": "ENUFFT_MASK_CIRCLE"}),
        (enufft._KERNEL, {"es": "ENUFFT_KERNEL_ES", "kb": "ENUFFT_KERNEL_KB"}),
        (enufft._FRAME, {"centroid": "ENUFFT_FRAME_CENTROID", "edge": "ENUFFT_FRAME_EDGE"}),
    ]
    for table, names in expect:
        assert set(table) == set(names)
        for key, cname in names.items():
            assert table[key] == values[cname], (key, cname)


def test_tune_cache_round_trip(tmp_path, lib):
    """The tuning cache file (enufft_tune_cache_store / _lookup, host only): records round-trip with
    their timings, keys coexist and are replaced, a missing key, a missing file and a malformed file
    are misses, a malformed file is replaced by the next store, and the file is plain JSON."""
    import json
    path = str(tmp_path / "tune.json")
    a = {"tc_max_points": 512, "fused_blocks_per_sm": 2, "ladder": [128, 256, 512, 1024],
         "ns_fused": [0.31, 0.16, 0.09, 0.05], "ns_tc": [0.2, 0.15, 0.08, 0.07], "large_tile": 64}
    b = {"tc_max_points": 0, "fused_blocks_per_sm": 1, "ladder": [], "ns_fused": [], "ns_tc": []}
    assert enufft.tune_cache_lookup(path, "k1") is None                       # no file yet
    enufft.tune_cache_store(path, "gpu=X|P=64", a)
    enufft.tune_cache_store(path, "gpu=X|P=32", b)
    got = enufft.tune_cache_lookup(path, "gpu=X|P=64")
    assert got["tc_max_points"] == 512 and got["fused_blocks_per_sm"] == 2 and got["ladder"] == a["ladder"]
    assert got["ns_fused"] == pytest.approx(a["ns_fused"], rel=1e-5) and got["ns_tc"] == pytest.approx(a["ns_tc"], rel=1e-5)
    assert got["from_cache"] is True and got["large_tile"] == 64
    assert enufft.tune_cache_lookup(path, "gpu=X|P=32")["tc_max_points"] == 0
    assert enufft.tune_cache_lookup(path, "gpu=Y|P=64") is None
    enufft.tune_cache_store(path, "gpu=X|P=64", {**a, "tc_max_points": 1024})  # replaced, not duplicated
    d = json.load(open(path))
    assert sorted(d) == ["gpu=X|P=32", "gpu=X|P=64"] and d["gpu=X|P=64"]["tc_max_points"] == 1024
    open(path, "w").write("{not json")
    assert enufft.tune_cache_lookup(path, "gpu=X|P=64") is None
    enufft.tune_cache_store(path, "k", b)
    assert json.load(open(path)) == {"k": {"tc_max_points": 0, "fused_blocks_per_sm": 1, "large_tile": 0,
                                           "ladder": [], "ns_fused": [], "ns_tc": []}}
    # records written before the tile field existed read as large_tile 0
    open(path, "w").write('{"old": {"tc_max_points": 0, "fused_blocks_per_sm": 1, "ladder": [], "ns_fused": [], '
                          '"ns_tc": []}}')
    assert enufft.tune_cache_lookup(path, "old")["large_tile"] == 0
    with pytest.raises(enufft.EnufftError):
        enufft.tune_cache_store(path, 'bad"key', b)
