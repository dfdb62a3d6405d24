"""The C-ABI library builds, loads and exports every entry point declared in
include/dmn.h; argument errors are reported before any CUDA work (no GPU
needed)."""
import ctypes
import os
import re

import numpy as np
import pytest

from paper_2103_08253_gb300 import dmn, fe, workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols(header="dmn.h", prefix="dmn_"):
    src = open(os.path.join(ROOT, "include", header)).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(%s[a-z_0-9]+)\s*\(" % prefix, src)))


def test_library_exports_every_declared_symbol():
    lib = dmn.load_library()
    syms = declared_symbols()
    assert "dmn_update" in syms and "dmn_create" in syms
    for s in syms:
        assert hasattr(lib, s), s
    assert set(dmn.EXPORTS) == set(syms)
    fsyms = declared_symbols("fe.h", "fe_")
    assert "fe_pcg" in fsyms
    for s in fsyms:
        assert hasattr(lib, s), s
    assert set(fe.FE_EXPORTS) == set(fsyms)
    psyms = declared_symbols("dmn_peak.h")
    assert psyms == ["dmn_fma_throughput", "dmn_peak_gflops"] and set(dmn.PEAK_EXPORTS) == set(psyms)
    for s in psyms:
        assert hasattr(lib, s), s


def test_peak_measurement_rejects_bad_arguments_without_touching_the_gpu():
    lib = dmn.load_library()
    g, ms = ctypes.c_double(), ctypes.c_double()
    assert lib.dmn_peak_gflops(7, 1.0, ctypes.byref(g), ctypes.byref(ms), None) == -1
    assert "unknown kind" in lib.dmn_last_error(None).decode()
    assert lib.dmn_peak_gflops(0, 0.0, ctypes.byref(g), ctypes.byref(ms), None) == -1
    assert lib.dmn_peak_gflops(0, 1.0, None, ctypes.byref(ms), None) == -1
    for bad in ((0, 6, 8, 32), (0, 64, 3, 32), (0, 64, 8, 0), (0, 65, 8, 32), (2, 64, 8, 32)):
        assert lib.dmn_fma_throughput(*bad, 0.1, ctypes.byref(g), ctypes.byref(ms), None) == -1, bad


def test_fe_mesh_create_rejects_bad_meshes_without_touching_the_gpu():
    lib = fe.load_library()
    m = W.plate_with_hole_mesh(4, 2, 1)
    h = ctypes.c_void_p(5)
    bad = m.conn.copy()
    bad[3, 2] = len(m.xyz)
    rc = lib.fe_mesh_create(len(m.xyz), len(bad), m.xyz.ctypes.data_as(ctypes.c_void_p),
                            bad.ctypes.data_as(ctypes.c_void_p), ctypes.byref(h))
    assert rc == -1 and h.value is None and "out of range" in lib.fe_last_error(None).decode()
    inv = np.ascontiguousarray(m.conn[:, [1, 0, 3, 2, 5, 4, 7, 6]])       # mirrored: det(J) < 0
    rc = lib.fe_mesh_create(len(m.xyz), len(inv), m.xyz.ctypes.data_as(ctypes.c_void_p),
                            inv.ctypes.data_as(ctypes.c_void_p), ctypes.byref(h))
    assert rc == -1 and "det(J)" in lib.fe_last_error(None).decode()


def _desc(K=3, M=3, w=None, kind=1):
    tree = W.tree_d10_fit(K, seed=1)
    p = np.ascontiguousarray(tree.p.reshape(-1)); q = np.ascontiguousarray(tree.q.reshape(-1))
    w = np.ascontiguousarray(tree.w if w is None else w, dtype=np.float64)
    d = dmn.TreeDesc_()
    dp = ctypes.POINTER(ctypes.c_double)
    d.K, d.M = K, M
    d.p, d.q, d.w = p.ctypes.data_as(dp), q.ctypes.data_as(dp), w.ctypes.data_as(dp)
    d.phase[0] = dmn.Phase_(0, 72000.0, 0.22, 0.0, 0.0)
    d.phase[1] = dmn.Phase_(kind, 3000.0, 0.35, 40.0, 300.0)
    return d, (p, q, w)


@pytest.mark.parametrize("case,msg", [
    (dict(K=9), "K must be"), (dict(K=0), "K must be"), (dict(M=5), "M must be"),
    (dict(w=np.r_[np.ones(7), -1.0]), "weights"), (dict(w=np.r_[np.ones(7), np.nan]), "weights"),
    (dict(w=np.zeros(8)), "all be zero"),
    (dict(kind=7), "phase kind"), (dict(kind=2), "exponential-linear")])
def test_create_rejects_bad_arguments_without_touching_the_gpu(case, msg):
    lib = dmn.load_library()
    d, keep = _desc(**case)
    h = ctypes.c_void_p(123)
    rc = lib.dmn_create(ctypes.byref(d), 1, None, ctypes.byref(h))
    assert rc == -1
    assert h.value is None
    assert msg in lib.dmn_last_error(None).decode()


@pytest.mark.parametrize("opt,msg", [((1e-12, 50, 3, 0, 0, 0), "unknown precision"),
                                     ((1e-12, 50, -1, 0, 0, 0), "unknown precision"),
                                     ((1e-12, 50, dmn.PREC_MIXED_F32_TANGENT, 48, 0, 0), "multiple of 32"),
                                     ((1e-12, 50, dmn.PREC_F64, 128, 3, 1), "256 with the line search")])
def test_create_rejects_bad_options_without_touching_the_gpu(opt, msg):
    lib = dmn.load_library()
    d, keep = _desc()
    o = dmn.Options_(*opt)
    h = ctypes.c_void_p(123)
    assert lib.dmn_create(ctypes.byref(d), 1, ctypes.byref(o), ctypes.byref(h)) == -1
    assert h.value is None and msg in lib.dmn_last_error(None).decode()
    assert set(dmn.PRECISIONS.values()) == {dmn.PREC_F64, dmn.PREC_MIXED, dmn.PREC_MIXED_F32_TANGENT}


def test_predictor_option_is_checked_without_touching_the_gpu():
    lib = dmn.load_library()
    d, keep = _desc()
    h = ctypes.c_void_p(123)
    o = dmn.Options_(1e-12, 50, dmn.PREC_F64, 0, 0, 0, 2)
    assert lib.dmn_create(ctypes.byref(d), 1, ctypes.byref(o), ctypes.byref(h)) == -1
    assert h.value is None and "predictor must be 0 or 1" in lib.dmn_last_error(None).decode()
    # the allocation-free update has no extrapolated start
    o = dmn.Options_(1e-12, 50, dmn.PREC_F64, 0, 0, 0, 1)
    rc = lib.dmn_update_noalloc(ctypes.byref(d), ctypes.byref(o), 8, *([None] * 10), None)
    assert rc == -1 and "extrapolated start" in lib.dmn_last_error(None).decode()


def test_first_stage_option_is_checked_without_touching_the_gpu():
    lib = dmn.load_library()
    d, keep = _desc()
    for bad in (2, -2):
        h = ctypes.c_void_p(123)
        o = dmn.Options_(1e-12, 50, dmn.PREC_MIXED, 0, 0, 0, 0, bad)
        assert lib.dmn_create(ctypes.byref(d), 1, ctypes.byref(o), ctypes.byref(h)) == -1
        assert h.value is None and "first_stage must be -1, 0 or 1" in lib.dmn_last_error(None).decode()
    for bad in (1, 5, 9):
        h = ctypes.c_void_p(123)
        o = dmn.Options_(1e-12, 50, dmn.PREC_MIXED, 0, 0, 0, 0, 0, bad)
        assert lib.dmn_create(ctypes.byref(d), 1, ctypes.byref(o), ctypes.byref(h)) == -1
        assert h.value is None and "stage_ctas_per_sm must be" in lib.dmn_last_error(None).decode()
    for bad in (2, -2):
        h = ctypes.c_void_p(123)
        o = dmn.Options_(1e-12, 50, dmn.PREC_F64, 0, 0, 0, 0, 0, 0, bad)
        assert lib.dmn_create(ctypes.byref(d), 1, ctypes.byref(o), ctypes.byref(h)) == -1
        assert h.value is None and "warp_per_point must be -1, 0 or 1" in lib.dmn_last_error(None).decode()
    for bad in (4, 24, 64, -8):
        h = ctypes.c_void_p(123)
        o = dmn.Options_(1e-12, 50, dmn.PREC_F64, 0, 0, 0, 0, 0, 0, 0, bad)
        assert lib.dmn_create(ctypes.byref(d), 1, ctypes.byref(o), ctypes.byref(h)) == -1
        assert h.value is None and "warp_lanes must be 0, 8, 16 or 32" in lib.dmn_last_error(None).decode()
    assert [f[0] for f in dmn.Options_._fields_][-4:] == ["first_stage", "stage_ctas_per_sm", "warp_per_point",
                                                          "warp_lanes"]


def _noalloc(d, o, n=8, arrays=None):
    lib = dmn.load_library()
    arrays = arrays if arrays is not None else [None] * 10
    return lib.dmn_update_noalloc(ctypes.byref(d), None if o is None else ctypes.byref(o), n, *arrays, None), \
        lib.dmn_last_error(None).decode()


@pytest.mark.parametrize("case,msg", [
    (dict(opt=(1e-12, 50, dmn.PREC_MIXED, 0, 0, 0, 0)), "only the FP64 form"),
    (dict(opt=(1e-12, 50, dmn.PREC_F64, 0, 0, 0, 1)), "extrapolated start"),
    (dict(opt=(1e-12, 50, dmn.PREC_F64, 0, 0, 1, 0)), "line search"),
    (dict(w=np.r_[np.ones(7), 0.0]), "weights"),
    (dict(K=9), "K must be"),
    (dict(alias=True), "must differ"),
])
def test_allocation_free_update_rejects_what_it_does_not_offer(case, msg):
    """Each of these returns before any CUDA call, so it needs no GPU."""
    d, keep = _desc(K=case.get("K", 3), w=case.get("w"))
    o = dmn.Options_(*case["opt"]) if "opt" in case else None
    arrays = None
    if case.get("alias"):
        fake = [ctypes.c_void_p(4096 * (k + 1)) for k in range(10)]
        fake[5] = fake[4]   # state_out == state_in
        arrays = fake
    rc, err = _noalloc(d, o, arrays=arrays)
    assert rc == -1 and msg in err, (rc, err)


def test_calls_on_null_handle_are_argument_errors():
    lib = dmn.load_library()
    assert lib.dmn_update(None, 4, None, *([None] * 10), None) == -1
    lib.dmn_update_host.argtypes = [ctypes.c_void_p, ctypes.c_int64] + [ctypes.c_void_p] * 11 + [ctypes.c_int64,
                                                                                            ctypes.c_void_p]
    assert lib.dmn_update_host(None, 4, *([None] * 11), 0, None) == -1
    assert lib.dmn_interp_orientation(None, 4, None, None, None, None) == -1
    assert lib.dmn_state_size(None, 0) == -1
    assert lib.dmn_update_lanes_per_point(None, 16) == -1
    lib.dmn_destroy(None)


def test_state_size_formula():
    # 6 per inelastic leaf + 3 per laminate; the paper's count for K = 8 is 1533
    assert W.state_size(8) == 1533
    assert W.state_size(4) == 6 * 8 + 3 * 15
    assert W.state_size(3, (W.MATRIX, W.MATRIX)) == 6 * 8 + 3 * 7
