"""dmn_update_noalloc: the update for callers that cannot allocate device memory.

Such callers (code whose device memory is owned by an application's pool or
arena, or that may not call cudaMalloc after start-up) get an entry point whose
work space is a fixed static device array inside the library.  This test calls
it through the C ABI twice in a row -- the second call continuing from the
first call's state -- and checks each result against dmn_update on the same
inputs, and sampled points against the CPU oracle run along the same history.
It lives in its own file, collected last, and passes alone or after the other
tests.
"""
import ctypes

import numpy as np
import pytest
import torch

import oracle
from paper_2103_08253_gb300 import dmn, workloads as W

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda:0")


def _lib():
    lib = dmn.load_library()
    vp = ctypes.c_void_p
    lib.dmn_update_noalloc.argtypes = [ctypes.POINTER(dmn.TreeDesc_), ctypes.POINTER(dmn.Options_), ctypes.c_int64,
                                       vp, vp, vp, vp, vp, vp, vp, vp, vp, vp, vp]
    lib.dmn_update_noalloc.restype = ctypes.c_int
    return lib


def _desc(tree):
    keep = [np.ascontiguousarray(x, dtype=np.float64).reshape(-1) for x in (tree.p, tree.q, tree.w)]
    d = dmn.TreeDesc_()
    dp = ctypes.POINTER(ctypes.c_double)
    d.K, d.M = tree.K, tree.M
    d.p, d.q, d.w = (k.ctypes.data_as(dp) for k in keep)
    for f, ph in enumerate(tree.phases):
        d.phase[f] = dmn.Phase_(ph.kind, ph.E, ph.nu, ph.sigma0, ph.H)
    return d, keep


def _rel(a, b):
    a = a.reshape(a.shape[0], -1)
    b = b.reshape(b.shape[0], -1)
    return (np.linalg.norm(a - b, axis=1) / np.maximum(np.linalg.norm(b, axis=1), 1e-300)).max()


def test_noalloc_update_matches_dmn_update_on_two_calls_in_a_row():
    lib = _lib()
    K, n = 8, 3001
    tree = W.tree_d10_fit(K, seed=123)
    A2, lam, Q = W.orientation_field(n, seed=124)
    Ef = W.random6_path_final(n, 0.03, seed=125)
    S = W.state_size(K)
    d, keep = _desc(tree)
    m = dmn.DMN(tree, precision="f64", warp_per_point=-1)   # the organisation of the allocation-free call
    lam_d = torch.from_numpy(lam).to(DEV)
    Q_d = torch.from_numpy(Q).to(DEV)
    st_ref = torch.zeros((S, n), dtype=torch.float64, device=DEV)
    for step in range(1, 10):                  # a plastic history through the existing entry point
        En, dE = W.proportional_increment(Ef, step, 12)
        st_ref = m.update(lam_d, Q_d, torch.from_numpy(En).to(DEV), torch.from_numpy(dE).to(DEV), st_ref)["state_out"]
    st_na = st_ref.clone()
    stream = torch.cuda.current_stream(DEV).cuda_stream
    # the oracle along the same history, on its own states, for a sample of the points
    pidx = np.random.default_rng(126).choice(n, 12, replace=False)
    st_o = np.zeros((S, pidx.size))
    for step in range(1, 10):
        En, dE = W.proportional_increment(Ef, step, 12)
        st_o = oracle.update(tree, lam[pidx], Q[pidx], En[pidx], dE[pidx], st_o)[0]
    for step in (10, 11):                      # two consecutive calls, each continuing from its own last state
        En, dE = W.proportional_increment(Ef, step, 12)
        En_d, dE_d = torch.from_numpy(En).to(DEV), torch.from_numpy(dE).to(DEV)
        ref = m.update(lam_d, Q_d, En_d, dE_d, st_ref)
        out = m.alloc_outputs(n, DEV)
        p = lambda t: ctypes.c_void_p(t.data_ptr())
        rc = lib.dmn_update_noalloc(ctypes.byref(d), None, n, p(lam_d), p(Q_d), p(En_d), p(dE_d), p(st_na),
                                    p(out["state_out"]), p(out["stress"]), p(out["tangent"]), p(out["iters"]),
                                    p(out["status"]), ctypes.c_void_p(stream))
        assert rc == 0, lib.dmn_last_error(None).decode()
        torch.cuda.synchronize()
        assert torch.equal(out["status"], ref["status"]) and torch.equal(out["iters"], ref["iters"])
        ok = (ref["status"] == 0).cpu().numpy()
        assert ok.mean() > 0.99
        assert _rel(out["stress"].cpu().numpy()[ok], ref["stress"].cpu().numpy()[ok]) <= 1e-10
        assert _rel(out["tangent"].cpu().numpy()[ok], ref["tangent"].cpu().numpy()[ok]) <= 1e-10
        okd = torch.from_numpy(ok).to(DEV)
        so, sr = out["state_out"][:, okd], ref["state_out"][:, okd]
        scale = sr.abs().amax(dim=1, keepdim=True) + 1e-300
        assert ((so - sr).abs() / scale).max().item() <= 1e-9
        st_o, sig_o, C_o, it_o, stat_o, _ = oracle.update(tree, lam[pidx], Q[pidx], En[pidx], dE[pidx], st_o)
        keep_o = (stat_o == 0) & ok[pidx]
        assert keep_o.sum() >= 10
        assert _rel(out["stress"].cpu().numpy()[pidx][keep_o], sig_o[keep_o]) <= 1e-10
        assert _rel(out["tangent"].cpu().numpy()[pidx][keep_o], C_o[keep_o]) <= 1e-10
        st_ref, st_na = ref["state_out"], out["state_out"]
    m.close()


def test_noalloc_rejects_what_it_cannot_do():
    lib = _lib()
    tree = W.tree_d10_fit(3, seed=1)
    d, keep = _desc(tree)
    opt = dmn.Options_(1e-12, 50, dmn.PREC_MIXED, 0, 0)
    rc = lib.dmn_update_noalloc(ctypes.byref(d), ctypes.byref(opt), 8, *([None] * 10), None)
    assert rc == -1 and "only the FP64 form" in lib.dmn_last_error(None).decode()
    d.K = 9
    rc = lib.dmn_update_noalloc(ctypes.byref(d), None, 8, *([None] * 10), None)
    assert rc == -1 and "K must be" in lib.dmn_last_error(None).decode()


def test_python_binding_matches_dmn_update():
    """dmn.update_noalloc (the binding of the same entry point) on a depth-5 tree, along a plastic
    path: statuses and iteration counts equal, stress and tangent within 1e-10 of dmn_update."""
    K, n = 5, 777
    tree = W.tree_d10_fit(K, seed=126)
    A2, lam, Q = W.orientation_field(n, seed=127)
    Ef = W.random6_path_final(n, 0.03, seed=128)
    m = dmn.DMN(tree, precision="f64", warp_per_point=-1)   # the organisation of the allocation-free call
    lam_d, Q_d = torch.from_numpy(lam).to(DEV), torch.from_numpy(Q).to(DEV)
    st = torch.zeros((m.state_size, n), dtype=torch.float64, device=DEV)
    for step in range(1, 6):
        En, dE = W.proportional_increment(Ef, step, 8)
        args = (lam_d, Q_d, torch.from_numpy(En).to(DEV), torch.from_numpy(dE).to(DEV), st)
        ref = m.update(*args)
        out = dmn.update_noalloc(tree, *args)
        torch.cuda.synchronize()
        assert torch.equal(out["status"], ref["status"]) and torch.equal(out["iters"], ref["iters"])
        ok = (ref["status"] == 0).cpu().numpy()
        assert ok.mean() > 0.99
        assert _rel(out["stress"].cpu().numpy()[ok], ref["stress"].cpu().numpy()[ok]) <= 1e-10
        assert _rel(out["tangent"].cpu().numpy()[ok], ref["tangent"].cpu().numpy()[ok]) <= 1e-10
        st = ref["state_out"]
    m.close()
