"""The warp organisation for small batches (heap trees): a point per group of 32, 16 or 8 lanes of a
warp, through the C ABI.

The warp kernel runs the same per-laminate functions as the thread-per-point kernel, level by level
with the group's lanes sharing a level; the residual's sum of squares is added in another order, and the two
kernels are compiled separately, so their roundings differ.  Its iterates must be those of the
thread-per-point kernel to rounding (the same statuses, the same correction counts except where the
criterion ties within rounding) and it must meet the oracle's tolerances in every form, with and
without the line search, at depths 1..8 and ragged batch sizes.
"""
import numpy as np
import pytest
import torch

from paper_2103_08253_gb300 import dmn, workloads as W
from test_gpu_parity import d, rel, run_path

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda:0")


@pytest.mark.parametrize("prec,lanes", [("f64", 32), ("mixed", 32), ("mixed-f32-tangent", 32), ("f64", 16),
                                        ("f64", 8), ("mixed", 8)])
def test_warp_kernel_reproduces_the_thread_kernel(prec, lanes):
    K, n = 8, 1000
    tree = W.tree_d10_fit(K, seed=401)
    A2, lam, Q = W.orientation_field(n, seed=402)
    Ef = W.random6_path_final(n, 0.03, seed=403)
    outs = {}
    for mode in (1, -1):
        m = dmn.DMN(tree, precision=prec, warp_per_point=mode, first_stage=False,
                    warp_lanes=lanes if mode == 1 else 0)
        st = torch.zeros((m.state_size, n), dtype=torch.float64, device=DEV)
        for s in range(1, 6):
            En, dE = W.proportional_increment(Ef, s, 20)
            out = m.update(d(lam), d(Q), d(En), d(dE), st)
            st = out["state_out"]
        outs[mode] = {k: v.cpu().numpy() for k, v in out.items()}
        m.close()
    a, b = outs[1], outs[-1]
    np.testing.assert_array_equal(a["status"], b["status"])
    same = a["iters"] == b["iters"]
    assert same.mean() >= 0.99
    tol = {"f64": 1e-11, "mixed": 1e-8, "mixed-f32-tangent": 1e-8}[prec]
    assert rel(a["stress"][same], b["stress"][same]).max() <= tol
    assert rel(a["tangent"][same], b["tangent"][same]).max() <= (tol if prec != "mixed-f32-tangent" else 1e-5)
    assert rel(a["stress"], b["stress"]).max() <= 1e-9


@pytest.mark.parametrize("prec,lanes", [("f64", 32), ("mixed", 32), ("mixed-f32-tangent", 32), ("f64", 8),
                                        ("mixed-f32-tangent", 16)])
def test_warp_kernel_against_the_oracle_ragged(prec, lanes):
    tol_t = {"f64": 1e-10, "mixed": 1e-6, "mixed-f32-tangent": 1e-4}[prec]
    tol_s = {"f64": 1e-10, "mixed": 1e-6, "mixed-f32-tangent": 1e-6}[prec]
    for K, n in ((1, 1), (2, 33), (3, 129), (5, 257), (8, 37)):
        tree = W.tree_d10_fit(K, seed=410 + K)
        A2, lam, Q = W.orientation_field(n, seed=420 + K)
        Ef = W.random6_path_final(n, 0.025, seed=430 + K)
        worst, out, _ = run_path(tree, lam, Q, Ef, 4, prec, warp_per_point=1, warp_lanes=lanes)
        assert worst["stress"] <= tol_s and worst["tangent"] <= tol_t, (K, n, worst)


@pytest.mark.parametrize("lanes", [32, 8])
def test_warp_kernel_with_the_line_search(lanes):
    """Large cyclic steps, where the line search halves steps: the warp kernel's two buffers (accepted and
    trial) against the thread kernel's, and the oracle's line search."""
    import oracle
    K, n, n_steps = 7, 300, 8
    tree = W.tree_d10_fit(K, seed=440)
    A2, lam, Q = W.orientation_field(n, seed=441)
    amp = W.random6_path_final(n, 0.025, seed=442)
    S = W.state_size(K)
    ms = {mode: dmn.DMN(tree, precision="f64", line_search=True, warp_per_point=mode,
                        warp_lanes=lanes if mode == 1 else 0) for mode in (1, -1)}
    st = {mode: torch.zeros((S, n), dtype=torch.float64, device=DEV) for mode in ms}
    so = np.zeros((S, n))
    for s in range(1, n_steps + 1):
        En, dE = W.cyclic_increment(amp, s, n_steps)
        outs = {}
        for mode, m in ms.items():
            outs[mode] = m.update(d(lam), d(Q), d(En), d(dE), st[mode])
            st[mode] = outs[mode]["state_out"]
        so, sig_o, C_o, it_o, stat_o, gap = oracle.update(tree, lam, Q, En, dE, so, line_search=True)
        a, b = ({k: v.cpu().numpy() for k, v in outs[mode].items()} for mode in (1, -1))
        ok = (stat_o == 0) & (a["status"] == 0) & (b["status"] == 0)
        assert ok.mean() > 0.97
        assert rel(a["stress"][ok], sig_o[ok]).max() <= 1e-10
        assert rel(a["stress"][ok], b["stress"][ok]).max() <= 1e-10
    for m in ms.values():
        m.close()


@pytest.mark.parametrize("lanes", [32, 16])
def test_warp_kernel_unknown_tree_and_several_depths(lanes):
    """Several heap trees of different depths in one handle, points selected by tree_id, one of them out
    of range: the warp kernel reports it and updates the others as the thread kernel does."""
    trees = [W.tree_d10_fit(K, seed=450 + K) for K in (5, 8)]
    n = 500
    A2, lam, Q = W.orientation_field(n, seed=460)
    Ef = W.random6_path_final(n, 0.03, seed=461)
    tid = (np.arange(n) % 2).astype(np.int32)
    tid[7] = 5
    En, dE = W.proportional_increment(Ef, 6, 20)
    outs = {}
    for mode in (1, -1):
        m = dmn.DMN(trees, precision="f64", warp_per_point=mode, warp_lanes=lanes if mode == 1 else 0)
        st = torch.zeros((m.state_size, n), dtype=torch.float64, device=DEV)
        outs[mode] = {k: v.cpu().numpy() for k, v in m.update(d(lam), d(Q), d(En), d(dE), st,
                                                               tree_id=d(tid)).items()}
        m.close()
    a, b = outs[1], outs[-1]
    assert a["status"][7] == dmn.STATUS_BAD_TREE and b["status"][7] == dmn.STATUS_BAD_TREE
    ok = np.arange(n) != 7
    same = ok & (a["iters"] == b["iters"])
    assert same.sum() >= 0.99 * ok.sum()
    assert rel(a["stress"][same], b["stress"][same]).max() <= 1e-11


@pytest.mark.parametrize("lanes", [32, 8])
def test_warp_kernel_points_are_independent_of_the_batch(lanes):
    """In the warp organisation too a point's update depends on that point alone: the same points as
    two uneven parts in the reverse order give the whole batch's results bit for bit."""
    K, n, cut = 7, 3000, 1801
    tree = W.tree_d10_fit(K, seed=470)
    A2, lam, Q = W.orientation_field(n, seed=471)
    Ef = W.random6_path_final(n, 0.03, seed=472)
    m = dmn.DMN(tree, precision="mixed", warp_per_point=1, warp_lanes=lanes)
    lam_d, Q_d = d(lam), d(Q)
    st = torch.zeros((m.state_size, n), dtype=torch.float64, device=DEV)
    for s in range(1, 4):
        En, dE = W.proportional_increment(Ef, s, 20)
        En_d, dE_d = d(En), d(dE)
        whole = m.update(lam_d, Q_d, En_d, dE_d, st)
        parts = {}
        for a, b in ((cut, n), (0, cut)):
            o = m.update(lam_d[a:b], Q_d[a:b], En_d[a:b], dE_d[a:b], st[:, a:b].contiguous())
            for k, v in o.items():
                parts.setdefault(k, [None, None])[0 if a == 0 else 1] = v
        for k, (lo, hi) in parts.items():
            assert torch.equal(torch.cat([lo, hi], dim=1 if k == "state_out" else 0), whole[k]), (s, k)
        st = whole["state_out"]
    m.close()


@pytest.mark.parametrize("prec,per_sm,lanes", [("f64", 1024, 8), ("mixed", 256, 16)])
def test_the_default_organisation_is_chosen_per_call(prec, per_sm, lanes):
    """By default a call of at most 1024 points per SM (FP64 form) or 256 (mixed forms) runs the warp
    kernel, with 32 lanes per point up to 16 points per SM and 8 (FP64) or 16 (mixed) above, and a
    larger call the thread kernel: bit for bit the results of warp_per_point = 1 and -1.
    dmn_update_host decides on the whole call, so its chunks get the kernel of the device call;
    first_stage = True keeps the thread kernel with its stage."""
    K = 5
    n_sm = torch.cuda.get_device_properties(DEV).multi_processor_count
    limit = per_sm * n_sm
    tree = W.tree_d10_fit(K, seed=480)
    handles = {mode: dmn.DMN(tree, precision=prec, warp_per_point=mode) for mode in (0, 1, -1)}
    assert handles[0].lanes_per_point(16 * n_sm) == 32 and handles[0].lanes_per_point(16 * n_sm + 1) == lanes
    for n in (limit, limit + 1):
        A2, lam, Q = W.orientation_field(n, seed=481)
        Ef = W.random6_path_final(n, 0.03, seed=482)
        En, dE = W.proportional_increment(Ef, 6, 20)
        S = handles[0].state_size
        st = torch.zeros((S, n), dtype=torch.float64, device=DEV)
        outs = {mode: m.update(d(lam), d(Q), d(En), d(dE), st) for mode, m in handles.items()}
        ref = outs[1] if n <= limit else outs[-1]
        assert handles[0].lanes_per_point(n) == (lanes if n <= limit else 1)
        assert handles[1].lanes_per_point(n) == lanes and handles[-1].lanes_per_point(n) == 1
        for k in outs[0]:
            assert torch.equal(outs[0][k], ref[k]), (n, k)
        # the same call from host arrays in chunks smaller than the limit
        out_h = handles[0].update_host(*(torch.from_numpy(np.ascontiguousarray(x)) for x in (lam, Q, En, dE)),
                                       torch.zeros((S, n), dtype=torch.float64), chunk=limit // 3)
        for k in ("stress", "iters", "status"):
            assert np.array_equal(out_h[k].numpy().reshape(outs[0][k].shape), outs[0][k].cpu().numpy()), (n, k)
    for m in handles.values():
        m.close()
    m = dmn.DMN(tree, precision="f64", first_stage=True)
    n = 512
    assert m.lanes_per_point(n) == 1
    A2, lam, Q = W.orientation_field(n, seed=483)
    Ef = W.random6_path_final(n, 0.03, seed=484)
    En, dE = W.proportional_increment(Ef, 6, 20)
    m.profile(True)
    m.update(d(lam), d(Q), d(En), d(dE), torch.zeros((m.state_size, n), dtype=torch.float64, device=DEV))
    _, passes, _ = m.profile_read_stages()
    assert passes["stage"] >= n
    m.close()


@pytest.mark.parametrize("prec,lanes", [("f64", 8), ("f64", 32), ("mixed", 16), ("mixed-f32-tangent", 16)])
def test_warp_kernel_on_compressed_trees(prec, lanes):
    """Trees with weightless leaves in the warp organisation (level by level of the full tree's heap
    positions, kept laminates at their positions, leaves beside laminates evaluated by their parent)
    against the oracle's compression, and against the thread kernel's table traversal to rounding."""
    import oracle
    tol_s = {"f64": 1e-10, "mixed": 1e-6, "mixed-f32-tangent": 1e-6}[prec]
    tol_t = {"f64": 1e-10, "mixed": 1e-6, "mixed-f32-tangent": 1e-4}[prec]
    for K, n in ((5, 65), (7, 300), (8, 129)):
        tree = W.tree_with_zero_weights(K, seed=490 + K)
        A2, lam, Q = W.orientation_field(n, seed=500 + K)
        Ef = W.random6_path_final(n, 0.03, seed=510 + K)
        S = oracle.state_size(K, tree.phases, tree.w)
        ms = {mode: dmn.DMN(tree, precision=prec, warp_per_point=mode, warp_lanes=lanes if mode == 1 else 0)
              for mode in (1, -1)}
        assert ms[1].lanes_per_point(n) == lanes and ms[-1].lanes_per_point(n) == 1
        st = {mode: torch.zeros((S, n), dtype=torch.float64, device=DEV) for mode in ms}
        so = np.zeros((S, n))
        for s in range(1, 7):
            En, dE = W.proportional_increment(Ef, s, 20)
            outs = {}
            for mode, m in ms.items():
                outs[mode] = {k: v.cpu().numpy() for k, v in m.update(d(lam), d(Q), d(En), d(dE), st[mode]).items()}
                st[mode] = torch.from_numpy(outs[mode]["state_out"]).to(DEV)
            so, sig_o, C_o, it_o, stat_o, gap = oracle.update(tree, lam, Q, En, dE, so)
            a, b = outs[1], outs[-1]
            ok = (stat_o == 0) & (a["status"] == 0)
            assert ok.mean() > 0.95, (K, s)
            assert rel(a["stress"][ok], sig_o[ok]).max() <= tol_s, (K, s)
            tie = gap < 1e-9
            assert rel(a["tangent"][ok & ~tie], C_o[ok & ~tie]).max() <= tol_t, (K, s)
            # per-field scale, floored at 1e-5 of the largest field: some fields of these trees are zero
            # to rounding (a jump of a laminate whose children still deform alike)
            scale = np.maximum(np.abs(so[:, ok]).max(axis=1, keepdims=True), 1e-5 * np.abs(so[:, ok]).max())
            if prec == "f64":
                assert (np.abs(a["state_out"][:, ok] - so[:, ok]) / scale).max() <= 1e-9, (K, s)
            np.testing.assert_array_equal(a["status"], b["status"])
            assert rel(a["stress"], b["stress"]).max() <= (1e-10 if prec == "f64" else 1e-8), (K, s)
        for m in ms.values():
            m.close()


def test_warp_kernel_on_a_compressed_tree_with_the_line_search():
    """The line search's two buffers on a compressed tree, large cyclic steps, against the oracle's line
    search; the same statuses as the thread kernel."""
    import oracle
    K, n, n_steps = 7, 200, 8
    tree = W.tree_with_zero_weights(K, seed=520)
    A2, lam, Q = W.orientation_field(n, seed=521)
    amp = W.random6_path_final(n, 0.025, seed=522)
    S = oracle.state_size(K, tree.phases, tree.w)
    ms = {mode: dmn.DMN(tree, precision="f64", line_search=True, warp_per_point=mode) for mode in (0, -1)}
    assert ms[0].lanes_per_point(n) == 32 and ms[0].lanes_per_point(4096) == 8
    st = {mode: torch.zeros((S, n), dtype=torch.float64, device=DEV) for mode in ms}
    so = np.zeros((S, n))
    for s in range(1, n_steps + 1):
        En, dE = W.cyclic_increment(amp, s, n_steps)
        outs = {}
        for mode, m in ms.items():
            outs[mode] = m.update(d(lam), d(Q), d(En), d(dE), st[mode])
            st[mode] = outs[mode]["state_out"]
        so, sig_o, C_o, it_o, stat_o, gap = oracle.update(tree, lam, Q, En, dE, so, line_search=True)
        a, b = ({k: v.cpu().numpy() for k, v in outs[mode].items()} for mode in (0, -1))
        ok = (stat_o == 0) & (a["status"] == 0) & (b["status"] == 0)
        assert ok.mean() > 0.95
        assert rel(a["stress"][ok], sig_o[ok]).max() <= 1e-10
        assert rel(a["stress"][ok], b["stress"][ok]).max() <= 1e-10
    for m in ms.values():
        m.close()
