"""Compressed trees (leaf weights of zero, Sec. 3.1) on the GPU.

Parity with the oracle's compression; agreement to rounding between the
table-driven traversal and the heap traversal on equivalent trees (a full
tree walked both ways; a tree whose right half is weightless against the
depth-(K-1) tree of its left half).  The two traversals are separately
compiled code, so the compiler's choice of fused multiply-adds may differ
between them: the comparison allows 1e-12 relative instead of bit equality."""
import numpy as np
import pytest
import torch

import oracle
from paper_2103_08253_gb300 import dmn, workloads as W

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda:0")
TOL = {"f64": 1e-10, "mixed": 1e-6}


def d(x):
    return torch.from_numpy(np.ascontiguousarray(x)).to(DEV)


def rel(a, b):
    a = a.reshape(a.shape[0], -1)
    b = b.reshape(b.shape[0], -1)
    return np.linalg.norm(a - b, axis=1) / np.maximum(np.linalg.norm(b, axis=1), 1e-300)


def close(x, y, tol=1e-12):
    """Equal to rounding: same iterations and status, values within tol of the array's scale."""
    if x.dtype.kind == "i":
        np.testing.assert_array_equal(x, y)
    else:
        assert np.abs(x - y).max() <= tol * (np.abs(y).max() + 1e-300)


def gpu_path(m, lam, Q, Ef, steps, n_steps, tree_id=None, S=None):
    n = lam.shape[0]
    st = torch.zeros((S or m.state_size, n), dtype=torch.float64, device=DEV)
    outs = []
    for s in range(1, steps + 1):
        En, dE = W.proportional_increment(Ef, s, n_steps)
        o = m.update(d(lam), d(Q), d(En), d(dE), st, tree_id=tree_id)
        st = o["state_out"]
        outs.append({k: v.cpu().numpy() for k, v in o.items()})
    return outs


@pytest.mark.parametrize("K,prec", [(5, "f64"), (8, "f64"), (8, "mixed")])
def test_compressed_tree_matches_the_oracle(K, prec):
    tree = W.tree_with_zero_weights(K, seed=20 + K)
    n, steps, n_steps = 40, 8, 20
    A2, lam, Q = W.orientation_field(n, seed=21)
    Ef = W.random6_path_final(n, 0.03, seed=22)
    m = dmn.DMN(tree, precision=prec)
    S = oracle.state_size(K, tree.phases, tree.w)
    assert m.state_size == S < W.state_size(K)
    outs = gpu_path(m, lam, Q, Ef, steps, n_steps)
    st = np.zeros((S, n))
    for s in range(1, steps + 1):
        En, dE = W.proportional_increment(Ef, s, n_steps)
        st, sig, C, it, stat, gap = oracle.update(tree, lam, Q, En, dE, st)
        o = outs[s - 1]
        np.testing.assert_array_equal(o["status"], stat)
        ok = stat == 0
        assert rel(o["stress"][ok], sig[ok]).max() <= TOL[prec]
        tie = gap < 1e-9
        assert rel(o["tangent"][ok & ~tie], C[ok & ~tie]).max() <= TOL[prec]
        if prec == "f64":
            assert np.abs(o["iters"] - it).max() <= 1
            # leaf variables and jumps, each against the largest entry of its block (a leaf that
            # barely yields at one point may flip with the rounding order there)
            nz6 = 6 * int(sum(1 for l in range(1 << K) if tree.w[l] > 0 and tree.phases[l % 2].kind != 0))
            for blk in (slice(0, nz6), slice(nz6, S)):
                ref = st[blk]
                assert np.abs(o["state_out"][blk] - ref).max() <= 1e-9 * (np.abs(ref).max() + 1e-300)
    m.close()


@pytest.mark.parametrize("prec", ["f64", "mixed"])
def test_table_traversal_equals_the_heap_traversal(prec):
    """A handle that holds a compressed tree walks every tree by tables; the full tree
    in it must give exactly what a handle of the full tree alone (heap arithmetic) gives."""
    K, n = 6, 200
    full = W.tree_d10_fit(K, seed=30)
    other = W.tree_with_zero_weights(4, seed=31)
    A2, lam, Q = W.orientation_field(n, seed=32)
    Ef = W.random6_path_final(n, 0.03, seed=33)
    # the thread-per-point kernel's heap and table arithmetic
    heap = dmn.DMN(full, precision=prec, warp_per_point=-1)
    table = dmn.DMN([full, other], precision=prec, warp_per_point=-1)
    assert table.tree_state_sizes[0] == heap.state_size
    a = gpu_path(heap, lam, Q, Ef, 4, 10)
    b = gpu_path(table, lam, Q, Ef, 4, 10, tree_id=d(np.zeros(n, dtype=np.int32)))
    for x, y in zip(a, b):
        # the mixed form's FP32 condensation rounds differently in the two traversals: its iterates,
        # and so the converged jumps, agree to the FP64 criterion, not to the last bit
        tol = 1e-12 if prec == "f64" else 1e-9
        for k in ("stress", "tangent", "iters", "status"):
            close(x[k], y[k], tol)
        close(x["state_out"], y["state_out"][: heap.state_size], tol)
    heap.close()
    table.close()


def test_weightless_half_equals_the_smaller_tree():
    K = 5
    big = W.tree_d10_fit(K, seed=40)
    w = big.w.copy()
    w[16:] = 0.0
    big = W.TreeParams(K, big.M, big.p, big.q, w, big.phases)
    rows = [(1 << K) - (1 << k) + i - 1 for k in range(K, 1, -1) for i in range(1, (1 << (k - 2)) + 1)]
    small = W.TreeParams(K - 1, big.M, big.p[rows], big.q[rows], w[:16], big.phases)
    n = 100
    A2, lam, Q = W.orientation_field(n, seed=41)
    Ef = W.random6_path_final(n, 0.03, seed=42)
    mb, ms = dmn.DMN(big), dmn.DMN(small)
    assert mb.state_size == ms.state_size
    for x, y in zip(gpu_path(mb, lam, Q, Ef, 4, 10), gpu_path(ms, lam, Q, Ef, 4, 10)):
        for k in x:
            close(x[k], y[k])


def test_single_leaf_parameters_and_gradient():
    K = 3
    t = W.tree_d10_fit(K, seed=50)
    w = np.zeros(1 << K)
    w[3] = 1.0
    t = W.TreeParams(K, t.M, t.p, t.q, w, t.phases)
    m = dmn.DMN(t)
    assert m.state_size == 6
    lam, Q = W.identity_orientation(5)
    Ef = W.random6_path_final(5, 0.03, seed=51)
    o = gpu_path(m, lam, Q, Ef, 3, 3)[-1]
    st = np.zeros((6, 5))
    for s in range(1, 4):
        En, dE = W.proportional_increment(Ef, s, 3)
        st, sig, C, it, stat, gap = oracle.update(t, lam, Q, En, dE, st)
    assert (o["status"] == 0).all() and (o["iters"] == 0).all()
    assert rel(o["stress"], sig).max() <= 1e-12 and rel(o["tangent"], C).max() <= 1e-12
    m.set_params(t.p + 0.1, t.q, 2.0 * t.w)          # same zero pattern: accepted
    w2 = t.w.copy()
    w2[0] = 0.5
    with pytest.raises(RuntimeError):                # another compressed tree: a new handle is needed
        m.set_params(t.p, t.q, w2)
    # one leaf left: the stress does not depend on p, q or w
    st0 = torch.zeros((6, 5), dtype=torch.float64, device=DEV)
    En, dE = W.proportional_increment(Ef, 3, 3)
    o = m.update(d(lam), d(Q), d(En), d(dE), st0)
    g_p, g_q, g_w, g_E = m.grad(d(lam), d(Q), d(En), d(dE), st0, o["state_out"], d(np.ones((5, 6))))
    assert float(g_p.abs().max()) == 0.0 and float(g_q.abs().max()) == 0.0 and float(g_w.abs().max()) == 0.0
    m.close()


@pytest.mark.parametrize("prec,ls", [("f64", True), ("mixed-f32-tangent", False), ("mixed-f32-tangent", True)])
def test_compressed_tree_with_line_search_and_fp32_tangent(prec, ls):
    """The table-driven traversal in its other instantiations: the line search (large cyclic
    steps, where it halves) and the mixed form with an FP32 tangent, against the oracle with the
    same options on a depth-7 tree compressed to 90 leaves."""
    K, n, n_steps = 7, 200, 8
    tree = W.tree_with_zero_weights(K, seed=540)
    A2, lam, Q = W.orientation_field(n, seed=541)
    amp = W.random6_path_final(n, 0.025, seed=542)
    m = dmn.DMN(tree, precision=prec, line_search=ls)
    S = oracle.state_size(K, tree.phases, tree.w)
    assert m.state_size == S
    st_g = torch.zeros((S, n), dtype=torch.float64, device=DEV)
    st_o = np.zeros((S, n))
    tol_s, tol_c = (1e-10, 1e-10) if prec == "f64" else (1e-6, 1e-4)
    worst = [0.0, 0.0, 0.0]
    alive = np.ones(n, dtype=bool)
    for s in range(1, n_steps + 1):
        En, dE = W.cyclic_increment(amp, s, n_steps) if ls else W.proportional_increment(amp, s, 20)
        out = m.update(d(lam), d(Q), d(En), d(dE), st_g)
        st_g = out["state_out"]
        st_o, so, Co, io, sto, gap = oracle.update(tree, lam, Q, En, dE, st_o, line_search=ls)
        stat = out["status"].cpu().numpy()
        alive &= (sto == 0) & (stat == 0)
        sig, C, it = out["stress"].cpu().numpy(), out["tangent"].cpu().numpy(), out["iters"].cpu().numpy()
        worst[0] = max(worst[0], rel(sig[alive], so[alive]).max(initial=0.0))
        ok = alive & (gap > 1e-9)
        worst[1] = max(worst[1], rel(C[ok], Co[ok]).max(initial=0.0))
        sg = st_g.cpu().numpy()
        scale = np.abs(st_o[:, alive]).max(axis=1, keepdims=True) + 1e-300
        worst[2] = max(worst[2], (np.abs(sg[:, alive] - st_o[:, alive]) / scale).max(initial=0.0))
        if prec == "f64":
            assert np.abs(it[alive] - io[alive]).max(initial=0) <= 1
    print(prec, ls, "worst", worst, "alive", alive.mean())
    assert worst[0] <= tol_s and worst[1] <= tol_c, worst
    assert worst[2] <= (1e-9 if prec == "f64" else 1e-5), worst
    assert alive.mean() > 0.97
    m.close()
