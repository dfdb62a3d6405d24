"""Batching: several trees of different depth in one launch, invalid tree ids,
cyclic and elastic-range loading in the same batch, and CUDA-graph capture of
the update.  Every point is compared with the CPU oracle run on its own tree."""
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


def batch(n, seed):
    depths = (5, 6, 7, 8)
    trees = [W.tree_d10_fit(K, seed=seed + K) for K in depths]
    tid, elastic = W.mixed_depth_batch(n, seed, depths)
    A2, lam, Q = W.orientation_field(n, seed=seed + 1)
    Edir = W.random6_path_final(n, 1.0, seed=seed + 2)       # unit equivalent strain
    amp = np.where(elastic, 0.001, 0.02)[:, None] * Edir
    return trees, tid, elastic, lam, Q, amp


def path(amp, elastic, step, n_steps):
    En_c, dE_c = W.cyclic_increment(amp, step, n_steps)
    En_r, dE_r = W.proportional_increment(amp, min(step, n_steps // 2), n_steps // 2)
    if step > n_steps // 2:
        En_r, dE_r = amp.copy(), np.zeros_like(amp)
    e = elastic[:, None]
    return np.where(e, En_r, En_c), np.where(e, dE_r, dE_c)


@pytest.mark.parametrize("prec", ["f64", "mixed"])
def test_mixed_depth_cyclic_batch_against_oracle(prec):
    n, n_steps = 600, 16
    trees, tid, elastic, lam, Q, amp = batch(n, 300)
    tid[[3, 77]] = [-1, 9]                               # two points with unknown trees
    m = dmn.DMN(trees, precision=prec)
    assert m.state_size == max(m.tree_state_sizes) == W.state_size(8)
    st_g = torch.zeros((m.state_size, n), dtype=torch.float64, device=DEV)
    st_o = {k: np.zeros((m.tree_state_sizes[k], int((tid == k).sum()))) for k in range(4)}
    tid_d = d(tid)
    worst = [0.0, 0.0]
    alive = (tid >= 0) & (tid < 4)
    for s in range(1, n_steps + 1):
        En, dE = path(amp, elastic, s, n_steps)
        out = m.update(d(lam), d(Q), d(En), d(dE), st_g, tree_id=tid_d)
        st_g = out["state_out"]
        stat = out["status"].cpu().numpy()
        assert stat[3] == dmn.STATUS_BAD_TREE and stat[77] == dmn.STATUS_BAD_TREE
        assert np.isnan(out["stress"][3].cpu().numpy()).all()
        sig, C, it = out["stress"].cpu().numpy(), out["tangent"].cpu().numpy(), out["iters"].cpu().numpy()
        for k in range(4):
            idx = np.nonzero(tid == k)[0]
            st_o[k], so, Co, io, sto, gap = oracle.update(trees[k], lam[idx], Q[idx], En[idx], dE[idx], st_o[k])
            # plain Newton (no line search) may exhaust max_iter on a reversal step; such a
            # point's state then depends on rounding, so it leaves the comparison for good
            assert (sto != dmn.STATUS_NONFINITE).all()
            alive[idx] &= (sto == 0) & (stat[idx] == 0)
            a = alive[idx]
            worst[0] = max(worst[0], rel(sig[idx][a], so[a]).max(initial=0.0))
            ok = a & (gap > 1e-9)
            worst[1] = max(worst[1], rel(C[idx][ok], Co[ok]).max(initial=0.0))
            if prec == "f64":
                assert np.abs(it[idx][a] - io[a]).max(initial=0) <= 1
            sg = st_g[: m.tree_state_sizes[k]][:, idx[a]].cpu().numpy()
            ref = st_o[k][:, a]
            assert np.abs(sg - ref).max(initial=0.0) <= 1e-7 * (np.abs(ref).max(initial=0.0) + 1e-30)
    assert worst[0] <= TOL[prec] and worst[1] <= TOL[prec], worst
    assert alive.mean() > 0.9
    # the elastic-range half needs at most two corrections, the cyclic half more
    assert it[elastic & (tid >= 0) & (tid < 4)].max() <= 2
    m.close()


def test_update_is_capturable_in_a_cuda_graph():
    n, n_steps = 700, 6
    trees, tid, elastic, lam, Q, amp = batch(n, 400)
    m = dmn.DMN(trees, precision="mixed")
    S = m.state_size
    lam_d, Q_d, tid_d = d(lam), d(Q), d(tid)
    En_all = [d(path(amp, elastic, s, n_steps)[0]) for s in range(1, n_steps + 1)]
    dE_all = [d(path(amp, elastic, s, n_steps)[1]) for s in range(1, n_steps + 1)]
    # eager reference
    st = torch.zeros((S, n), dtype=torch.float64, device=DEV)
    eager = []
    for s in range(n_steps):
        o = m.update(lam_d, Q_d, En_all[s], dE_all[s], st, tree_id=tid_d)
        st = o["state_out"].clone()
        eager.append({k: v.clone() for k, v in o.items()})
    # graph of all increments, state ping-pong between two fixed buffers
    bufs = [torch.zeros((S, n), dtype=torch.float64, device=DEV) for _ in range(2)]
    outs = [m.alloc_outputs(n, DEV) for _ in range(n_steps)]
    for s in range(n_steps):
        outs[s]["state_out"] = bufs[(s + 1) % 2]
    m.update(lam_d, Q_d, En_all[0], dE_all[0], bufs[0], out=outs[0], tree_id=tid_d)  # work space allocated
    bufs[0].zero_()
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):
        with torch.cuda.graph(g, stream=side):
            for s in range(n_steps):
                m.update(lam_d, Q_d, En_all[s], dE_all[s], bufs[s % 2], out=outs[s], tree_id=tid_d)
    torch.cuda.current_stream().wait_stream(side)
    for rep in range(2):
        bufs[0].zero_()
        g.replay()
        torch.cuda.synchronize()
        for s in range(n_steps):
            for k in ("stress", "tangent", "iters", "status"):
                assert torch.equal(outs[s][k], eager[s][k]) or torch.allclose(outs[s][k], eager[s][k], equal_nan=True), (s, k)
        assert torch.equal(bufs[n_steps % 2], eager[-1]["state_out"])
    m.close()


@pytest.mark.parametrize("prec", ["f64", "mixed"])
def test_eight_trees_in_one_handle(prec):
    """The largest handle: 8 trees, depths 1-8, the exponential-linear matrix on every other
    tree, points of all trees interleaved at random; each point against the oracle on its tree."""
    rng = np.random.default_rng(600)
    trees = [W.tree_d10_fit(K, seed=600 + K, phases=(W.FIBER, W.MATRIX_EXPLIN if K % 2 else W.MATRIX))
             for K in range(1, 9)]
    n = 8 * 61 + 3
    tid = rng.permutation(np.arange(n) % 8).astype(np.int32)
    A2, lam, Q = W.orientation_field(n, seed=601)
    Ef = W.random6_path_final(n, 0.025, seed=602)
    m = dmn.DMN(trees, precision=prec)
    assert m.n_trees == dmn.MAX_TREES
    assert m.tree_state_sizes == [W.state_size(t.K, t.phases) for t in trees]
    st_g = torch.zeros((m.state_size, n), dtype=torch.float64, device=DEV)
    st_o = [np.zeros((m.tree_state_sizes[k], int((tid == k).sum()))) for k in range(8)]
    worst = [0.0, 0.0]
    alive = np.ones(n, dtype=bool)     # converged on both sides in every increment so far
    for s in range(1, 5):
        En, dE = W.proportional_increment(Ef, s, 10)
        out = m.update(d(lam), d(Q), d(En), d(dE), st_g, tree_id=d(tid))
        st_g = out["state_out"]
        sig, C, stat = out["stress"].cpu().numpy(), out["tangent"].cpu().numpy(), out["status"].cpu().numpy()
        it = out["iters"].cpu().numpy()
        for k in range(8):
            idx = np.nonzero(tid == k)[0]
            st_o[k], so, Co, io, sto, gap = oracle.update(trees[k], lam[idx], Q[idx], En[idx], dE[idx], st_o[k])
            # a point at max_iter keeps a rounding-dependent state: it leaves the comparison for good
            alive[idx] &= (sto == 0) & (stat[idx] == 0)
            a = alive[idx]
            worst[0] = max(worst[0], rel(sig[idx][a], so[a]).max(initial=0.0))
            ok = a & (gap > 1e-9)
            worst[1] = max(worst[1], rel(C[idx][ok], Co[ok]).max(initial=0.0))
            if prec == "f64":
                assert np.abs(it[idx][a] - io[a]).max(initial=0) <= 1
            sg = st_g[: m.tree_state_sizes[k]][:, idx[a]].cpu().numpy()
            ref = st_o[k][:, a]
            assert np.abs(sg - ref).max(initial=0.0) <= 1e-7 * (np.abs(ref).max(initial=0.0) + 1e-30), (k, s)
    assert worst[0] <= TOL[prec] and worst[1] <= TOL[prec], worst
    assert alive.mean() > 0.97
    m.close()
