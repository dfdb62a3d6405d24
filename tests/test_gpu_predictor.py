"""GPU parity of the extrapolated start (dmn_options.predictor = 1) with the
oracle's same option, through the C ABI.

Both sides start each update's Newton iteration from the last update's jumps
extrapolated along the new strain increment and then take the same iterates,
so the tolerances of the plain parity tests apply: FP64 <= 1e-10 relative in
stress and tangent and iteration counts within one; the mixed form with an FP32
tangent <= 1e-6 in stress and 1e-4 in tangent.  The state's extra fields (jump
change, strain increment) are compared too.  Also covered: a compressed tree, a
handle of several depths, dmn_update_host, and the state size.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2103_08253_gb300 import dmn, workloads as W

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda:0")
TOL = {"f64": (1e-10, 1e-10), "mixed-f32-tangent": (1e-6, 1e-4)}


def d(x):
    return torch.from_numpy(np.ascontiguousarray(x)).to(DEV)


def rel(a, b):
    a = a.reshape(a.shape[0], -1)
    b = b.reshape(b.shape[0], -1)
    return np.linalg.norm(a - b, axis=1) / np.maximum(np.linalg.norm(b, axis=1), 1e-300)


def run(tree, lam, Q, Ef, n_inc, prec, cyclic=False):
    n = lam.shape[0]
    S0, J = oracle.jump_fields(tree)
    m = dmn.DMN(tree, precision=prec, predictor=True)
    assert m.state_size == S0 + J + 6
    st_g = torch.zeros((m.state_size, n), dtype=torch.float64, device=DEV)
    st_o = np.zeros((m.state_size, n))
    worst = dict(stress=0.0, tangent=0.0, state=0.0, iters=0, restarts=0)
    its = []
    clean = np.ones(n, dtype=bool)   # converged in every increment so far (both sides agree on status)
    for s in range(1, n_inc + 1):
        En, dE = (W.cyclic_increment(Ef, s, n_inc) if cyclic else W.proportional_increment(Ef, s, 50))
        out = m.update(d(lam), d(Q), d(En), d(dE), st_g)
        st_g = out["state_out"]
        st_o, sig, C, it, stat, gap = oracle.update(tree, lam, Q, En, dE, st_o, predictor=True)
        torch.cuda.synchronize()
        sg_stat = out["status"].cpu().numpy()
        np.testing.assert_array_equal(sg_stat[clean], stat[clean])
        clean &= stat == 0
        ok = clean & (gap >= 1e-9)
        worst["stress"] = max(worst["stress"], rel(out["stress"].cpu().numpy()[clean], sig[clean]).max(initial=0.0))
        worst["tangent"] = max(worst["tangent"], rel(out["tangent"].cpu().numpy()[ok], C[ok]).max(initial=0.0))
        sg = st_g.cpu().numpy()
        scale = np.abs(st_o[:, clean]).max(axis=1, keepdims=True) + 1e-300
        worst["state"] = max(worst["state"], (np.abs(sg[:, clean] - st_o[:, clean]) / scale).max(initial=0.0))
        np.testing.assert_array_equal(sg[S0 + J:], dE.T)              # strain increment stored exactly
        gi = out["iters"].cpu().numpy()
        worst["iters"] = max(worst["iters"], int(np.abs(gi[clean] - it[clean]).max(initial=0)))
        worst["restarts"] += int((it > oracle.PRED_TRIES).sum())
        its.append(gi.mean())
    worst["clean"] = float(clean.mean())
    m.close()
    return worst, its


@pytest.mark.parametrize("prec", ["f64", "mixed-f32-tangent"])
def test_depth8_random_paths(prec):
    tree = W.tree_d10_fit(8, seed=130)
    A2, lam, Q = W.orientation_field(48, seed=131)
    Ef = W.random6_path_final(48, 0.03, seed=132)
    worst, its = run(tree, lam, Q, Ef, 10, prec)
    print(prec, worst, np.round(its, 2))
    assert worst["stress"] <= TOL[prec][0] and worst["tangent"] <= TOL[prec][1], worst
    assert worst["state"] <= (1e-9 if prec == "f64" else 1e-5), worst
    if prec == "f64":
        assert worst["iters"] <= 1


def test_compressed_tree_and_cyclic_path():
    tree = W.tree_with_zero_weights(6, seed=140)
    A2, lam, Q = W.orientation_field(64, seed=141)
    Ef = W.random6_path_final(64, 0.02, seed=142)
    worst, _ = run(tree, lam, Q, Ef, 24, "f64", cyclic=True)     # load reversals: rho = 0 there
    print(worst)
    assert worst["stress"] <= 1e-10 and worst["tangent"] <= 1e-10 and worst["state"] <= 1e-9, worst
    assert worst["clean"] >= 0.9 and worst["iters"] <= 1, worst


def test_several_depths_and_host_buffers():
    """A handle of depths 4 and 7 with the extrapolated start: each tree's state has its
    own size; dmn_update_host gives dmn_update's results bit for bit."""
    trees = [W.tree_d10_fit(4, seed=150), W.tree_d10_fit(7, seed=151)]
    n = 300
    tid = (np.arange(n) % 2).astype(np.int32)
    A2, lam, Q = W.orientation_field(n, seed=152)
    Ef = W.random6_path_final(n, 0.03, seed=153)
    m = dmn.DMN(trees, predictor=True)
    sizes = [sum(oracle.jump_fields(t)) + 6 for t in trees]
    assert m.tree_state_sizes == sizes and m.state_size == max(sizes)
    st = torch.zeros((m.state_size, n), dtype=torch.float64, device=DEV)
    st_h = torch.zeros((m.state_size, n), dtype=torch.float64).pin_memory()
    so = [np.zeros((sizes[k], int((tid == k).sum()))) for k in range(2)]
    for s in range(1, 6):
        En, dE = W.proportional_increment(Ef, s, 50)
        out = m.update(d(lam), d(Q), d(En), d(dE), st, tree_id=d(tid))
        oh = m.update_host(torch.from_numpy(lam).pin_memory(), torch.from_numpy(Q).pin_memory(),
                           torch.from_numpy(En).pin_memory(), torch.from_numpy(dE).pin_memory(), st_h,
                           out=dict(m.alloc_host_outputs(n), state_out=st_h), tree_id=torch.from_numpy(tid))
        torch.cuda.synchronize()
        for key in ("stress", "tangent", "iters", "status"):
            np.testing.assert_array_equal(oh[key].numpy().reshape(out[key].shape), out[key].cpu().numpy())
        for k in range(2):
            idx = np.nonzero(tid == k)[0]
            np.testing.assert_array_equal(st_h.numpy()[:sizes[k], idx], out["state_out"].cpu().numpy()[:sizes[k], idx])
            so[k], sig, C, it, stat, gap = oracle.update(trees[k], lam[idx], Q[idx], En[idx], dE[idx], so[k],
                                                         predictor=True)
            assert rel(out["stress"].cpu().numpy()[idx], sig).max() <= 1e-10
        st = out["state_out"]
    m.close()


def test_adjoint_on_a_handle_with_the_extrapolated_start():
    """dmn_grad reads the jumps and leaf states of the longer state: its gradients match those of
    a handle with the paper's start at the same path (the two converged states agree to the
    stopping criterion, so the gradients to 1e-6)."""
    tree = W.tree_d10_fit(5, seed=160)
    n = 16
    A2, lam, Q = W.orientation_field(n, seed=161)
    Ef = W.random6_path_final(n, 0.03, seed=162)
    g = np.random.default_rng(163).standard_normal((n, 6))
    grads = []
    for pred in (False, True):
        m = dmn.DMN(tree, predictor=pred)
        st = torch.zeros((m.state_size, n), dtype=torch.float64, device=DEV)
        for s in range(1, 7):
            En, dE = W.proportional_increment(Ef, s, 20)
            prev = st
            st = m.update(d(lam), d(Q), d(En), d(dE), prev)["state_out"]
        gp, gq, gw, gE = m.grad(d(lam), d(Q), d(En), d(dE), prev, st, d(g))
        grads.append([x.cpu().numpy() for x in (gp, gq, gw, gE)])
        m.close()
    for a, b in zip(*grads):
        assert np.abs(a - b).max() <= 1e-6 * np.abs(a).max(), np.abs(a - b).max() / np.abs(a).max()
