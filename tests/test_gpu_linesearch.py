"""Backtracking line search (a step in (0, 1], Sec. 3.2) against the oracle's.

Large cyclic increments make plain Newton exhaust its iterations on some
reversal steps; with the line search every point converges and the GPU path
follows the oracle's accepted iterates (same trial steps, same halving rule)."""
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


@pytest.mark.parametrize("prec", ["f64", "mixed"])
def test_line_search_on_large_cyclic_steps(prec):
    K, n, n_steps = 6, 400, 8
    tree = W.tree_d10_fit(K, seed=500)
    A2, lam, Q = W.orientation_field(n, seed=501)
    amp = W.random6_path_final(n, 0.025, seed=502)
    S = W.state_size(K)
    plain_fail = 0
    m = dmn.DMN(tree, precision=prec, line_search=True)
    mp = dmn.DMN(tree, precision=prec)
    st_g = torch.zeros((S, n), dtype=torch.float64, device=DEV)
    st_o = np.zeros((S, n))
    worst = [0.0, 0.0]
    alive = np.ones(n, dtype=bool)
    for s in range(1, n_steps + 1):
        En, dE = W.cyclic_increment(amp, s, n_steps)
        plain = mp.update(d(lam), d(Q), d(En), d(dE), st_g)
        plain_fail += int((plain["status"] != 0).sum().item())
        out = m.update(d(lam), d(Q), d(En), d(dE), st_g)
        st_g = out["state_out"]
        st_o, so, Co, io, sto, gap = oracle.update(tree, lam, Q, En, dE, st_o, line_search=True)
        stat = out["status"].cpu().numpy()
        assert (sto == 0).mean() > 0.99 and (stat == 0).mean() > 0.99
        alive &= (sto == 0) & (stat == 0)
        sig, C, it = out["stress"].cpu().numpy(), out["tangent"].cpu().numpy(), out["iters"].cpu().numpy()
        worst[0] = max(worst[0], rel(sig[alive], so[alive]).max(initial=0.0))
        ok = alive & (gap > 1e-9)
        worst[1] = max(worst[1], rel(C[ok], Co[ok]).max(initial=0.0))
        if prec == "f64":
            assert np.abs(it[alive] - io[alive]).max(initial=0) <= 1
    print(prec, "plain Newton non-converged point-increments:", plain_fail, "worst", worst)
    assert plain_fail > 0                  # the load path needs the line search
    assert worst[0] <= TOL[prec] and worst[1] <= TOL[prec], worst
    assert alive.mean() > 0.97
    m.close()
    mp.close()


def test_line_search_reaches_the_plain_newton_solution_on_easy_steps():
    K, n = 5, 256
    tree = W.tree_d10_fit(K, seed=510)
    A2, lam, Q = W.orientation_field(n, seed=511)
    Ef = W.random6_path_final(n, 0.02, seed=512)
    S = W.state_size(K)
    a = dmn.DMN(tree, line_search=True)
    b = dmn.DMN(tree)
    sa = torch.zeros((S, n), dtype=torch.float64, device=DEV)
    sb = sa.clone()
    for s in range(1, 6):
        En, dE = W.proportional_increment(Ef, s, 20)
        oa = a.update(d(lam), d(Q), d(En), d(dE), sa)
        ob = b.update(d(lam), d(Q), d(En), d(dE), sb)
        sa, sb = oa["state_out"], ob["state_out"]
        assert torch.equal(oa["status"], ob["status"])
        # a shortened step changes the iterates, not the converged solution
        assert rel(oa["stress"].cpu().numpy(), ob["stress"].cpu().numpy()).max() < 1e-10


@pytest.mark.parametrize("prec", ["f64", "mixed-f32-tangent"])
def test_line_search_with_the_extrapolated_start(prec):
    """Both options at once (the FE driver's setting): the large cyclic steps above, where the
    extrapolation factor is clipped to 0 at the reversals and halvings occur, against the oracle
    with the same two options; stress, tangent, the whole state (jumps, leaf states, last jump
    change and strain increment) and iteration counts."""
    K, n, n_steps = 6, 400, 8
    tree = W.tree_d10_fit(K, seed=520)
    A2, lam, Q = W.orientation_field(n, seed=521)
    amp = W.random6_path_final(n, 0.025, seed=522)
    m = dmn.DMN(tree, precision=prec, line_search=True, predictor=True)
    S = m.state_size
    st_g = torch.zeros((S, n), dtype=torch.float64, device=DEV)
    st_o = np.zeros((S, n))
    tol_s, tol_c = (1e-10, 1e-10) if prec == "f64" else (1e-6, 1e-4)
    worst = [0.0, 0.0, 0.0]
    alive = np.ones(n, dtype=bool)
    for s in range(1, n_steps + 1):
        En, dE = W.cyclic_increment(amp, s, n_steps)
        out = m.update(d(lam), d(Q), d(En), d(dE), st_g)
        st_g = out["state_out"]
        st_o, so, Co, io, sto, gap = oracle.update(tree, lam, Q, En, dE, st_o, line_search=True, predictor=True)
        stat = out["status"].cpu().numpy()
        assert (sto == 0).mean() > 0.99 and (stat == 0).mean() > 0.99
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
    print(prec, "worst", worst, "alive", alive.mean())
    assert worst[0] <= tol_s and worst[1] <= tol_c, worst
    assert worst[2] <= (1e-9 if prec == "f64" else 1e-5), worst
    assert alive.mean() > 0.97
    m.close()
