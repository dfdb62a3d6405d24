"""Adjoint (dmn_grad) and the torch.autograd bindings.

* GPU gradient vs the oracle's implicit-function gradient (exact partial
  derivatives by dual numbers, Cholesky solve with J), full parameter vectors,
  to 1e-9;
* GPU gradient vs central finite differences (h = 1e-6) of the converged
  solve, along random parameter directions (target: <= 1e-5 relative);
* dL/dE = C^T g against the tangent;
* depth-8 training loss of elastic stiffnesses and elastoplastic stresses
  against a seeded target DMN, through torch.autograd, vs finite differences.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2103_08253_gb300 import autograd as ag, dmn, workloads as W

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda:0")
EL_MATRIX = W.Phase(0, 3000.0, 0.35)


def d(x):
    return torch.from_numpy(np.ascontiguousarray(x)).to(DEV)


def states(tree, lam, Q, Ef, steps, n_steps):
    """GPU run of `steps` increments; returns (state before the last, state after, E_n, dE of the last)."""
    m = dmn.DMN(tree)
    n = lam.shape[0]
    st = torch.zeros((m.state_size, n), dtype=torch.float64, device=DEV)
    prev = st
    for s in range(1, steps + 1):
        En, dE = W.proportional_increment(Ef, s, n_steps)
        prev = st
        st = m.update(d(lam), d(Q), d(En), d(dE), st)["state_out"]
    return m, prev, st, En, dE


@pytest.mark.parametrize("K,steps", [(3, 1), (3, 6), (5, 7)])
def test_adjoint_matches_oracle_ift_gradient(K, steps):
    n = 3
    tree = W.tree_d10_fit(K, seed=60 + K)
    A2, lam, Q = W.orientation_field(n, seed=61 + K)
    Ef = W.random6_path_final(n, 0.03, seed=62 + K)
    m, prev, st, En, dE = states(tree, lam, Q, Ef, steps, 10)
    g = np.random.default_rng(K).standard_normal((n, 6))
    g_p, g_q, g_w, g_E = m.grad(d(lam), d(Q), d(En), d(dE), prev, st, d(g))
    # oracle on its own states
    S = oracle.state_size(K, tree.phases)
    so = np.zeros((S, n))
    so_prev = so
    for s in range(1, steps + 1):
        E1, d1 = W.proportional_increment(Ef, s, 10)
        so_prev = so
        so = oracle.update(tree, lam, Q, E1, d1, so)[0]
    tot = dict(p=0.0, q=0.0, w=0.0)
    for i in range(n):
        gi = oracle.gradient_ift(tree, lam[i], Q[i], (En + dE)[i], oracle.jumps(tree, so, i),
                                 oracle.leaf_states(tree, so_prev, i), g[i])
        for k in tot:
            tot[k] = tot[k] + gi[k]
    for k, gg in (("p", g_p), ("q", g_q), ("w", g_w)):
        ref = tot[k]
        err = np.abs(gg.cpu().numpy() - ref).max() / np.abs(ref).max()
        assert err < 1e-9, (k, err)
    # dL/dE = C^T g with C the algorithmic tangent of the update
    C = m.update(d(lam), d(Q), d(En), d(dE), prev)["tangent"].cpu().numpy()
    np.testing.assert_allclose(g_E.cpu().numpy(), np.einsum("nji,nj->ni", C, g), rtol=1e-10, atol=1e-10)


def test_adjoint_of_a_compressed_tree_matches_oracle_ift_gradient():
    """Leaf weights of zero: the adjoint walks the compressed tree; laminates that are
    passed through and weightless leaves get no gradient."""
    n, K, steps = 3, 5, 6
    tree = W.tree_with_zero_weights(K, seed=70)
    A2, lam, Q = W.orientation_field(n, seed=71)
    Ef = W.random6_path_final(n, 0.03, seed=72)
    m = dmn.DMN(tree)
    S = oracle.state_size(K, tree.phases, tree.w)
    assert m.state_size == S
    st = torch.zeros((S, n), dtype=torch.float64, device=DEV)
    so = np.zeros((S, n))
    for s in range(1, steps + 1):
        En, dE = W.proportional_increment(Ef, s, 10)
        prev, so_prev = st, so
        st = m.update(d(lam), d(Q), d(En), d(dE), st)["state_out"]
        so = oracle.update(tree, lam, Q, En, dE, so)[0]
    g = np.random.default_rng(73).standard_normal((n, 6))
    g_p, g_q, g_w, _ = m.grad(d(lam), d(Q), d(En), d(dE), prev, st, d(g))
    tot = dict(p=0.0, q=0.0, w=0.0)
    for i in range(n):
        gi = oracle.gradient_ift(tree, lam[i], Q[i], (En + dE)[i], oracle.jumps(tree, so, i),
                                 oracle.leaf_states(tree, so_prev, i), g[i])
        for k in tot:
            tot[k] = tot[k] + gi[k]
    for k, gg in (("p", g_p), ("q", g_q), ("w", g_w)):
        ref = tot[k]
        err = np.abs(gg.cpu().numpy() - ref).max() / np.abs(ref).max()
        assert err < 1e-9, (k, err)
    assert (g_w.cpu().numpy()[tree.w == 0] == 0).all()
    m.close()


def test_adjoint_matches_finite_differences_of_the_solve():
    K, n = 6, 16
    tree = W.tree_d10_fit(K, seed=70)
    A2, lam, Q = W.orientation_field(n, seed=71)
    Ef = W.random6_path_final(n, 0.03, seed=72)
    m, prev, st, En, dE = states(tree, lam, Q, Ef, 5, 10)
    g = np.random.default_rng(5).standard_normal((n, 6))
    g_p, g_q, g_w, _ = m.grad(d(lam), d(Q), d(En), d(dE), prev, st, d(g))
    rng = np.random.default_rng(6)
    h = 1e-6
    for _ in range(3):
        dp, dq = rng.standard_normal(tree.p.shape), rng.standard_normal(tree.q.shape)
        dw = rng.standard_normal(tree.w.shape) * tree.w
        pred = (g_p.cpu().numpy() * dp).sum() + (g_q.cpu().numpy() * dq).sum() + (g_w.cpu().numpy() * dw).sum()
        vals = []
        for sc in (h, -h):
            m.set_params(tree.p + sc * dp, tree.q + sc * dq, tree.w + sc * dw)
            sig = m.update(d(lam), d(Q), d(En), d(dE), prev)["stress"].cpu().numpy()
            vals.append((g * sig).sum())
        m.set_params(tree.p, tree.q, tree.w)
        fd = (vals[0] - vals[1]) / (2 * h)
        assert abs(pred - fd) <= 1e-5 * abs(fd), (pred, fd)


def test_training_loss_through_autograd_depth8():
    """Depth-8 DMN with trainable angle coefficients and leaf weights: relative
    Frobenius errors of elastic stiffnesses and of elastoplastic stresses
    (one increment from the virgin state, 1-3 % equivalent strain) against a
    seeded target DMN; autograd gradient vs finite differences."""
    K, ne, npl = 8, 64, 64
    base = W.tree_d10_fit(K, seed=80)
    target = W.tree_d10_fit(K, seed=81)
    el = W.TreeParams(K, 3, base.p, base.q, base.w, (W.FIBER, EL_MATRIX))
    A2e, lame, Qe = W.orientation_field(ne, seed=82)
    A2p, lamp, Qp = W.orientation_field(npl, seed=83)
    rng = np.random.default_rng(84)
    Ep = W.random6_path_final(npl, 1.0, seed=85) * rng.uniform(0.01, 0.03, (npl, 1))
    # one large increment from the virgin state: the line search keeps Newton convergent
    m_el, m_pl = dmn.DMN(el), dmn.DMN(base, line_search=True)
    t_el = dmn.DMN(W.TreeParams(K, 3, target.p, target.q, target.w, (W.FIBER, EL_MATRIX)))
    t_pl = dmn.DMN(target, line_search=True)
    z = lambda nn: torch.zeros((m_pl.state_size, nn), dtype=torch.float64, device=DEV)
    zE = torch.zeros((npl, 6), dtype=torch.float64, device=DEV)
    with torch.no_grad():
        C_t = ag.dmn_stiffness(t_el, d(lame), d(Qe), d(target.p), d(target.q), d(target.w))
        s_t = ag.dmn_stress(t_pl, d(lamp), d(Qp), zE, d(Ep), z(npl), d(target.p), d(target.q), d(target.w))[0]

    def loss(p, q, w):
        C = ag.dmn_stiffness(m_el, d(lame), d(Qe), p, q, w)
        s, _, stat = ag.dmn_stress(m_pl, d(lamp), d(Qp), zE, d(Ep), z(npl), p, q, w)
        assert (stat == 0).all()
        le = (torch.linalg.norm((C - C_t).reshape(ne, -1), dim=1) / torch.linalg.norm(C_t.reshape(ne, -1), dim=1)).mean()
        lp = (torch.linalg.norm(s - s_t, dim=1) / torch.linalg.norm(s_t, dim=1)).mean()
        return le + lp

    p = d(base.p).requires_grad_()
    q = d(base.q).requires_grad_()
    w = d(base.w).requires_grad_()
    L = loss(p, q, w)
    L.backward()
    h = 1e-6
    for trial in range(3):
        dp, dq = rng.standard_normal(base.p.shape), rng.standard_normal(base.q.shape)
        dw = rng.standard_normal(base.w.shape) * base.w
        pred = float((p.grad.cpu().numpy() * dp).sum() + (q.grad.cpu().numpy() * dq).sum()
                     + (w.grad.cpu().numpy() * dw).sum())
        with torch.no_grad():
            Lp = loss(d(base.p + h * dp), d(base.q + h * dq), d(base.w + h * dw)).item()
            Lm = loss(d(base.p - h * dp), d(base.q - h * dq), d(base.w - h * dw)).item()
        fd = (Lp - Lm) / (2 * h)
        assert abs(pred - fd) <= 1e-5 * abs(fd), (trial, pred, fd)


def _elastic(tree):
    return W.TreeParams(tree.K, tree.M, tree.p, tree.q, tree.w, (W.FIBER, EL_MATRIX))


@pytest.mark.parametrize("K,compressed", [(3, False), (5, False), (6, False), (5, True), (6, True)])
def test_tangent_seed_adjoint_matches_the_exact_oracle_gradient(K, compressed):
    """dmn_grad with g_tangent on a tree of elastic phases (the linear DMN of the offline
    training, Sec. 3.1): the reverse pass through the laminate recursion against the oracle's
    dual-number gradient of G : C, summed over the points, to 1e-9; full and compressed trees."""
    base = W.tree_with_zero_weights(K, seed=90 + K) if compressed else W.tree_d10_fit(K, seed=90 + K)
    tree = _elastic(base)
    n = 4
    A2, lam, Q = W.orientation_field(n, seed=91 + K)
    G = np.random.default_rng(92 + K).standard_normal((n, 6, 6))
    m = dmn.DMN(tree)
    g_p, g_q, g_w, g_E = m.grad(d(lam), d(Q), None, None, None, None, None, g_tangent=d(G.reshape(n, 36)))
    assert np.abs(g_E.cpu().numpy()).max() == 0.0
    S = oracle.state_size(K, tree.phases, tree.w)
    nz = 0
    a0 = np.zeros(S)                      # the solution at zero strain: no jumps
    z = np.zeros((1 << K, 7))
    tot = dict(p=0.0, q=0.0, w=0.0)
    for i in range(n):
        gi = oracle.gradient_ift(tree, lam[i], Q[i], np.zeros(6), a0[6 * nz:], z, np.zeros(6), G_glob=G[i])
        for k in tot:
            tot[k] = tot[k] + gi[k]
    for k, gg in (("p", g_p), ("q", g_q), ("w", g_w)):
        ref = tot[k]
        err = np.abs(gg.cpu().numpy() - ref).max() / np.abs(ref).max()
        assert err < 1e-9, (k, err)
    if compressed:
        assert (g_w.cpu().numpy()[tree.w == 0] == 0).all()
    m.close()


def test_tangent_seed_at_depth8_matches_oracle_directional_derivatives():
    K, n = 8, 3
    tree = _elastic(W.tree_d10_fit(K, seed=95))
    A2, lam, Q = W.orientation_field(n, seed=96)
    rng = np.random.default_rng(97)
    G = rng.standard_normal((n, 6, 6))
    m = dmn.DMN(tree)
    g_p, g_q, g_w, _ = m.grad(d(lam), d(Q), None, None, None, None, None, g_tangent=d(G.reshape(n, 36)))
    dirs = [(rng.standard_normal(tree.p.shape), rng.standard_normal(tree.q.shape),
             rng.standard_normal(tree.w.shape) * tree.w) for _ in range(2)]
    ref = np.zeros(len(dirs))
    for i in range(n):
        ref += np.asarray(oracle.gradient_ift(tree, lam[i], Q[i], np.zeros(6), np.zeros(3 * 255),
                                              np.zeros((256, 7)), np.zeros(6), directions=dirs, G_glob=G[i]))
    pred = np.array([(g_p.cpu().numpy() * dp).sum() + (g_q.cpu().numpy() * dq).sum() + (g_w.cpu().numpy() * dw).sum()
                     for dp, dq, dw in dirs])
    assert np.abs(pred - ref).max() <= 1e-9 * np.abs(ref).max(), (pred, ref)
    m.close()


def test_stress_and_tangent_seeds_add_and_the_stiffness_paths_agree():
    """Both seeds in one call give the sum of the two calls; dmn_stiffness through the tangent
    (one update, one tangent adjoint per sample) equals the six-stress path in value and gradient."""
    K, n = 5, 8
    tree = _elastic(W.tree_d10_fit(K, seed=98))
    A2, lam, Q = W.orientation_field(n, seed=99)
    rng = np.random.default_rng(100)
    m = dmn.DMN(tree)
    E = d(rng.standard_normal((n, 6)) * 1e-3)
    z = torch.zeros((m.state_size, n), dtype=torch.float64, device=DEV)
    zE = torch.zeros_like(E)
    out = m.update(d(lam), d(Q), zE, E, z)
    g, G = d(rng.standard_normal((n, 6))), d(rng.standard_normal((n, 36)))
    both = m.grad(d(lam), d(Q), zE, E, z, out["state_out"], g, g_tangent=G)
    s_only = m.grad(d(lam), d(Q), zE, E, z, out["state_out"], g)
    t_only = m.grad(d(lam), d(Q), None, None, None, None, None, g_tangent=G)
    for a, b, c in zip(both[:3], s_only[:3], t_only[:3]):
        np.testing.assert_allclose(a.cpu().numpy(), (b + c).cpu().numpy(), rtol=1e-12,
                                   atol=1e-12 * np.abs((b + c).cpu().numpy()).max())
    np.testing.assert_allclose(both[3].cpu().numpy(), s_only[3].cpu().numpy(), rtol=1e-13, atol=0)
    p, q, w = (d(x).requires_grad_() for x in (tree.p, tree.q, tree.w))
    Gs = d(rng.standard_normal((n, 6, 6)))
    grads = []
    Cs = []
    for method in ("tangent", "stress"):
        for x in (p, q, w):
            x.grad = None
        C = ag.dmn_stiffness(m, d(lam), d(Q), p, q, w, method=method)
        (C * Gs).sum().backward()
        Cs.append(C.detach().cpu().numpy())
        grads.append([x.grad.cpu().numpy().copy() for x in (p, q, w)])
    np.testing.assert_allclose(Cs[0], Cs[1], rtol=0, atol=1e-10 * np.abs(Cs[1]).max())
    for a, b in zip(*grads):
        np.testing.assert_allclose(a, b, rtol=0, atol=1e-8 * np.abs(b).max())
    m.close()


def test_tangent_seed_needs_elastic_phases():
    tree = W.tree_d10_fit(3, seed=101)
    m = dmn.DMN(tree)
    A2, lam, Q = W.orientation_field(2, seed=102)
    with pytest.raises(RuntimeError, match="elastic phases"):
        m.grad(d(lam), d(Q), None, None, None, None, None, g_tangent=d(np.ones((2, 36))))
    m.close()
