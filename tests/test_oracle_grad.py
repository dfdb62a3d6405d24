"""Pins of the oracle's exact derivatives (dual numbers) and of its implicit-function gradient.

* The values a dual evaluation carries are those of the double oracle: R = A^T W sigma and
  sigma_bar of its Newton system, the algorithmic tangent of its update.
* Its derivatives along random directions in (p, q, w, E, a) agree with central differences
  of the double oracle's R, sigma_bar and tangent (h = 1e-6; the difference quotient's own
  error is ~1e-10 here), for linear and exponential-linear hardening, at plastic iterates.
* Linear-elastic trees: the stiffness is Milton's laminate recursion (Sec. 3.1), which is
  analytic in p, q, w; its complex-step derivative (exact to rounding) must equal the dual
  derivative of the tangent and, through sigma_bar = C E, the implicit-function gradient.
* The adjoint assembly (one solve with J) equals the forward, tangent-linear route
  (da = -J^-1 dR/dtheta), and dL/dE equals C^T g.
* The gradient of the full Newton solve equals central differences of the converged
  solve (stress seed and tangent seed).
"""
import types

import numpy as np
import pytest

import oracle
from paper_2103_08253_gb300 import workloads as W
from test_oracle_pins import C_FIB, C_MAT, ELASTIC_MATRIX, linear_dmn_alpha

H = 1e-6


def _path(tree, n, steps, seed, n_steps=10):
    A2, lam, Q = W.orientation_field(n, seed=seed)
    Ef = W.random6_path_final(n, 0.03, seed=seed + 1)
    S = oracle.state_size(tree.K, tree.phases)
    st = np.zeros((S, n))
    prev = st
    for s in range(1, steps + 1):
        En, dE = W.proportional_increment(Ef, s, n_steps)
        prev = st
        st = oracle.update(tree, lam, Q, En, dE, st)[0]
    return lam, Q, En, dE, prev, st


def _E_loc(Q, E):
    _, e = oracle.rotate(np.asarray(Q).reshape(3, 3).T, np.zeros((6, 6)), E)
    return e


def _directions(tree, n_a, rng):
    return dict(dp=rng.standard_normal(tree.p.shape), dq=rng.standard_normal(tree.q.shape),
                dw=rng.standard_normal(tree.w.shape) * tree.w, dE=rng.standard_normal(6) * 1e-3,
                da=rng.standard_normal(n_a) * 1e-4)


def _rel(a, b):
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


@pytest.mark.parametrize("K,matrix", [(3, "linear"), (4, "linear"), (4, "explin"), (5, "linear")])
def test_dual_values_and_derivatives_match_the_double_oracle(K, matrix):
    phases = (W.FIBER, W.MATRIX_EXPLIN if matrix == "explin" else W.MATRIX)
    tree = W.tree_d10_fit(K, seed=20 + K, phases=phases)
    lam, Q, En, dE, prev, st = _path(tree, 2, 7, seed=30 + K)
    rng = np.random.default_rng(K)
    n_plastic = 0
    for i in range(2):
        z = oracle.leaf_states(tree, prev, i)
        # a plastic iterate away from the solution: R is not small there
        a = oracle.jumps(tree, st, i) + rng.standard_normal(3 * W.n_nodes(tree.K)) * 1e-4
        E = _E_loc(Q[i], (En + dE)[i])
        d = _directions(tree, a.size, rng)
        r = oracle.eval_dual(tree, lam[i, 0], lam[i, 1], E, a, z, tangent=True, **d)
        ns = oracle.newton_system(tree, lam[i, 0], lam[i, 1], E, a, z)
        assert _rel(r["R"], ns["R"]) < 1e-12
        assert _rel(r["sbar"], ns["sbar"]) < 1e-13
        n_plastic += int(np.any(z[:, 0] > 0))   # leaves that have yielded before

        def at(sc):
            t2 = types.SimpleNamespace(**vars(tree))
            t2.p, t2.q, t2.w = tree.p + sc * d["dp"], tree.q + sc * d["dq"], tree.w + sc * d["dw"]
            return (oracle.newton_system(t2, lam[i, 0], lam[i, 1], E + sc * d["dE"], a + sc * d["da"], z),
                    oracle.eval_dual(t2, lam[i, 0], lam[i, 1], E + sc * d["dE"], a + sc * d["da"], z,
                                     tangent=True)["C"])
        (np_, Cp), (nm, Cm) = at(H), at(-H)
        assert _rel(r["dR"], (np_["R"] - nm["R"]) / (2 * H)) < 1e-7
        assert _rel(r["dsbar"], (np_["sbar"] - nm["sbar"]) / (2 * H)) < 1e-7
        assert _rel(r["dC"], (Cp - Cm) / (2 * H)) < 1e-6
    assert n_plastic > 0


def test_dual_tangent_value_is_the_update_tangent():
    K = 4
    tree = W.tree_d10_fit(K, seed=41)
    lam, Q, En, dE, prev, st = _path(tree, 3, 6, seed=42)
    out = oracle.update(tree, lam, Q, En, dE, prev)
    for i in range(3):
        Cl, _ = oracle.rotate(Q[i].reshape(3, 3).T, out[2][i], np.zeros(6))
        r = oracle.eval_dual(tree, lam[i, 0], lam[i, 1], _E_loc(Q[i], (En + dE)[i]), oracle.jumps(tree, st, i),
                             oracle.leaf_states(tree, prev, i), tangent=True)
        assert _rel(r["C"], Cl) < 1e-12


def _linear_dmn(tree, p, q, w, lam1, lam2):
    """Milton's laminate recursion of the linear DMN (complex-safe: analytic in p, q, w)."""
    phi = oracle.barycentric(lam1, lam2)
    al, be = p @ phi, q @ phi
    nrm = np.stack([np.sin(al) * np.cos(be), np.sin(al) * np.sin(be), np.cos(al)], axis=1)
    t = types.SimpleNamespace(K=tree.K, w=w)
    return linear_dmn_alpha(t, (C_FIB, C_MAT), nrm, 3e5)


@pytest.mark.parametrize("K", [2, 3, 5])
def test_elastic_derivatives_are_exact_by_complex_step(K):
    tree = W.tree_d10_fit(K, seed=50 + K, phases=(W.FIBER, ELASTIC_MATRIX))
    A2, lam, Q = W.orientation_field(2, seed=51 + K)
    rng = np.random.default_rng(52 + K)
    h = 1e-30
    for i in range(2):
        d = _directions(tree, 3 * W.n_nodes(tree.K), rng)
        cs = _linear_dmn(tree, tree.p + 1j * h * d["dp"], tree.q + 1j * h * d["dq"], tree.w + 1j * h * d["dw"],
                         *lam[i])
        dC_cs = cs.imag / h
        E = rng.standard_normal(6) * 1e-3
        z = np.zeros((1 << K, 7))
        r = oracle.eval_dual(tree, lam[i, 0], lam[i, 1], E, np.zeros(3 * W.n_nodes(K)), z, d["dp"], d["dq"],
                             d["dw"], tangent=True)
        assert _rel(r["C"], cs.real) < 1e-11
        assert _rel(r["dC"], dC_cs) < 1e-10
        # implicit-function gradient of g.sigma_bar + G:C at the solution of E: sigma_bar = C E
        S = oracle.state_size(K, tree.phases)
        Qm = Q[i].reshape(3, 3)
        _, Eg = oracle.rotate(Qm, np.zeros((6, 6)), E)
        st = oracle.update(tree, lam[i:i + 1], Q[i:i + 1], np.zeros((1, 6)), Eg[None], np.zeros((S, 1)))[0]
        g, G = rng.standard_normal(6), rng.standard_normal((6, 6))
        Gg, gg = oracle.rotate(Qm, G, g)     # seeds given in the global frame
        full = oracle.gradient_ift(tree, lam[i], Q[i], Eg, oracle.jumps(tree, st, 0), z, gg, G_glob=Gg)
        pred = (full["p"] * d["dp"]).sum() + (full["q"] * d["dq"]).sum() + (full["w"] * d["dw"]).sum()
        exact = g @ (dC_cs @ E) + (G * dC_cs).sum()
        assert abs(pred - exact) <= 1e-10 * abs(exact)


@pytest.mark.parametrize("K,steps", [(3, 6), (4, 8)])
def test_adjoint_equals_forward_sensitivities_and_strain_gradient_is_tangent(K, steps):
    tree = W.tree_d10_fit(K, seed=60 + K)
    lam, Q, En, dE, prev, st = _path(tree, 2, steps, seed=61 + K)
    C = oracle.update(tree, lam, Q, En, dE, prev)[2]
    rng = np.random.default_rng(62 + K)
    for i in range(2):
        z = oracle.leaf_states(tree, prev, i)
        a = oracle.jumps(tree, st, i)
        g, G = rng.standard_normal(6), rng.standard_normal((6, 6))
        dirs = [(rng.standard_normal(tree.p.shape), rng.standard_normal(tree.q.shape),
                 rng.standard_normal(tree.w.shape) * tree.w) for _ in range(2)]
        for Gs in (None, G):
            full = oracle.gradient_ift(tree, lam[i], Q[i], (En + dE)[i], a, z, g, G_glob=Gs)
            fwd = oracle.gradient_ift(tree, lam[i], Q[i], (En + dE)[i], a, z, g, directions=dirs, G_glob=Gs)
            for (dp, dq, dw), v in zip(dirs, fwd):
                pred = (full["p"] * dp).sum() + (full["q"] * dq).sum() + (full["w"] * dw).sum()
                assert abs(pred - v) <= 1e-10 * abs(v)
            if Gs is None:
                np.testing.assert_allclose(full["E"], C[i].T @ g, rtol=0, atol=1e-12 * np.abs(C[i].T @ g).max())


@pytest.mark.parametrize("K,steps", [(2, 1), (3, 6), (4, 8)])
def test_ift_gradient_matches_finite_differences_of_the_solve(K, steps):
    tree = W.tree_d10_fit(K, seed=20 + K)
    lam, Q, En, dE, prev, st = _path(tree, 2, steps, seed=30 + K)
    rng = np.random.default_rng(K)
    for i in range(2):
        g, G = rng.standard_normal(6), rng.standard_normal((6, 6))
        dp, dq = rng.standard_normal(tree.p.shape), rng.standard_normal(tree.q.shape)
        dw = rng.standard_normal(tree.w.shape) * tree.w
        for Gs in (None, G):
            full = oracle.gradient_ift(tree, lam[i], Q[i], (En + dE)[i], oracle.jumps(tree, st, i),
                                       oracle.leaf_states(tree, prev, i), g, G_glob=Gs)
            pred = (full["p"] * dp).sum() + (full["q"] * dq).sum() + (full["w"] * dw).sum()

            def f(sc):
                t2 = types.SimpleNamespace(**vars(tree))
                t2.p, t2.q, t2.w = tree.p + sc * dp, tree.q + sc * dq, tree.w + sc * dw
                out = oracle.update(t2, lam[i:i + 1], Q[i:i + 1], En[i:i + 1], dE[i:i + 1], prev[:, i:i + 1])
                return g @ out[1][0] + (0.0 if Gs is None else (Gs * out[2][0]).sum())
            fd = (f(H) - f(-H)) / (2 * H)
            assert abs(pred - fd) <= 1e-6 * abs(fd) + 1e-9
