"""Pins of the oracle's extrapolated start (the `predictor` option of oracle.update).

The paper starts every update's Newton iteration from the last converged jumps
(Sec. 4.7).  The option starts from a^n + rho (a^n - a^{n-1}) with
rho = (dE . dE_prev) / (dE_prev . dE_prev) clipped to [0, 1], and restarts a
point from a^n when PRED_TRIES corrections have not converged.  What pins it:

* With both phases linear elastic, the laminate equilibrium (Sec. 3.2) is a
  linear system, so the jumps are a linear function of the macro strain.  On
  an increment parallel to the previous one with 0 < rho <= 1, the start is
  then the solution: zero Newton corrections (repeated increment, rho = 1;
  halved, rho = 1/2).  A wrong sign, factor or field index breaks this.  A
  reversed or orthogonal increment has rho = 0: the paper's start, bit for
  bit, and one correction.  A doubled increment is clipped to rho = 1: not the
  solution, one correction.
* A point whose extrapolated attempt fails restarts from a^n: its result is the
  paper start's and its count is PRED_TRIES more (a cyclic path with large
  increments, where the undamped Newton iteration fails from the
  extrapolation after a reversal).
* On the first update (zero state), rho = 0: bit-identical to the paper's start.
* On plastic paths the solution is the same (the incremental problem has one
  solution) up to the stopping criterion, reached with fewer corrections; also
  on a compressed tree, whose jump fields are fewer.
* The extra state fields hold this update's jump change and dE.
"""
import numpy as np

import oracle
from paper_2103_08253_gb300 import workloads as W

ELASTIC = (W.FIBER, W.Phase(0, 3000.0, 0.35))


def ext_state(tree, n):
    S0, J = oracle.jump_fields(tree)
    return np.zeros((S0 + J + 6, n)), S0, J


def test_elastic_tree_exact_start_needs_no_correction():
    K, n = 4, 12
    tree = W.tree_d10_fit(K, seed=1, phases=ELASTIC)
    A2, lam, Q = W.orientation_field(n, seed=2)
    rng = np.random.default_rng(3)
    d0 = rng.standard_normal((n, 6)) * 1e-3
    st, S0, J = ext_state(tree, n)
    E = np.zeros((n, 6))
    st, sig, C, it, stat, _ = oracle.update(tree, lam, Q, E, d0, st, predictor=True)
    assert (it == 1).all() and (stat == 0).all()          # rho = 0: the paper's start, one correction
    np.testing.assert_array_equal(st[S0 + J:], d0.T)       # the strain increment is stored
    E = E + d0
    for scale, exact in ((1.0, True), (0.5, True), (-1.0, False), (2.0, False)):
        dE = scale * st[S0 + J:].T
        st_p, sig_p, _, it_p, stat_p, _ = oracle.update(tree, lam, Q, E, dE, st, predictor=True)
        st_0, sig_0, _, it_0, _, _ = oracle.update(tree, lam, Q, E, dE, st[:S0])
        assert (stat_p == 0).all() and (it_0 == 1).all()
        if exact:
            assert (it_p == 0).all(), (scale, it_p)
        else:
            assert (it_p == 1).all(), (scale, it_p)
        if scale < 0:   # rho = 0
            np.testing.assert_array_equal(sig_p, sig_0)
            np.testing.assert_array_equal(st_p[:S0], st_0)
        np.testing.assert_allclose(sig_p, sig_0, rtol=1e-10, atol=1e-12 * np.abs(sig_0).max())
        np.testing.assert_allclose(st_p[S0:S0 + J], st_p[S0 - J:S0] - st[S0 - J:S0], atol=1e-18)
        E, st = E + dE, st_p
    # an increment orthogonal to the last one: rho = 0, the paper's start
    last = st[S0 + J:].T
    v = rng.standard_normal((n, 6))
    v -= (np.einsum("ni,ni->n", v, last) / np.einsum("ni,ni->n", last, last))[:, None] * last
    st_p, _, _, it_p, _, _ = oracle.update(tree, lam, Q, E, 1e-3 * v, st, predictor=True)
    st_0, _, _, it_0, _, _ = oracle.update(tree, lam, Q, E, 1e-3 * v, st[:S0])
    np.testing.assert_array_equal(it_p, it_0)
    np.testing.assert_allclose(st_p[:S0], st_0, rtol=1e-12, atol=1e-15)   # rho is 0 up to rounding


def _path(tree, n, n_inc, seed):
    A2, lam, Q = W.orientation_field(n, seed=seed)
    Ef = W.random6_path_final(n, 0.03, seed=seed + 1)
    S0 = oracle.state_size(tree.K, tree.phases, tree.w)
    sp, _, _ = ext_state(tree, n)
    s0 = np.zeros((S0, n))
    its = [[], []]
    for s in range(1, n_inc + 1):
        En, dE = W.proportional_increment(Ef, s, 50)
        sp, sig_p, C_p, it_p, stat_p, _ = oracle.update(tree, lam, Q, En, dE, sp, predictor=True)
        s0, sig_0, C_0, it_0, stat_0, _ = oracle.update(tree, lam, Q, En, dE, s0)
        assert (stat_p == 0).all() and (stat_0 == 0).all()
        if s == 1:   # zero state: rho = 0, bit-identical
            np.testing.assert_array_equal(sig_p, sig_0)
            np.testing.assert_array_equal(it_p, it_0)
        err = np.abs(sig_p - sig_0).max() / np.abs(sig_0).max()
        assert err <= 1e-7, (s, err)
        assert np.abs(C_p - C_0).max() <= 1e-6 * np.abs(C_0).max()
        its[0].append(it_0.mean())
        its[1].append(it_p.mean())
    return np.array(its)


def test_plastic_path_same_solution_fewer_corrections():
    its = _path(W.tree_d10_fit(5, seed=10), 16, 14, seed=11)
    assert its[1, 3:].mean() < its[0, 3:].mean() - 0.3, its


def test_compressed_tree():
    tree = W.tree_with_zero_weights(5, seed=20)
    S0, J = oracle.jump_fields(tree)
    assert J % 3 == 0 and 0 < J < 3 * 31 and (S0 - J) % 6 == 0
    its = _path(tree, 12, 10, seed=21)
    assert its[1, 3:].mean() < its[0, 3:].mean(), its


def test_failed_extrapolation_restarts_from_the_stored_jumps():
    K, n, n_inc = 6, 64, 12
    tree = W.tree_d10_fit(K, seed=140)
    A2, lam, Q = W.orientation_field(n, seed=141)
    amp = W.random6_path_final(n, 0.02, seed=142)
    S0, J = oracle.jump_fields(tree)
    sp = np.zeros((S0 + J + 6, n))
    restarts = 0
    for s in range(1, n_inc + 1):
        En, dE = W.cyclic_increment(amp, s, n_inc)
        # the paper's start from the same state, for comparison
        st_0, sig_0, _, it_0, stat_0, _ = oracle.update(tree, lam, Q, En, dE, sp[:S0])
        sp_new, sig_p, _, it_p, stat_p, _ = oracle.update(tree, lam, Q, En, dE, sp, predictor=True)
        prev = sp[S0 + J:].T
        den = np.einsum("ni,ni->n", prev, prev)
        rho = np.where(den > 0, np.clip(np.einsum("ni,ni->n", dE, prev) / np.where(den > 0, den, 1.0), 0, 1), 0)
        # rho = 0: the paper's start itself
        z = rho == 0
        np.testing.assert_array_equal(it_p[z], it_0[z])
        np.testing.assert_array_equal(sig_p[z], sig_0[z])
        r = (rho > 0) & (it_p > oracle.PRED_TRIES)
        restarts += int(r.sum())
        # a restarted point repeats the paper start's iterates after its failed attempt
        np.testing.assert_array_equal(it_p[r], it_0[r] + oracle.PRED_TRIES)
        np.testing.assert_array_equal(stat_p[r], stat_0[r])
        np.testing.assert_array_equal(sig_p[r], sig_0[r])
        np.testing.assert_array_equal(sp_new[:S0][:, r], st_0[:, r])
        sp = sp_new
    assert restarts > 0

