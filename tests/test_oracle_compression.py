"""Tree compression in the oracle (Sec. 3.1: leaves of weight zero are removed
and laminates with one weightless subtree pass the other through), pinned by
what it must reduce to: a smaller perfect tree, the limit of vanishing
weights, and the phase law for a single remaining leaf."""
import numpy as np

import oracle
from paper_2103_08253_gb300 import workloads as W


def run(tree, lam, Q, Ef, steps, n_steps):
    S = oracle.state_size(tree.K, tree.phases, tree.w)
    st = np.zeros((S, lam.shape[0]))
    for s in range(1, steps + 1):
        En, dE = W.proportional_increment(Ef, s, n_steps)
        st, sig, C, it, stat, gap = oracle.update(tree, lam, Q, En, dE, st)
    return st, sig, C, it, stat


def paper_index(K, k, i):
    return (1 << K) - (1 << k) + i - 1


def test_weightless_right_subtree_equals_the_left_subtree_tree():
    """Zero weight on the root's right half: the root passes its left subtree through, so
    the depth-K tree is the depth-(K-1) tree of that subtree (same normals, same weights)."""
    K = 4
    big = W.tree_d10_fit(K, seed=3)
    w = big.w.copy()
    w[8:] = 0.0
    big = W.TreeParams(K, big.M, big.p, big.q, w, big.phases)
    rows = [paper_index(K, k, i) for k in range(K, 1, -1) for i in range(1, (1 << (k - 2)) + 1)]
    small = W.TreeParams(K - 1, big.M, big.p[rows], big.q[rows], w[:8], big.phases)
    assert oracle.state_size(K, big.phases, big.w) == oracle.state_size(K - 1, small.phases)
    A2, lam, Q = W.orientation_field(6, seed=4)
    Ef = W.random6_path_final(6, 0.03, seed=5)
    a = run(big, lam, Q, Ef, 5, 10)
    b = run(small, lam, Q, Ef, 5, 10)
    assert (a[4] == 0).all() and (b[4] == 0).all()
    np.testing.assert_allclose(a[1], b[1], rtol=0, atol=1e-12 * np.abs(b[1]).max())
    np.testing.assert_allclose(a[2], b[2], rtol=0, atol=1e-12 * np.abs(b[2]).max())
    np.testing.assert_allclose(a[0], b[0], rtol=0, atol=1e-12 * np.abs(b[0]).max())
    np.testing.assert_array_equal(a[3], b[3])


def test_vanishing_weights_converge_to_the_compressed_tree():
    """Weights eps -> 0 on the leaves that compression removes: the stress approaches the
    compressed tree's linearly in eps."""
    t0 = W.tree_with_zero_weights(5, seed=6)
    dead = t0.w == 0
    A2, lam, Q = W.orientation_field(4, seed=7)
    Ef = W.random6_path_final(4, 0.02, seed=8)
    ref = run(t0, lam, Q, Ef, 3, 6)
    errs = []
    for eps in (1e-7, 1e-8):
        w = t0.w.copy()
        w[dead] = eps
        te = W.TreeParams(t0.K, t0.M, t0.p, t0.q, w, t0.phases)
        r = run(te, lam, Q, Ef, 3, 6)
        assert (r[4] == 0).all()
        errs.append(np.abs(r[1] - ref[1]).max() / np.abs(ref[1]).max())
    assert errs[1] < 1e-4 and errs[1] < 0.3 * errs[0]


def test_single_remaining_leaf_is_the_phase_law():
    K = 3
    t = W.tree_d10_fit(K, seed=9)
    w = np.zeros(1 << K)
    w[5] = 0.7                                   # leaf 6: even, the J2 matrix
    t = W.TreeParams(K, t.M, t.p, t.q, w, t.phases)
    assert oracle.state_size(K, t.phases, t.w) == 6
    lam, Q = W.identity_orientation(3)
    Ef = W.random6_path_final(3, 0.03, seed=10)
    st, sig, C, it, stat = run(t, lam, Q, Ef, 4, 4)
    for i in range(3):
        z = np.zeros(7)
        for s in range(1, 5):
            En, dE = W.proportional_increment(Ef[i:i + 1], s, 4)
            s1, D1, z = oracle.phase_law(W.MATRIX, (En + dE)[0], z)
        np.testing.assert_allclose(sig[i], s1, rtol=0, atol=1e-12 * np.abs(s1).max())
        np.testing.assert_allclose(C[i], D1, rtol=0, atol=1e-10 * np.abs(D1).max())
    assert (it == 0).all()


def test_compressed_state_size_counts_remaining_leaves_and_laminates():
    t = W.tree_with_zero_weights(8, seed=11)
    alive = t.w > 0
    Wh = np.zeros(512)                           # heap subtree weights, 1-based
    Wh[256:] = t.w
    for k in range(255, 0, -1):
        Wh[k] = Wh[2 * k] + Wh[2 * k + 1]
    active = sum(1 for k in range(1, 256) if Wh[2 * k] > 0 and Wh[2 * k + 1] > 0)
    n_inel = int(alive[1::2].sum())              # even leaves: the matrix
    assert active == alive.sum() - 1             # a full binary tree
    assert oracle.state_size(8, t.phases, t.w) == 6 * n_inel + 3 * active
