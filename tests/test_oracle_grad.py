"""Pin of the oracle's implicit-function gradient: it must equal central finite
differences (h = 1e-6) of the oracle's full Newton solve, along random
parameter directions, for elastic and plastic states."""
import numpy as np
import pytest

import oracle
from paper_2103_08253_gb300 import workloads as W


@pytest.mark.parametrize("K,steps", [(2, 1), (3, 6), (4, 8)])
def test_ift_gradient_matches_finite_differences_of_the_solve(K, steps):
    n = 2
    tree = W.tree_d10_fit(K, seed=20 + K)
    A2, lam, Q = W.orientation_field(n, seed=30 + K)
    Ef = W.random6_path_final(n, 0.03, seed=40 + K)
    S = oracle.state_size(K, tree.phases)
    st = np.zeros((S, n))
    st_prev = st
    for s in range(1, steps + 1):
        En, dE = W.proportional_increment(Ef, s, 10)
        st_prev = st
        st = oracle.update(tree, lam, Q, En, dE, st)[0]
    rng = np.random.default_rng(K)
    for i in range(n):
        g = rng.standard_normal(6)
        dirs = [(rng.standard_normal(tree.p.shape), rng.standard_normal(tree.q.shape),
                 rng.standard_normal(tree.w.shape) * tree.w) for _ in range(2)]
        full = oracle.gradient_ift(tree, lam[i], Q[i], (En + dE)[i], oracle.jumps(tree, st, i),
                                   oracle.leaf_states(tree, st_prev, i), g)
        direc = oracle.gradient_ift(tree, lam[i], Q[i], (En + dE)[i], oracle.jumps(tree, st, i),
                                    oracle.leaf_states(tree, st_prev, i), g, directions=dirs)
        for (dp, dq, dw), dval in zip(dirs, direc):
            pred = (full["p"] * dp).sum() + (full["q"] * dq).sum() + (full["w"] * dw).sum()

            def f(sc):
                t2 = oracle._with_params(tree, tree.p + sc * dp, tree.q + sc * dq, tree.w + sc * dw)
                return g @ oracle.update(t2, lam[i:i + 1], Q[i:i + 1], En[i:i + 1], dE[i:i + 1],
                                         st_prev[:, i:i + 1])[1][0]
            h = 1e-6
            fd = (f(h) - f(-h)) / (2 * h)
            assert abs(pred - fd) <= 1e-6 * abs(fd) + 1e-9
            assert abs(dval - pred) <= 1e-7 * abs(pred) + 1e-9
