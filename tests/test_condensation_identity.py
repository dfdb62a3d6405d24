"""The tree condensation that the CUDA kernels use is the paper's Newton step.

The paper solves J da = -R with J = A^T W D A, R = A^T W sigma (Sec. 3.2) by a
sparse Cholesky factorisation (Sec. 4.6).  The kernels instead eliminate the
laminates leaf to root: given the affine responses s + C d_eps of its two
children, a laminate with normal n, volume fractions c1, c2 and N = sym(. (x) n)
forms

    Kn = N^T (c2 C_L + c1 C_R) N,   B = (C_R - C_L) N,
    g = -Kn^-1 N^T (s_R - s_L),     H = -Kn^-1 B^T,
    s = c1 s_L + c2 s_R + c1 c2 B g,   C = c1 C_L + c2 C_R + c1 c2 B H,

and then, root to leaves from d_eps = 0 at the root, da = g + H d_eps with
d_eps_L = d_eps - c2 N da, d_eps_R = d_eps + c1 N da.

This test restates that recursion in numpy, independent of the CUDA code, and
checks on the oracle's leaf stresses and tangents at random iterates that
  * da equals the oracle's Cholesky step -J^-1 R;
  * the root's C equals the homogenised tangent of the linearised problem,
    sum_l w_l D_l (I + A_l X) with X = -J^-1 A^T W D [I ... I];
  * the root's s equals the linearised average stress after the step,
    sum_l w_l (sigma_l + D_l A_l da).
"""
import numpy as np
import pytest

import oracle
from paper_2103_08253_gb300 import workloads as W

R2 = np.sqrt(2.0)


def sym_operator(n):
    """6x3: column m is the Mandel vector of sym(e_m (x) n)."""
    N = np.zeros((6, 3))
    for m in range(3):
        T = np.zeros((3, 3))
        T[m, :] += 0.5 * n
        T[:, m] += 0.5 * n
        N[:, m] = [T[0, 0], T[1, 1], T[2, 2], R2 * T[1, 2], R2 * T[0, 2], R2 * T[0, 1]]
    return N


def condense_and_step(K, w, nrm, sig, D):
    """Newton step of the whole tree by condensation: (da [3N], root s, root C)."""
    L = 1 << K
    node = lambda k, i: L - (1 << k) + (i - 1)          # paper ordering: level K first, root last

    def weight(k, i):                                    # level K + 1 = the leaves
        span = 1 << (K + 1 - k)
        return w[(i - 1) * span:i * span].sum()

    stash = {}

    def up(k, i):
        if k == K + 1:
            return sig[i - 1], D[i - 1]
        sL, CL = up(k + 1, 2 * i - 1)
        sR, CR = up(k + 1, 2 * i)
        WL, WR = weight(k + 1, 2 * i - 1), weight(k + 1, 2 * i)
        c1, c2 = WL / (WL + WR), WR / (WL + WR)
        N = sym_operator(nrm[node(k, i)])
        Kn = N.T @ (c2 * CL + c1 * CR) @ N
        B = (CR - CL) @ N
        g = -np.linalg.solve(Kn, N.T @ (sR - sL))
        H = -np.linalg.solve(Kn, B.T)
        stash[(k, i)] = (g, H, c1, c2, N)
        return c1 * sL + c2 * sR + c1 * c2 * B @ g, c1 * CL + c2 * CR + c1 * c2 * B @ H

    s_root, C_root = up(1, 1)
    da = np.zeros(3 * (L - 1))

    def down(k, i, deps):
        if k == K + 1:
            return
        g, H, c1, c2, N = stash[(k, i)]
        d = g + H @ deps
        da[3 * node(k, i):3 * node(k, i) + 3] = d
        down(k + 1, 2 * i - 1, deps - c2 * N @ d)
        down(k + 1, 2 * i, deps + c1 * N @ d)

    down(1, 1, np.zeros(6))
    return da, s_root, C_root


def random_iterate(tree, rng, plastic_history):
    L = 1 << tree.K
    E = rng.standard_normal(6)
    E *= 0.02 / np.linalg.norm(E)
    a = 1e-3 * rng.standard_normal(3 * (L - 1))
    z = np.zeros((L, 7))
    if plastic_history:
        for l in range(L):
            if tree.phases[l % 2].kind != 0:
                ep = rng.standard_normal(6) * 3e-3
                ep[2] = -ep[0] - ep[1]                   # deviatoric: ep33 = -ep11 - ep22
                z[l] = [abs(rng.normal(0.0, 0.01))] + list(ep)
    return E, a, z


@pytest.mark.parametrize("K,M,history", [(3, 3, False), (4, 3, True), (6, 4, True), (5, 6, False)])
def test_condensation_is_the_newton_step(K, M, history):
    rng = np.random.default_rng(100 + K + M)
    tree = (W.tree_d10_fit(K, seed=K) if M == 3 else W.tree_nodal_angles(K, M, seed=K))
    A2, lam, Q = W.orientation_field(4, seed=K + 1)
    w = np.asarray(tree.w, dtype=np.float64) / np.sum(tree.w)
    L = 1 << K
    for pt in range(4):
        E, a, z = random_iterate(tree, rng, history)
        ns = oracle.newton_system(tree, lam[pt, 0], lam[pt, 1], E, a, z)
        assert ns["rc"] == 0
        D = np.array([oracle.phase_law(tree.phases[l % 2], ns["eps"][l], z[l])[1] for l in range(L)])
        nrm = oracle.normals(tree, lam[pt, 0], lam[pt, 1])
        da, s_root, C_root = condense_and_step(K, w, nrm, ns["sig"], D)
        assert np.abs(da - ns["da"]).max() <= 1e-9 * np.abs(ns["da"]).max(), (K, pt)
        # the linearised problem through the oracle's assembled operators
        A = oracle.gradient_operator(tree, lam[pt, 0], lam[pt, 1])
        WD = np.zeros((6 * L, 6 * L))
        for l in range(L):
            WD[6 * l:6 * l + 6, 6 * l:6 * l + 6] = w[l] * D[l]
        ones = np.tile(np.eye(6), (L, 1))                # [I ... I]^T
        X = -np.linalg.solve(ns["J"], A.T @ WD @ ones)
        C_lin = ones.T @ WD @ (ones + A @ X)
        np.testing.assert_allclose(C_root, C_lin, rtol=0, atol=1e-9 * np.abs(C_lin).max())
        s_lin = sum(w[l] * (ns["sig"][l] + D[l] @ (A[6 * l:6 * l + 6] @ ns["da"])) for l in range(L))
        np.testing.assert_allclose(s_root, s_lin, rtol=0, atol=1e-9 * np.abs(s_lin).max())
        # and the plain average of the leaf stresses is the oracle's sigma_bar
        np.testing.assert_allclose(w @ ns["sig"], ns["sbar"], rtol=0, atol=1e-12 * np.abs(ns["sbar"]).max())


def test_identities_of_the_bottom_laminate():
    """For a unit normal n: N^T 1 = n and N^T N = (I + n (x) n) / 2, the identities that shorten the
    condensation of two leaves whose tangents have the form lam 1(x)1 + 2 mu I - c m(x)m."""
    rng = np.random.default_rng(5)
    one = np.array([1.0, 1.0, 1.0, 0.0, 0.0, 0.0])
    for _ in range(20):
        n = rng.standard_normal(3)
        n /= np.linalg.norm(n)
        N = sym_operator(n)
        np.testing.assert_allclose(N.T @ one, n, atol=1e-15)
        np.testing.assert_allclose(N.T @ N, 0.5 * (np.eye(3) + np.outer(n, n)), atol=1e-15)


def test_leaf_tangent_has_the_isotropic_rank_one_form():
    """The leaf tangent is lam 1(x)1 + 2 mu I - c m(x)m with m the unit flow direction (Mandel, deviatoric):
    for J2 leaves lam + 2 mu / 3 = K, mu < G and c > 0 once they yield; elastic leaves have mu = G, c = 0.
    With m deviatoric and of unit length, m^T D m = 2 mu - c and 1^T D 1 = 9 lam + 6 mu."""
    rng = np.random.default_rng(6)
    one = np.array([1.0, 1.0, 1.0, 0.0, 0.0, 0.0])
    for ph in (W.MATRIX, W.MATRIX_EXPLIN, W.FIBER):
        Kb, G = ph.E / (3 * (1 - 2 * ph.nu)), ph.E / (2 * (1 + ph.nu))
        for _ in range(10):
            eps = rng.standard_normal(6) * 0.02
            sig, D, z = oracle.phase_law(ph, eps)
            dev = eps - np.r_[np.full(3, eps[:3].sum() / 3), np.zeros(3)]
            m = dev / np.linalg.norm(dev)                # the flow direction from the virgin state
            e = np.linalg.svd(np.vstack([one, m]))[2][2]  # a unit direction orthogonal to 1 and m
            mu = 0.5 * (e @ D @ e)
            c = 2 * mu - m @ D @ m
            lam = (one @ D @ one - 6 * mu) / 9.0
            rebuilt = lam * np.outer(one, one) + 2 * mu * np.eye(6) - c * np.outer(m, m)
            np.testing.assert_allclose(D, rebuilt, atol=1e-9 * np.abs(D).max())
            assert abs(lam + 2 * mu / 3 - Kb) <= 1e-9 * Kb
            if ph.kind == 0:
                assert abs(mu - G) <= 1e-9 * G and abs(c) <= 1e-9 * G
            else:
                assert z[0] > 0 and c > 0 and mu < G     # yielded
