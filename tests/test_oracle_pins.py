"""Pins of the CPU oracle against what the paper and the mathematics fix.

Each test checks the oracle against something other than itself:

* the depth-3 gradient operator printed in the paper (golden fixture);
* Milton's laminate formula with the projection P(n) and a free shift alpha
  (Sec. 3.1, Eq. of the linear laminate homogenisation), for one laminate and
  recursively for whole trees (the linear DMN of Sec. 3.1), for several alpha;
* identical phases, Voigt/Reuss bounds, symmetry (consequences of that formula);
* the J2 law against the bilinear equivalent-stress/strain closed form of
  proportional loading, its invariants and finite differences;
* the Hill-Mandel identity, the strain average, the converged residual;
* the Cholesky step against numpy's dense solve, J against A^T W D A built
  here from the dense A, and the algorithmic tangent against finite
  differences of the effective stress;
* the orientation steps against their defining properties and numpy.eigh.
"""
import os

import math

import numpy as np
import pytest

import oracle
from paper_2103_08253_gb300 import workloads as W

HERE = os.path.dirname(os.path.abspath(__file__))
R2 = np.sqrt(2.0)
MI = [(0, 0), (1, 1), (2, 2), (1, 2), (0, 2), (0, 1)]
ONE = np.array([1.0, 1.0, 1.0, 0.0, 0.0, 0.0])


def wI(I):
    return 1.0 if I < 3 else R2


def iso(E, nu):
    K = E / (3 * (1 - 2 * nu))
    G = E / (2 * (1 + nu))
    return K * np.outer(ONE, ONE) + 2 * G * (np.eye(6) - np.outer(ONE, ONE) / 3)


def P_mandel(n):
    """Projection P(n) from its index formula (Sec. 3.1) in Mandel form."""
    d = np.eye(3)
    P4 = (0.5 * (np.einsum("m,no,p->mnop", n, d, n) + np.einsum("n,mo,p->mnop", n, d, n)
                 + np.einsum("m,np,o->mnop", n, d, n) + np.einsum("n,mp,o->mnop", n, d, n))
          - np.einsum("m,n,o,p->mnop", n, n, n, n))
    return np.array([[P4[MI[I][0], MI[I][1], MI[J][0], MI[J][1]] * wI(I) * wI(J) for J in range(6)]
                     for I in range(6)])


def laminate_alpha(C1, C2, c1, n, al):
    """Solve (P + al [C - al I]^-1)^-1 = c1 (P + al [C1 - al I]^-1)^-1 + c2 (...)^-1 for C."""
    I6 = np.eye(6)
    P = P_mandel(n)
    Y = (c1 * np.linalg.inv(P + al * np.linalg.inv(C1 - al * I6))
         + (1 - c1) * np.linalg.inv(P + al * np.linalg.inv(C2 - al * I6)))
    return al * I6 + al * np.linalg.inv(np.linalg.inv(Y) - P)


def linear_dmn_alpha(tree, C_phase, nrm, al):
    """Linear DMN by propagating stiffnesses level by level (Sec. 3.1, Fig. of the
    stiffness propagation): laminate (k, i) homogenises children 2i-1, 2i."""
    K = tree.K
    w = tree.w / tree.w.sum()
    C = [C_phase[l % 2] for l in range(1 << K)]
    Wt = list(w)
    for k in range(K, 0, -1):
        off = (1 << K) - (1 << k)
        Cn, Wn = [], []
        for i in range(1 << (k - 1)):
            wl, wr = Wt[2 * i], Wt[2 * i + 1]
            Cn.append(laminate_alpha(C[2 * i], C[2 * i + 1], wl / (wl + wr), nrm[off + i], al))
            Wn.append(wl + wr)
        C, Wt = Cn, Wn
    return C[0]


def mandel_to_T(v):
    return np.array([[v[0], v[5] / R2, v[4] / R2], [v[5] / R2, v[1], v[3] / R2], [v[4] / R2, v[3] / R2, v[2]]])


def T_to_mandel(T):
    return np.array([T[0, 0], T[1, 1], T[2, 2], R2 * T[1, 2], R2 * T[0, 2], R2 * T[0, 1]])


def sym_block(n):
    """6x3 block of a -> sym(a (x) n) built from tensors."""
    B = np.zeros((6, 3))
    for m in range(3):
        a = np.zeros(3)
        a[m] = 1.0
        B[:, m] = T_to_mandel(0.5 * (np.outer(a, n) + np.outer(n, a)))
    return B


ELASTIC_MATRIX = W.Phase(0, 3000.0, 0.35)
C_FIB = iso(72000.0, 0.22)
C_MAT = iso(3000.0, 0.35)


def run_path(tree, lam, Q, E_final, n_steps, upto=None, **kw):
    n = lam.shape[0]
    S = oracle.state_size(tree.K, tree.phases)
    st = np.zeros((S, n))
    out = None
    for s in range(1, (upto or n_steps) + 1):
        En, dE = W.proportional_increment(E_final, s, n_steps)
        out = oracle.update(tree, lam, Q, En, dE, st, **kw)
        st = out[0]
    return out


# ----------------------------------------------------------------------------- operator A


def test_gradient_operator_matches_printed_depth3_example():
    tree = W.tree_constant_normals(3, seed=11)
    lam1, lam2 = 0.6, 0.3
    A = oracle.gradient_operator(tree, lam1, lam2)
    nrm = oracle.normals(tree, lam1, lam2)
    w = tree.w / tree.w.sum()
    # subtree weights per level k (k = 4 are the leaves)
    Wl = {4: list(w)}
    for k in (3, 2, 1):
        Wl[k] = [Wl[k + 1][2 * i] + Wl[k + 1][2 * i + 1] for i in range(1 << (k - 1))]

    def c(m, k):  # fraction of child m (level k+1) inside its level-k laminate
        i = (m + 1) // 2
        return Wl[k + 1][m - 1] / (Wl[k + 1][2 * i - 2] + Wl[k + 1][2 * i - 1])

    def col(i, k):  # paper ordering of laminate (k, i) for K = 3
        return (8 - (1 << k)) + (i - 1)

    rows = [ln.split() for ln in open(os.path.join(HERE, "golden", "gradient_operator_K3.txt"))
            if ln.strip() and not ln.startswith("#")]
    assert len(rows) == 8 and all(len(r) == 7 for r in rows)
    for r, toks in enumerate(rows):
        for cidx, tok in enumerate(toks):
            blk = A[6 * r:6 * r + 6, 3 * cidx:3 * cidx + 3]
            if tok == "0":
                assert np.all(blk == 0.0)
                continue
            sgn = -1.0 if tok[0] == "-" else 1.0
            cpart, npart = tok[2:].split("N")
            m, k = (int(x) for x in cpart.split("_"))
            i, k2 = (int(x) for x in npart.split("_"))
            assert k == k2 and col(i, k) == cidx
            expect = sgn * c(m, k) * sym_block(nrm[col(i, k)])
            np.testing.assert_allclose(blk, expect, rtol=0, atol=1e-15)
    # a column of A sums (with weights) to zero: every laminate keeps the average strain
    np.testing.assert_allclose((w[:, None, None] * A.reshape(8, 6, 21)).sum(axis=0), 0.0, atol=1e-15)


# ----------------------------------------------------------------------------- laminates


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_one_laminate_matches_milton_alpha_formula(seed):
    tree = W.tree_constant_normals(1, seed=seed, phases=(W.FIBER, ELASTIC_MATRIX))
    lam, Q = W.identity_orientation(1)
    E = np.random.default_rng(seed).standard_normal((1, 6)) * 1e-3
    S = oracle.state_size(1, tree.phases)
    _, sig, C, it, stat, _ = oracle.update(tree, lam, Q, np.zeros((1, 6)), E, np.zeros((S, 1)))
    assert stat[0] == 0
    nrm = oracle.normals(tree, 1 / 3, 1 / 3)[0]
    w = tree.w / tree.w.sum()
    for al in (2e5, 5e5, 1e3, -1e3):      # large or small shift: the result does not depend on it
        Cl = laminate_alpha(C_FIB, C_MAT, w[0], nrm, al)
        np.testing.assert_allclose(C[0], Cl, rtol=0, atol=1e-12 * np.abs(Cl).max())
    np.testing.assert_allclose(sig[0], C[0] @ E[0], rtol=0, atol=1e-10 * np.abs(sig).max())


@pytest.mark.parametrize("K,seed", [(2, 4), (3, 5), (5, 6)])
def test_linear_dmn_matches_recursive_laminate_formula(K, seed):
    tree = W.tree_d10_fit(K, seed=seed, phases=(W.FIBER, ELASTIC_MATRIX))
    A2, lam, Q = W.orientation_field(3, seed=seed + 100)
    E = np.random.default_rng(seed).standard_normal((3, 6)) * 1e-3
    S = oracle.state_size(K, tree.phases)
    _, sig, C, it, stat, _ = oracle.update(tree, lam, Q, np.zeros((3, 6)), E, np.zeros((S, 3)))
    assert np.all(stat == 0)
    for i in range(3):
        nrm = oracle.normals(tree, *lam[i])
        for al in (3e5, -500.0):
            Cl = linear_dmn_alpha(tree, (C_FIB, C_MAT), nrm, al)
            Cg, _ = oracle.rotate(Q[i].reshape(3, 3), Cl, np.zeros(6))
            np.testing.assert_allclose(C[i], Cg, rtol=0, atol=1e-11 * np.abs(Cg).max())
        np.testing.assert_allclose(sig[i], C[i] @ E[i], rtol=0, atol=1e-10 * np.abs(sig[i]).max())


def test_identical_elastic_phases_return_the_phase_law():
    ph = W.Phase(0, 5000.0, 0.3)
    tree = W.tree_d10_fit(4, seed=7, phases=(ph, ph))
    A2, lam, Q = W.orientation_field(4, seed=8)
    E = np.random.default_rng(9).standard_normal((4, 6)) * 1e-3
    S = oracle.state_size(4, tree.phases)
    st, sig, C, it, stat, _ = oracle.update(tree, lam, Q, np.zeros((4, 6)), E, np.zeros((S, 4)))
    Ci = iso(5000.0, 0.3)
    np.testing.assert_allclose(C, np.broadcast_to(Ci, C.shape), atol=1e-12 * 5000)
    np.testing.assert_allclose(sig, E @ Ci.T, atol=1e-12 * np.abs(sig).max())
    assert np.abs(st).max() < 1e-14       # no jumps open


def test_identical_j2_phases_return_the_phase_law():
    ph = W.MATRIX
    tree = W.tree_d10_fit(3, seed=12, phases=(ph, ph))
    A2, lam, Q = W.orientation_field(5, seed=13)
    Ef = W.random6_path_final(5, 0.03, seed=14)
    st, sig, C, it, stat, _ = run_path(tree, lam, Q, Ef, 6)
    assert np.all(stat == 0)
    S = st.shape[0]
    for i in range(5):
        z = np.zeros(7)
        for s in range(1, 7):                  # the same path through the single-phase law
            En, dE = W.proportional_increment(Ef[i:i + 1], s, 6)
            s1, D1, z = oracle.phase_law(ph, (En + dE)[0], z)
        np.testing.assert_allclose(sig[i], s1, atol=1e-10 * np.abs(s1).max())
        np.testing.assert_allclose(C[i], D1, atol=1e-10 * np.abs(D1).max())
    assert np.abs(st[S - 3 * 7:]).max() < 1e-12


def test_voigt_reuss_bounds_and_symmetry():
    tree = W.tree_d10_fit(4, seed=21, phases=(W.FIBER, ELASTIC_MATRIX))
    A2, lam, Q = W.orientation_field(8, seed=22)
    S = oracle.state_size(4, tree.phases)
    _, _, C, _, stat, _ = oracle.update(tree, lam, Q, np.zeros((8, 6)), np.full((8, 6), 1e-4), np.zeros((S, 8)))
    w = tree.w / tree.w.sum()
    wf, wm = w[0::2].sum(), w[1::2].sum()
    CV = wf * C_FIB + wm * C_MAT
    CR = np.linalg.inv(wf * np.linalg.inv(C_FIB) + wm * np.linalg.inv(C_MAT))
    for i in range(8):
        assert np.abs(C[i] - C[i].T).max() < 1e-12 * np.abs(C[i]).max()
        Cs = 0.5 * (C[i] + C[i].T)
        assert np.linalg.eigvalsh(CV - Cs).min() > -1e-9 * 72000
        assert np.linalg.eigvalsh(Cs - CR).min() > -1e-9 * 72000


# ----------------------------------------------------------------------------- J2 leaf


def j2_closed_form(ph, eps):
    """Bilinear equivalent-stress/strain response of proportional loading with
    linear isotropic hardening: sigma_eq = 3G e_eq (elastic),
    sigma_eq = 3G (sigma0 + H e_eq) / (3G + H) (plastic), stress deviator along
    the strain deviator; alpha_bar = (sigma_eq - sigma0) / H."""
    K = ph.E / (3 * (1 - 2 * ph.nu))
    G = ph.E / (2 * (1 + ph.nu))
    tr = eps[:3].sum()
    dev = eps - tr / 3 * ONE
    e_eq = np.sqrt(2.0 / 3.0) * np.linalg.norm(dev)
    s_eq = 3 * G * e_eq
    ab = 0.0
    if s_eq > ph.sigma0:
        s_eq = 3 * G * (ph.sigma0 + ph.H * e_eq) / (3 * G + ph.H)
        ab = (s_eq - ph.sigma0) / ph.H
    s = np.sqrt(2.0 / 3.0) * s_eq * dev / np.linalg.norm(dev)
    return K * tr * ONE + s, ab


@pytest.mark.parametrize("seed", range(4))
def test_j2_matches_closed_form_under_proportional_loading(seed):
    rng = np.random.default_rng(seed)
    d = rng.standard_normal(6)
    d /= np.linalg.norm(d)
    ph = W.MATRIX
    z = np.zeros(7)
    for s in range(1, 31):                      # 30 increments to |eps| = 4e-2
        eps = 4e-2 * s / 30 * d
        sig, D, z = oracle.phase_law(ph, eps, z)
        ref, ab = j2_closed_form(ph, eps)
        np.testing.assert_allclose(sig, ref, rtol=0, atol=1e-11 * max(1.0, np.abs(ref).max()))
        assert abs(z[0] - ab) < 1e-13
        # invariants: plastic strain deviatoric, consistency on the yield surface
        assert abs(z[1] + z[2] + z[3]) < 1e-15
        G = ph.E / (2 * (1 + ph.nu))
        sdev = sig - sig[:3].sum() / 3 * ONE
        if z[0] > 0:
            assert abs(np.linalg.norm(sdev) - np.sqrt(2 / 3) * (ph.sigma0 + ph.H * z[0])) < 1e-10
            # elastic law holds on the elastic part of the strain
            np.testing.assert_allclose(sdev, 2 * G * (eps - eps[:3].sum() / 3 * ONE - z[1:]), atol=1e-10)


# ----------------------------------------------------------------------------- J2, exponential-linear hardening


def explin_yield(ph, ab):
    """sigma_Y of the exponential-linear law (Sec. 4.1), written out."""
    return ph.sigma0 + ph.H * ab + (ph.sigma_inf - ph.sigma0) * (
        1.0 - math.exp(-(ph.k0 - ph.H) / (ph.sigma_inf - ph.sigma0) * ab))


def test_explin_law_with_k0_equal_kinf_is_the_linear_law():
    """k0 = k_inf removes the exponential term: the law is the linear-hardening one."""
    rng = np.random.default_rng(31)
    lin = W.MATRIX
    ex = W.Phase(kind=2, E=lin.E, nu=lin.nu, sigma0=lin.sigma0, H=lin.H, sigma_inf=2 * lin.sigma0, k0=lin.H)
    z1 = np.zeros(7)
    z2 = np.zeros(7)
    for s in range(1, 6):
        eps = 0.01 * s * rng.standard_normal(6)
        s1, D1, z1 = oracle.phase_law(lin, eps, z1)
        s2, D2, z2 = oracle.phase_law(ex, eps, z2)
        np.testing.assert_allclose(s2, s1, rtol=0, atol=1e-12 * np.abs(s1).max())
        np.testing.assert_allclose(D2, D1, rtol=0, atol=1e-12 * np.abs(D1).max())
        np.testing.assert_allclose(z2, z1, rtol=0, atol=1e-15)


@pytest.mark.parametrize("seed", range(3))
def test_explin_radial_return_against_bisection_and_path_independence(seed):
    """Proportional deviatoric loading from the virgin state: the stress deviator
    stays along the strain deviator d and |s| = 2G (|e| - dg), with dg the root of
    2G (|e| - dg) = sqrt(2/3) sigma_Y(sqrt(2/3) dg), found here by bisection.
    Radial return is exact for proportional loading, so 1 and 25 increments agree."""
    rng = np.random.default_rng(40 + seed)
    ph = W.MATRIX_EXPLIN
    G = ph.E / (2 * (1 + ph.nu))
    d = rng.standard_normal(6)
    d[:3] -= d[:3].sum() / 3
    d /= np.linalg.norm(d)
    for e in (0.005, 0.02, 0.08):
        lo, hi = 0.0, e
        for _ in range(200):
            mid = 0.5 * (lo + hi)
            if 2 * G * (e - mid) - math.sqrt(2 / 3) * explin_yield(ph, math.sqrt(2 / 3) * mid) > 0:
                lo = mid
            else:
                hi = mid
        dg = 0.5 * (lo + hi)
        sig1, _, z1 = oracle.phase_law(ph, e * d, np.zeros(7))
        np.testing.assert_allclose(sig1, 2 * G * (e - dg) * d, rtol=0, atol=1e-11 * 2 * G * e)
        assert abs(z1[0] - math.sqrt(2 / 3) * dg) < 1e-14
        z = np.zeros(7)
        for s in range(1, 26):
            sig, _, z = oracle.phase_law(ph, e * s / 25 * d, z)
        np.testing.assert_allclose(sig, sig1, rtol=0, atol=1e-11 * 2 * G * e)
        np.testing.assert_allclose(z, z1, rtol=0, atol=1e-14)


@pytest.mark.parametrize("plastic", [False, True])
def test_explin_tangent_matches_finite_differences(plastic):
    """The consistent tangent takes the hardening slope at the new alpha_bar."""
    rng = np.random.default_rng(15 + plastic)
    ph = W.MATRIX_EXPLIN
    z_n = np.zeros(7)
    if plastic:
        for s in range(1, 5):
            _, _, z_n = oracle.phase_law(ph, 0.01 * s * rng.standard_normal(6), z_n)
        assert z_n[0] > 0.002
    eps = z_n[1:] + (0.02 if plastic else 0.001) * rng.standard_normal(6)
    sig, D, _ = oracle.phase_law(ph, eps, z_n)
    h = 1e-7
    Dfd = np.zeros((6, 6))
    for j in range(6):
        e = np.zeros(6)
        e[j] = h
        Dfd[:, j] = (oracle.phase_law(ph, eps + e, z_n)[0] - oracle.phase_law(ph, eps - e, z_n)[0]) / (2 * h)
    np.testing.assert_allclose(D, Dfd, rtol=0, atol=1e-6 * np.abs(D).max())


def test_identical_explin_phases_return_the_phase_law():
    ph = W.MATRIX_EXPLIN
    tree = W.tree_d10_fit(3, seed=32, phases=(ph, ph))
    A2, lam, Q = W.orientation_field(4, seed=33)
    Ef = W.random6_path_final(4, 0.03, seed=34)
    st, sig, C, it, stat, _ = run_path(tree, lam, Q, Ef, 6)
    assert np.all(stat == 0)
    for i in range(4):
        z = np.zeros(7)
        for s in range(1, 7):
            En, dE = W.proportional_increment(Ef[i:i + 1], s, 6)
            s1, D1, z = oracle.phase_law(ph, (En + dE)[0], z)
        np.testing.assert_allclose(sig[i], s1, atol=1e-10 * np.abs(s1).max())
        np.testing.assert_allclose(C[i], D1, atol=1e-10 * np.abs(D1).max())


@pytest.mark.parametrize("plastic", [False, True])
def test_j2_tangent_matches_finite_differences(plastic):
    rng = np.random.default_rng(5 + plastic)
    ph = W.MATRIX
    z_n = np.zeros(7)
    if plastic:   # a non-proportional history
        for s in range(1, 5):
            _, _, z_n = oracle.phase_law(ph, 0.01 * s * rng.standard_normal(6), z_n)
    eps = z_n[1:] + (0.02 if plastic else 0.002) * rng.standard_normal(6)
    sig, D, _ = oracle.phase_law(ph, eps, z_n)
    h = 1e-7
    Dfd = np.zeros((6, 6))
    for j in range(6):
        e = np.zeros(6)
        e[j] = h
        Dfd[:, j] = (oracle.phase_law(ph, eps + e, z_n)[0] - oracle.phase_law(ph, eps - e, z_n)[0]) / (2 * h)
    np.testing.assert_allclose(D, Dfd, rtol=0, atol=1e-6 * np.abs(D).max())
    np.testing.assert_allclose(D, D.T, atol=1e-10 * np.abs(D).max())


# ----------------------------------------------------------------------------- Newton system


def _converged_config(K, seed, steps=6, n=3):
    tree = W.tree_d10_fit(K, seed=seed)
    A2, lam, Q = W.orientation_field(n, seed=seed + 1)
    Ef = W.random6_path_final(n, 0.03, seed=seed + 2)
    out = run_path(tree, lam, Q, Ef, 10, upto=steps)
    return tree, lam, Q, Ef, out


def _z_per_leaf(tree, st, i):
    L = 1 << tree.K
    z = np.zeros((L, 7))
    slot = 0
    for l in range(L):
        if tree.phases[l % 2].kind == 1:
            b = st[6 * slot:6 * slot + 6, i]
            z[l] = [b[0], b[1], b[2], -(b[1] + b[2]), b[3], b[4], b[5]]
            slot += 1
    return z


def _E_loc(Q, E):
    Qm = Q.reshape(3, 3)
    return T_to_mandel(Qm.T @ mandel_to_T(E) @ Qm)


@pytest.mark.parametrize("K", [2, 4, 5])
def test_newton_system_against_dense_algebra(K):
    tree, lam, Q, Ef, (st, sig, C, it, stat, _) = _converged_config(K, seed=30 + K, steps=4)
    i = 1
    L, N = 1 << K, (1 << K) - 1
    # a perturbed iterate near the solution, with the state of step 3 frozen
    st3 = run_path(tree, lam, Q, Ef, 10, upto=3)[0]
    z = _z_per_leaf(tree, st3, i)
    a = st[6 * (L // 2):, i] + 1e-4 * np.random.default_rng(K).standard_normal(3 * N)
    En, dE = W.proportional_increment(Ef, 4, 10)
    E_loc = _E_loc(Q[i], En[i] + dE[i])
    sysd = oracle.newton_system(tree, *lam[i], E_loc, a, z)
    assert sysd["rc"] == 0
    A = oracle.gradient_operator(tree, *lam[i])
    w = tree.w / tree.w.sum()
    eps = E_loc[None, :] + (A @ a).reshape(L, 6)
    np.testing.assert_allclose(sysd["eps"], eps, atol=1e-15)
    Ds, sigs = [], []
    for l in range(L):
        s_l, D_l, _ = oracle.phase_law(tree.phases[l % 2], eps[l], z[l])
        Ds.append(D_l)
        sigs.append(s_l)
    Wd = np.kron(np.diag(w), np.eye(6))
    Dbig = np.zeros((6 * L, 6 * L))
    for l in range(L):
        Dbig[6 * l:6 * l + 6, 6 * l:6 * l + 6] = Ds[l]
    R = A.T @ Wd @ np.concatenate(sigs)
    J = A.T @ Wd @ Dbig @ A
    np.testing.assert_allclose(sysd["R"], R, atol=1e-12 * np.abs(R).max())
    np.testing.assert_allclose(sysd["J"], J, atol=1e-12 * np.abs(J).max())
    assert np.linalg.eigvalsh(0.5 * (J + J.T)).min() > 0
    da = np.linalg.solve(J, -R)
    np.testing.assert_allclose(sysd["da"], da, atol=1e-9 * np.abs(da).max())
    np.testing.assert_allclose(sysd["sbar"], (w[:, None] * np.array(sigs)).sum(0), atol=1e-12)


@pytest.mark.parametrize("K", [3, 6])
def test_converged_state_equilibrium_hill_mandel_and_strain_average(K):
    tree, lam, Q, Ef, (st, sig, C, it, stat, _) = _converged_config(K, seed=40 + K, steps=5)
    assert np.all(stat == 0)
    L, N = 1 << K, (1 << K) - 1
    st4 = run_path(tree, lam, Q, Ef, 10, upto=4)[0]
    w = tree.w / tree.w.sum()
    En, dE = W.proportional_increment(Ef, 5, 10)
    nz = 6 * (L // 2)
    for i in range(lam.shape[0]):
        E_loc = _E_loc(Q[i], En[i] + dE[i])
        sysd = oracle.newton_system(tree, *lam[i], E_loc, st[nz:, i], _z_per_leaf(tree, st4, i))
        sbar = sysd["sbar"]
        assert np.linalg.norm(sysd["R"]) <= 1e-12 * N * np.linalg.norm(sbar)
        np.testing.assert_allclose((w[:, None] * sysd["eps"]).sum(0), E_loc, atol=1e-16)
        hm = (w * np.einsum("li,li->l", sysd["sig"], sysd["eps"])).sum()
        assert abs(hm - sbar @ E_loc) < 1e-10 * abs(hm)
        Qm = Q[i].reshape(3, 3)
        np.testing.assert_allclose(sig[i], T_to_mandel(Qm @ mandel_to_T(sbar) @ Qm.T), atol=1e-11 * np.abs(sbar).max())


def test_algorithmic_tangent_matches_finite_differences():
    K, n = 4, 4
    tree = W.tree_d10_fit(K, seed=50)
    A2, lam, Q = W.orientation_field(n, seed=51)
    Ef = W.random6_path_final(n, 0.03, seed=52)
    st = run_path(tree, lam, Q, Ef, 10, upto=6)[0]
    En, dE = W.proportional_increment(Ef, 7, 10)
    _, sig, C, it, stat, gap = oracle.update(tree, lam, Q, En, dE, st)
    assert np.all(stat == 0) and gap.min() > 1e-4
    h = 1e-8
    Cfd = np.zeros((n, 6, 6))
    for j in range(6):
        e = np.zeros(6)
        e[j] = h
        sp = oracle.update(tree, lam, Q, En, dE + e, st)[1]
        sm = oracle.update(tree, lam, Q, En, dE - e, st)[1]
        Cfd[:, :, j] = (sp - sm) / (2 * h)
    for i in range(n):
        np.testing.assert_allclose(C[i], Cfd[i], rtol=0, atol=1e-6 * np.abs(C[i]).max())


def test_unloading_tangent_is_the_elastic_dmn_stiffness():
    K, n = 4, 3
    tree = W.tree_d10_fit(K, seed=60)
    A2, lam, Q = W.orientation_field(n, seed=61)
    Ef = W.random6_path_final(n, 0.03, seed=62)
    st = run_path(tree, lam, Q, Ef, 10, upto=8)[0]
    assert np.abs(st[: 6 * (1 << (K - 1))]).max() > 1e-4        # plastic flow happened
    En, _ = W.proportional_increment(Ef, 9, 10)
    dE = -0.02 * (Ef / 10)                                     # small step back: all leaves unload
    _, sig, C, it, stat, _ = oracle.update(tree, lam, Q, En, dE, st)
    tree_el = W.TreeParams(K, tree.M, tree.p, tree.q, tree.w, (W.FIBER, ELASTIC_MATRIX))
    for i in range(n):
        Cl = linear_dmn_alpha(tree_el, (C_FIB, C_MAT), oracle.normals(tree, *lam[i]), 4e5)
        Cg, _ = oracle.rotate(Q[i].reshape(3, 3), Cl, np.zeros(6))
        np.testing.assert_allclose(C[i], Cg, atol=1e-10 * np.abs(Cg).max())


def test_newton_converges_quadratically_and_line_search_agrees():
    K, n = 5, 6
    tree = W.tree_d10_fit(K, seed=70)
    A2, lam, Q = W.orientation_field(n, seed=71)
    Ef = W.random6_path_final(n, 0.03, seed=72)
    out_a = run_path(tree, lam, Q, Ef, 5)
    out_b = run_path(tree, lam, Q, Ef, 5, line_search=True)
    assert np.all(out_a[4] == 0) and np.all(out_b[4] == 0)
    assert out_a[3].max() <= 6
    np.testing.assert_allclose(out_a[1], out_b[1], atol=1e-10 * np.abs(out_a[1]).max())
    # residual history of one increment: each step squares the relative error
    st = run_path(tree, lam, Q, Ef, 5, upto=2)[0]
    En, dE = W.proportional_increment(Ef, 3, 5)
    i = 0
    L, N = 1 << K, (1 << K) - 1
    z = _z_per_leaf(tree, st, i)
    E_loc = _E_loc(Q[i], En[i] + dE[i])
    a = st[6 * (L // 2):, i].copy()
    norms = []
    for _ in range(6):
        sysd = oracle.newton_system(tree, *lam[i], E_loc, a, z)
        norms.append(np.linalg.norm(sysd["R"]) / np.linalg.norm(sysd["sbar"]))
        a = a + sysd["da"]
    # once inside the basin (relative residual < 1e-6) the next step squares it
    k = next(k for k in range(1, len(norms)) if norms[k - 1] < 1e-6)
    assert norms[k] < 1e3 * norms[k - 1] ** 2 + 1e-15
    assert min(norms) < 1e-12 * N


def test_status_codes():
    K, n = 3, 4
    tree = W.tree_d10_fit(K, seed=80)
    A2, lam, Q = W.orientation_field(n, seed=81)
    S = oracle.state_size(K, tree.phases)
    E = np.full((n, 6), 0.02)
    E[1, 2] = np.nan
    st, sig, C, it, stat, _ = oracle.update(tree, lam, Q, np.zeros((n, 6)), E, np.zeros((S, n)), max_iter=1)
    assert stat[1] == 2 and np.isnan(sig[1]).all()
    assert stat[0] == 1 and it[0] == 1                # plastic first step needs more than one Newton step
    st, sig, C, it, stat, _ = oracle.update(tree, lam, Q, np.zeros((n, 6)), np.zeros((n, 6)), np.zeros((S, n)))
    assert np.all(stat == 0) and np.all(it == 0) and np.all(sig == 0)


# ----------------------------------------------------------------------------- orientation


def test_barycentric_coordinates_at_corners_and_centre():
    for lam, phi in (((1.0, 0.0), (1, 0, 0)), ((1 / 3, 1 / 3), (0, 1, 0)), ((0.5, 0.5), (0, 0, 1))):
        np.testing.assert_allclose(oracle.barycentric(*lam), phi, atol=1e-15)
    rng = np.random.default_rng(0)
    for _ in range(20):    # affine in lam: reproduces any convex combination of the corners
        t = rng.dirichlet(np.ones(3))
        lam = t @ W.TRIANGLE_CORNERS
        np.testing.assert_allclose(oracle.barycentric(*lam), t, atol=1e-14)


@pytest.mark.parametrize("M", [3, 4, 6])
def test_normals_are_unit_and_interpolate_nodal_angles(M):
    K = 3
    N = 7
    rng = np.random.default_rng(M)
    alpha, beta = rng.uniform(0, np.pi, N), rng.uniform(0, 2 * np.pi, N)
    # constant angles: shape functions are a partition of unity, so n does not depend on lam
    t0 = W.TreeParams(K, M, np.repeat(alpha[:, None], M, 1), np.repeat(beta[:, None], M, 1), np.ones(8))
    n_ref = oracle.normals(t0, 1 / 3, 1 / 3)
    for lam in ((1.0, 0.0), (0.5, 0.5), (0.6, 0.25)):
        np.testing.assert_allclose(oracle.normals(t0, *lam), n_ref, atol=1e-14)
    np.testing.assert_allclose(np.linalg.norm(n_ref, axis=1), 1.0, atol=1e-15)
    # spherical coordinates: alpha = 0 -> e3, (pi/2, 0) -> e1, (pi/2, pi/2) -> e2
    spec = W.TreeParams(1, M, np.array([[0.0] * M]), np.array([[0.3] * M]), np.ones(2))
    np.testing.assert_allclose(oracle.normals(spec, 0.5, 0.3)[0], [0, 0, 1], atol=1e-15)
    for b, e in ((0.0, [1, 0, 0]), (np.pi / 2, [0, 1, 0])):
        spec = W.TreeParams(1, M, np.array([[np.pi / 2] * M]), np.array([[b] * M]), np.ones(2))
        np.testing.assert_allclose(oracle.normals(spec, 0.5, 0.3)[0], e, atol=1e-15)
    # nodal property: coefficient m only acts at its own interpolation node
    nodes = {3: [(1.0, 0.0), (1 / 3, 1 / 3), (0.5, 0.5)],
             4: [(1.0, 0.0), (1 / 3, 1 / 3), (0.5, 0.5), tuple(np.ones(3) / 3 @ W.TRIANGLE_CORNERS)],
             6: [(1.0, 0.0), (1 / 3, 1 / 3), (0.5, 0.5), tuple(np.array([0.5, 0.5, 0]) @ W.TRIANGLE_CORNERS),
                 tuple(np.array([0.5, 0, 0.5]) @ W.TRIANGLE_CORNERS),
                 tuple(np.array([0, 0.5, 0.5]) @ W.TRIANGLE_CORNERS)]}[M]
    for m in range(M):
        p = np.zeros((1, M))
        p[0, m] = 1.0
        t1 = W.TreeParams(1, M, p, np.zeros((1, M)), np.ones(2))
        for mm, lam in enumerate(nodes):
            a = np.arccos(np.clip(oracle.normals(t1, *lam)[0, 2], -1, 1))
            assert abs(a - (1.0 if mm == m else 0.0)) < 1e-7


def test_eigen_decomposition_against_numpy():
    A2, lam, Q = W.orientation_field(200, seed=90)
    lo, Qo = oracle.interp_orientation(A2)
    for i in range(200):
        A = np.array([[A2[i, 0], A2[i, 5], A2[i, 4]], [A2[i, 5], A2[i, 1], A2[i, 3]], [A2[i, 4], A2[i, 3], A2[i, 2]]])
        ev, V = np.linalg.eigh(A)
        np.testing.assert_allclose(lo[i], ev[::-1][:2], atol=1e-14)
        Qm = Qo[i].reshape(3, 3)
        np.testing.assert_allclose(Qm.T @ Qm, np.eye(3), atol=1e-14)
        assert abs(np.linalg.det(Qm) - 1.0) < 1e-14
        l3 = np.array([lo[i, 0], lo[i, 1], np.trace(A) - lo[i].sum()])
        np.testing.assert_allclose(Qm @ np.diag(l3) @ Qm.T, A, atol=1e-14)
        for c in range(2):
            assert Qm[np.argmax(np.abs(Qm[:, c])), c] > 0
            assert abs(abs(Qm[:, c] @ V[:, 2 - c]) - 1.0) < 1e-10     # same direction as numpy's


def test_rotation_of_stiffness_and_stress():
    rng = np.random.default_rng(3)
    Qm = W.haar_rotations(rng, 1)[0]
    Ci = iso(1000.0, 0.25)
    v = rng.standard_normal(6)
    Cg, vg = oracle.rotate(Qm, Ci, v)
    np.testing.assert_allclose(Cg, Ci, atol=1e-10)                   # isotropy
    np.testing.assert_allclose(vg, T_to_mandel(Qm @ mandel_to_T(v) @ Qm.T), atol=1e-14)
    # Mandel rotation matrix: R_IJ = B_I : (Q B_J Q^T) ; C_glob = R C R^T
    B = [mandel_to_T(np.eye(6)[J]) for J in range(6)]
    R = np.array([[np.sum(B[I] * (Qm @ B[J] @ Qm.T)) for J in range(6)] for I in range(6)])
    Cr = rng.standard_normal((6, 6))
    Cr = Cr + Cr.T
    Cg, _ = oracle.rotate(Qm, Cr, v)
    np.testing.assert_allclose(Cg, R @ Cr @ R.T, atol=1e-13)
