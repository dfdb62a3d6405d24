"""Pins of the CPU FE oracle (oracle/fe_oracle.py) against what the mathematics
fixes: exact integration of the mesh volume, exact strains of linear
displacement fields, the patch test, rigid-body modes of the tangent, and the
consistency of internal force and tangent for a linear material."""
import math

import numpy as np

import oracle
from oracle import fe_oracle as FE
from paper_2103_08253_gb300 import workloads as W

ONE = np.array([1.0, 1.0, 1.0, 0.0, 0.0, 0.0])


def iso(E, nu):
    K = E / (3 * (1 - 2 * nu))
    G = E / (2 * (1 + nu))
    P1 = np.outer(ONE, ONE) / 3
    return 3 * K * P1 + 2 * G * (np.eye(6) - P1)


def mandel_sym(A):
    S = 0.5 * (A + A.T)
    s = math.sqrt(2.0)
    return np.array([S[0, 0], S[1, 1], S[2, 2], s * S[1, 2], s * S[0, 2], s * S[0, 1]])


def small_plate(n_t=4, n_r=3, n_z=2, perturb=0.0, seed=0):
    m = W.plate_with_hole_mesh(n_t, n_r, n_z, R=2.0, H=6.0, T=2.0)
    if perturb:
        rng = np.random.default_rng(seed)
        xyz = m.xyz.copy()
        interior = ~np.isin(np.arange(len(xyz)), boundary_nodes(m))
        xyz[interior] += perturb * rng.standard_normal((interior.sum(), 3))
        m.xyz = xyz
    return m


def boundary_nodes(m):
    """Nodes on the hole, the outer square and the two z faces."""
    x, y, z = m.xyz.T
    r = np.hypot(x, y)
    on = (np.abs(r - m.R) < 1e-9) | (np.abs(np.maximum(np.abs(x), np.abs(y)) - m.H) < 1e-9)
    on |= (np.abs(z) < 1e-9) | (np.abs(z - m.T / 2) < 1e-9)
    return np.nonzero(on)[0]


def test_mesh_volume_is_integrated_exactly():
    """Extruded trilinear elements have det(J) bilinear in the plane: 2-point Gauss is exact.
    The hole is the regular 4 n_t-gon through the hole nodes."""
    for n_t, n_r, n_z in ((4, 2, 1), (6, 3, 2)):
        m = W.plate_with_hole_mesh(n_t, n_r, n_z, R=2.0, H=6.0, T=2.0)
        mesh = FE.Mesh(m.xyz, m.conn)
        N = 4 * n_t
        hole = 0.5 * N * m.R ** 2 * math.sin(2 * math.pi / N)
        assert abs(mesh.volume() - (4 * m.H ** 2 - hole) * m.T / 2) < 1e-11 * mesh.volume()


def test_linear_displacement_gives_exact_uniform_strain():
    m = small_plate(perturb=0.15, seed=1)
    mesh = FE.Mesh(m.xyz, m.conn)
    A = np.random.default_rng(2).standard_normal((3, 3)) * 1e-3
    u = (m.xyz @ A.T).reshape(-1)
    E = mesh.strain(u)
    np.testing.assert_allclose(E, np.broadcast_to(mandel_sym(A), E.shape), rtol=0, atol=1e-15)


def test_patch_test_reproduces_a_linear_field():
    """Homogeneous linear elasticity, u = A x prescribed on every boundary node: the interior
    nodes of a distorted mesh take u = A x and the internal forces vanish there."""
    m = small_plate(n_t=4, n_r=4, n_z=3, perturb=0.12, seed=3)
    mesh = FE.Mesh(m.xyz, m.conn)
    A = np.random.default_rng(4).standard_normal((3, 3)) * 1e-3
    exact = (m.xyz @ A.T).reshape(-1)
    bnd = boundary_nodes(m)
    fixed = np.zeros((len(m.xyz), 3), dtype=bool)
    fixed[bnd] = True
    fixed = fixed.reshape(-1)
    assert (~fixed).sum() > 0
    C = np.broadcast_to(iso(3000.0, 0.35), (mesh.n_gp, 6, 6)).copy()
    K = mesh.stiffness(C)
    u0 = np.where(fixed, exact, 0.0)
    u = u0 - FE.solve_free(K, K @ u0, fixed)
    np.testing.assert_allclose(u, exact, rtol=0, atol=1e-12 * np.abs(exact).max())
    f = mesh.internal_force(mesh.strain(u) @ C[0].T)
    assert np.abs(f[~fixed]).max() < 1e-10 * np.abs(f).max()


def test_tangent_has_the_six_rigid_body_modes_and_is_symmetric():
    m = small_plate(perturb=0.1, seed=5)
    mesh = FE.Mesh(m.xyz, m.conn)
    rng = np.random.default_rng(6)
    L = rng.standard_normal((mesh.n_gp, 6, 6))
    C = np.einsum("gij,gkj->gik", L, L) + 6 * np.eye(6)[None]     # SPD per Gauss point
    K = mesh.stiffness(C)
    assert abs(K - K.T).max() < 1e-12 * abs(K).max()
    X = m.xyz
    modes = [np.tile(e, (len(X), 1)) for e in np.eye(3)]
    for ax in np.eye(3):
        modes.append(np.cross(ax, X))                                   # infinitesimal rotation
    for v in modes:
        assert np.abs(K @ v.reshape(-1)).max() < 1e-11 * abs(K).max() * np.abs(v).max()
    # and nothing else is free: K restricted to the non-rigid complement is definite
    rnd = rng.standard_normal(mesh.n_dofs)
    assert rnd @ (K @ rnd) > 0


def test_internal_force_is_the_tangent_times_u_for_a_linear_material():
    m = small_plate(perturb=0.1, seed=7)
    mesh = FE.Mesh(m.xyz, m.conn)
    rng = np.random.default_rng(8)
    L = rng.standard_normal((mesh.n_gp, 6, 6))
    C = np.einsum("gij,gkj->gik", L, L) + np.eye(6)[None]
    u = rng.standard_normal(mesh.n_dofs)
    sig = np.einsum("gij,gj->gi", C, mesh.strain(u))
    np.testing.assert_allclose(mesh.internal_force(sig), mesh.stiffness(C) @ u, rtol=1e-12,
                               atol=1e-12 * np.abs(sig).max())


def test_fe_dmn_elastic_run_is_linear_and_plastic_run_softens():
    m = W.plate_with_hole_mesh(4, 2, 1, R=2.0, H=6.0, T=2.0)
    mesh = FE.Mesh(m.xyz, m.conn)
    A2 = np.repeat(W.plate_orientation_field(m.centroid, m.R, m.H, m.T, seed=9), 8, axis=0)
    lam, Q = oracle.interp_orientation(A2)
    d = 0.015 * 2 * m.H
    el = W.tree_d10_fit(3, seed=10, phases=(W.FIBER, W.Phase(0, 3000.0, 0.35)))
    res = FE.run_fe_dmn(mesh, el, lam, Q, m.fixed, m.pull, [d / 3, 2 * d / 3, d], affine=m.affine)
    r = [x["reaction"] for x in res]
    assert abs(r[1] - 2 * r[0]) < 1e-9 * abs(r[1]) and abs(r[2] - 3 * r[0]) < 1e-9 * abs(r[2])
    assert res[0]["newton"] <= 1 and res[1]["newton"] <= 1  # at most one exact step for a linear problem
    pl = W.tree_d10_fit(3, seed=10)
    res = FE.run_fe_dmn(mesh, pl, lam, Q, m.fixed, m.pull, [d / 3, 2 * d / 3, d], affine=m.affine)
    r = [x["reaction"] for x in res]
    assert 0 < r[2] - r[1] < r[1] - r[0] < r[0]      # concave force-displacement curve
