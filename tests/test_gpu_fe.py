"""The FE operator (include/fe.h) and the FE-DMN driver against the CPU FE oracle.

Operators: strains, internal forces, the matrix-free tangent and its diagonal
against the oracle's explicit B matrices and assembled sparse tangent on a
distorted mesh.  Solver: Jacobi-PCG against a sparse direct solve.  Coupled
run: a small plate with a hole in tension, every Gauss point a depth-3 DMN,
against the oracle's FE-DMN Newton with direct solves."""
import numpy as np
import pytest
import torch

import oracle
from oracle import fe_oracle as FE
from paper_2103_08253_gb300 import fe, workloads as W

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda:0")


def d(x):
    return torch.from_numpy(np.ascontiguousarray(x)).to(DEV)


def distorted_plate(seed):
    m = W.plate_with_hole_mesh(6, 3, 2, R=2.0, H=6.0, T=2.0)
    rng = np.random.default_rng(seed)
    m.xyz = m.xyz + 0.08 * rng.standard_normal(m.xyz.shape)
    return m


def spd_field(n, seed):
    rng = np.random.default_rng(seed)
    L = rng.standard_normal((n, 6, 6))
    return np.einsum("gij,gkj->gik", L, L) + 3 * np.eye(6)[None]


def test_operators_match_the_oracle():
    m = distorted_plate(1)
    ref = FE.Mesh(m.xyz, m.conn)
    g = fe.Hex8Mesh(m.xyz, m.conn)
    assert g.n_gp == ref.n_gp and g.n_dofs == ref.n_dofs
    assert abs(g.volume - ref.volume()) < 1e-12 * ref.volume()
    rng = np.random.default_rng(2)
    u = rng.standard_normal(ref.n_dofs)
    sig = rng.standard_normal((ref.n_gp, 6))
    C = spd_field(ref.n_gp, 3)
    C[::5] += rng.standard_normal((len(C[::5]), 6, 6))       # some non-symmetric tangents too
    E = g.strain(d(u)).cpu().numpy()
    np.testing.assert_allclose(E, ref.strain(u), rtol=0, atol=1e-13 * np.abs(E).max())
    f = g.internal_force(d(sig)).cpu().numpy()
    np.testing.assert_allclose(f, ref.internal_force(sig), rtol=0, atol=1e-12 * np.abs(f).max())
    K = ref.stiffness(C)
    Kv = g.apply_tangent(d(C.reshape(-1, 36)), d(u)).cpu().numpy()
    np.testing.assert_allclose(Kv, K @ u, rtol=0, atol=1e-12 * np.abs(Kv).max())
    dg = g.tangent_diagonal(d(C.reshape(-1, 36))).cpu().numpy()
    np.testing.assert_allclose(dg, K.diagonal(), rtol=0, atol=1e-12 * np.abs(dg).max())
    assert abs(g.dot(d(u), d(f)) - u @ f) < 1e-12 * np.abs(u).max() * np.abs(f).sum()
    g.close()


def test_pcg_matches_a_direct_solve():
    m = distorted_plate(4)
    ref = FE.Mesh(m.xyz, m.conn)
    g = fe.Hex8Mesh(m.xyz, m.conn)
    C = spd_field(ref.n_gp, 5)
    K = ref.stiffness(C)
    rng = np.random.default_rng(6)
    b = rng.standard_normal(ref.n_dofs)
    x_ref = FE.solve_free(K, b, m.fixed)
    Cd = d(C.reshape(-1, 36))
    free = d((~m.fixed).astype(np.float64))
    diag = g.tangent_diagonal(Cd)
    x = torch.empty(ref.n_dofs, dtype=torch.float64, device=DEV)
    it, res = g.pcg(Cd, free, diag, d(b), x, rtol=1e-12, max_iter=5000)
    assert res <= 1e-12 and 0 < it < 5000
    xg = x.cpu().numpy()
    assert np.abs(xg[m.fixed]).max() == 0.0
    assert np.linalg.norm(xg - x_ref) <= 1e-9 * np.linalg.norm(x_ref)
    # FP32 products: the residual reachable is about 1e-6
    it32, res32 = g.pcg(Cd, free, diag, d(b), x, rtol=1e-6, max_iter=5000, f32=True)
    assert res32 <= 1e-6 and 0 < it32 < 5000
    assert np.linalg.norm(x.cpu().numpy() - x_ref) <= 1e-4 * np.linalg.norm(x_ref)
    # zero right-hand side: zero solution, no iterations
    it, res = g.pcg(Cd, free, diag, torch.zeros_like(x), x, rtol=1e-8)
    assert it == 0 and float(x.abs().max()) == 0.0
    g.close()


@pytest.mark.parametrize("prec,tol,cg32,pred", [("f64", 1e-8, False, False), ("mixed", 1e-6, False, False),
                                               ("f64", 1e-6, True, False), ("mixed-f32-tangent", 1e-6, True, False),
                                               ("f64", 1e-6, False, True)])
def test_fe_dmn_plate_matches_the_oracle(prec, tol, cg32, pred):
    """The FE oracle runs the paper's start; with the extrapolated start (pred) the DMN reaches
    the same solution up to its stopping criterion, so the same tolerance holds."""
    m = W.plate_with_hole_mesh(4, 2, 1, R=2.0, H=6.0, T=2.0)
    A2 = W.plate_orientation_field(m.centroid, m.R, m.H, m.T, seed=11)
    tree = W.tree_d10_fit(3, seed=12)
    deltas = [0.015 * 2 * m.H * k / 3 for k in (1, 2, 3)]
    lam, Q = oracle.interp_orientation(np.repeat(A2, 8, axis=0))
    ref = FE.run_fe_dmn(FE.Mesh(m.xyz, m.conn), tree, lam, Q, m.fixed, m.pull, deltas, affine=m.affine, rtol=1e-10)
    run = fe.FEDMN(m, tree, A2, precision=prec, newton_rtol=1e-10, cg_rtol=1e-6 if cg32 else 1e-13, cg_f32=cg32,
                   predictor=pred)
    for k, delta in enumerate(deltas):
        r = run.increment(delta)
        assert r["converged"] and r["dmn_status_bad"] == 0, r
        u = run.u.cpu().numpy()
        assert np.linalg.norm(u - ref[k]["u"]) <= tol * np.linalg.norm(ref[k]["u"]), k
        assert abs(r["reaction"] - ref[k]["reaction"]) <= tol * abs(ref[k]["reaction"]), k
        sig = run.out["stress"].cpu().numpy()
        assert np.abs(sig - ref[k]["stress"]).max() <= tol * 10 * np.abs(ref[k]["stress"]).max(), k
    assert ref[-1]["newton"] >= 2              # the last increment is plastic
    run.close()
