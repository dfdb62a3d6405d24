"""Parity of the CUDA path (through the C ABI) with the CPU oracle.

Tolerances: FP64 form <= 1e-10 relative in stress and tangent; mixed form
<= 1e-6 relative in stress and tangent (both forms stop on the same FP64
residual criterion, so both land on the FP64 fixed point; the mixed form's
tangent comes from an FP64 sweep).  The mixed form with an FP32 tangent has
the mixed form's stress and a tangent condensed in FP32: 8 levels of a
condensation whose 3x3 solves have condition numbers up to the phase
contrast (about 35 elastic, more once the matrix yields), each adding a few
FP32 roundings (6e-8), bound it by 1e-4.  Relative errors are per point,
||x_gpu - x_oracle||_F / ||x_oracle||_F.  Iteration counts of the FP64 form
must match the oracle's (the two compute the same Newton iterates by different
eliminations).  A yield decision that the rounding order could flip
(|f| / sigma_Y < 1e-9 at the final iterate) would allow a jump in the tangent;
such points are counted and excluded from the tangent check.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2103_08253_gb300 import dmn, workloads as W

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda:0")
TOL = {"f64": 1e-10, "mixed": 1e-6, "mixed-f32-tangent": 1e-6}
TOL_TANGENT = {"f64": 1e-10, "mixed": 1e-6, "mixed-f32-tangent": 1e-4}


def rel(a, b):
    a = a.reshape(a.shape[0], -1)
    b = b.reshape(b.shape[0], -1)
    return np.linalg.norm(a - b, axis=1) / np.maximum(np.linalg.norm(b, axis=1), 1e-300)


def d(x):
    return torch.from_numpy(np.ascontiguousarray(x)).to(DEV)


def run_path(tree, lam, Q, Ef, n_steps, prec, upto=None, compare=True, max_iter=50, **opt):
    """Run the same load path through the GPU and the oracle, comparing every increment."""
    n = lam.shape[0]
    S = W.state_size(tree.K, tree.phases)
    m = dmn.DMN(tree, precision=prec, max_iter=max_iter, **opt)
    assert m.state_size == S
    st_g = torch.zeros((S, n), dtype=torch.float64, device=DEV)
    st_o = np.zeros((S, n))
    lam_d, Q_d = d(lam), d(Q)
    worst = dict(stress=0.0, tangent=0.0, state=0.0, iters_mismatch=0, ties=0)
    for s in range(1, (upto or n_steps) + 1):
        En, dE = W.proportional_increment(Ef, s, n_steps)
        out = m.update(lam_d, Q_d, d(En), d(dE), st_g)
        st_g = out["state_out"]
        st_o, sig_o, C_o, it_o, stat_o, gap = oracle.update(tree, lam, Q, En, dE, st_o, max_iter=max_iter)
        if not compare:
            continue
        torch.cuda.synchronize()
        sig = out["stress"].cpu().numpy()
        C = out["tangent"].cpu().numpy()
        it = out["iters"].cpu().numpy()
        stat = out["status"].cpu().numpy()
        np.testing.assert_array_equal(stat, stat_o)
        ok = stat_o == 0
        es = rel(sig[ok], sig_o[ok])
        tie = gap[ok] < 1e-9
        ec = rel(C[ok][~tie], C_o[ok][~tie])
        sg = st_g.cpu().numpy()
        scale = np.abs(st_o).max(axis=1, keepdims=True) + 1e-300
        est = (np.abs(sg - st_o) / scale).max()
        worst["stress"] = max(worst["stress"], es.max(initial=0.0))
        worst["tangent"] = max(worst["tangent"], ec.max(initial=0.0))
        worst["state"] = max(worst["state"], est)
        worst["ties"] += int(tie.sum())
        if prec == "f64":
            worst["iters_mismatch"] += int((it != it_o).sum())
            assert np.abs(it - it_o).max(initial=0) <= 1
    m.close()
    return worst, out, st_o


@pytest.mark.parametrize("prec", ["f64", "mixed"])
def test_depth4_uniaxial_path_1024_points(prec):
    """Plain K = 4 DMN, 1024 points, uniaxial strain to 2 % in 20 increments with
    random load directions; every increment compared."""
    K, n = 4, 1024
    tree = W.tree_constant_normals(K, seed=1)
    lam, Q = W.identity_orientation(n)
    Ef = W.uniaxial_path_final(n, 0.02, seed=2)
    worst, out, _ = run_path(tree, lam, Q, Ef, 20, prec)
    print(prec, worst)
    assert worst["stress"] <= TOL[prec]
    assert worst["tangent"] <= TOL[prec]
    assert worst["state"] <= (1e-9 if prec == "f64" else 1e-5)
    if prec == "f64":
        assert worst["iters_mismatch"] <= 0.005 * n * 20


@pytest.mark.parametrize("prec", ["f64", "mixed", "mixed-f32-tangent"])
def test_depth8_interpolated_random_paths(prec):
    """K = 8 with D10-fitted normals, orientations uniform over the triangle,
    random 6-component paths to 3 % equivalent strain; 48 points through the
    first 12 of 50 increments, plus increments 48-50 of a second set."""
    K, n = 8, 48
    tree = W.tree_d10_fit(K, seed=5)
    A2, lam, Q = W.orientation_field(n, seed=6)
    Ef = W.random6_path_final(n, 0.03, seed=7)
    worst, _, _ = run_path(tree, lam, Q, Ef, 50, prec, upto=12)
    print(prec, worst)
    assert worst["stress"] <= TOL[prec]
    assert worst["tangent"] <= TOL_TANGENT[prec]


def test_ragged_sizes_depths_and_launch_shapes():
    """n not a multiple of a warp or a CTA; depths 1..8; several CTA shapes of the thread-per-point
    kernel give bit-identical FP64 results."""
    for K, n in ((1, 1), (2, 33), (3, 129), (5, 257), (8, 37)):
        tree = W.tree_d10_fit(K, seed=10 + K)
        A2, lam, Q = W.orientation_field(n, seed=20 + K)
        Ef = W.random6_path_final(n, 0.025, seed=30 + K)
        worst, out, _ = run_path(tree, lam, Q, Ef, 4, "f64")
        assert worst["stress"] <= 1e-10 and worst["tangent"] <= 1e-10, (K, n, worst)
    K, n = 5, 300
    tree = W.tree_d10_fit(K, seed=40)
    A2, lam, Q = W.orientation_field(n, seed=41)
    Ef = W.random6_path_final(n, 0.03, seed=42)
    outs = []
    for block, cps in ((128, 2), (64, 1), (32, 3), (128, 2)):
        _, out, _ = run_path(tree, lam, Q, Ef, 3, "f64", compare=False, block=block, ctas_per_sm=cps,
                             warp_per_point=-1)
        outs.append({k: v.cpu().numpy() for k, v in out.items()})
    for o in outs[1:]:
        for k in o:
            np.testing.assert_array_equal(o[k], outs[0][k])


@pytest.mark.parametrize("M", [4, 6])
def test_higher_order_shape_functions(M):
    K, n = 3, 64
    rng = np.random.default_rng(M)
    N = (1 << K) - 1
    tree = W.TreeParams(K, M, rng.uniform(0.2, 2.8, (N, M)), rng.uniform(0, 6.2, (N, M)),
                        rng.dirichlet(np.ones(1 << K)))
    A2, lam, Q = W.orientation_field(n, seed=M + 50)
    Ef = W.random6_path_final(n, 0.03, seed=M + 60)
    worst, _, _ = run_path(tree, lam, Q, Ef, 5, "f64")
    assert worst["stress"] <= 1e-10 and worst["tangent"] <= 1e-10


@pytest.mark.parametrize("M", [4, 6])
def test_higher_order_shape_functions_depth8(M):
    """The timed shape-function variants of the bench: K = 8 with seeded nodal
    angles for the tri-linear and quadratic shape functions, 40 points, both
    forms, the first 4 of 50 increments to 3 % equivalent strain."""
    tree = W.tree_nodal_angles(8, M, seed=120 + M)
    A2, lam, Q = W.orientation_field(40, seed=121 + M)
    Ef = W.random6_path_final(40, 0.03, seed=122 + M)
    for prec in ("f64", "mixed"):
        worst, _, _ = run_path(tree, lam, Q, Ef, 50, prec, upto=4)
        assert worst["stress"] <= TOL[prec] and worst["tangent"] <= TOL_TANGENT[prec], (prec, worst)


@pytest.mark.parametrize("phases", [(W.MATRIX, W.MATRIX), (W.FIBER, W.Phase(0, 3000.0, 0.35)),
                                    (W.Phase(1, 3000.0, 0.35, 40.0, 300.0), W.FIBER)])
def test_phase_combinations(phases):
    """Both phases inelastic (one state slot per leaf), both elastic (no leaf
    state), and the inelastic phase on the odd leaves."""
    K, n = 4, 100
    tree = W.tree_d10_fit(K, seed=70, phases=phases)
    A2, lam, Q = W.orientation_field(n, seed=71)
    Ef = W.random6_path_final(n, 0.03, seed=72)
    for prec in ("f64", "mixed"):
        worst, _, _ = run_path(tree, lam, Q, Ef, 6, prec)
        assert worst["stress"] <= TOL[prec] and worst["tangent"] <= TOL[prec], (prec, worst)


@pytest.mark.parametrize("prec", ["f64", "mixed", "mixed-f32-tangent"])
def test_exponential_linear_matrix_depth8(prec):
    """The paper's material set: glass fiber and the polyamide matrix with
    exponential-linear hardening (Sec. 4.1, material table); K = 8, 48 points,
    the first 10 of 30 increments to 3 % equivalent strain, plus both phases
    inelastic at K = 4."""
    K, n = 8, 48
    tree = W.tree_d10_fit(K, seed=90, phases=(W.FIBER, W.MATRIX_EXPLIN))
    A2, lam, Q = W.orientation_field(n, seed=91)
    Ef = W.random6_path_final(n, 0.03, seed=92)
    worst, out, st_o = run_path(tree, lam, Q, Ef, 30, prec, upto=10)
    print(prec, worst)
    assert worst["stress"] <= TOL[prec] and worst["tangent"] <= TOL_TANGENT[prec]
    assert np.abs(st_o[0]).max() > 1e-3          # the matrix leaves did yield
    tree = W.tree_d10_fit(4, seed=93, phases=(W.MATRIX_EXPLIN, W.MATRIX_EXPLIN))
    A2, lam, Q = W.orientation_field(64, seed=94)
    Ef = W.random6_path_final(64, 0.03, seed=95)
    worst, _, _ = run_path(tree, lam, Q, Ef, 8, prec)
    assert worst["stress"] <= TOL[prec] and worst["tangent"] <= TOL_TANGENT[prec], worst


def test_f32_tangent_form_shares_the_mixed_iteration():
    """The FP32-tangent form runs the mixed form's Newton iteration: same
    jumps, leaf states, iteration counts and status, bit for bit, and the same
    FP64 stress up to the summation order of the final sweep; K = 8, 1000
    points (ragged against the launch), on a full and on a compressed tree."""
    K, n = 8, 1000
    A2, lam, Q = W.orientation_field(n, seed=112)
    Ef = W.random6_path_final(n, 0.03, seed=113)
    for tree in (W.tree_d10_fit(K, seed=110), W.tree_with_zero_weights(K, seed=111)):
        outs = {}
        for prec in ("mixed", "mixed-f32-tangent"):
            m = dmn.DMN(tree, precision=prec)
            st = torch.zeros((m.state_size, n), dtype=torch.float64, device=DEV)
            for s in range(1, 7):
                En, dE = W.proportional_increment(Ef, s, 50)
                out = m.update(d(lam), d(Q), d(En), d(dE), st)
                st = out["state_out"]
            torch.cuda.synchronize()
            outs[prec] = {k: v.cpu().numpy() for k, v in out.items()}
            m.close()
        a, b = outs["mixed"], outs["mixed-f32-tangent"]
        for k in ("state_out", "iters", "status"):
            np.testing.assert_array_equal(a[k], b[k])
        assert (a["status"] == 0).all()
        assert rel(b["stress"], a["stress"]).max() <= 1e-13
        et = rel(b["tangent"], a["tangent"])
        print("f32 tangent vs FP64 sweep: max %.2e, median %.2e" % (et.max(), np.median(et)))
        assert et.max() <= 1e-4 and et.max() > 0.0


def test_status_codes_and_degenerate_inputs():
    K, n = 4, 64
    tree = W.tree_d10_fit(K, seed=80)
    A2, lam, Q = W.orientation_field(n, seed=81)
    S = W.state_size(K)
    E = np.full((n, 6), 0.02)
    E[5, 2] = np.nan
    E[7] = 0.0
    for prec in ("f64", "mixed", "mixed-f32-tangent"):
        m = dmn.DMN(tree, precision=prec, max_iter=1)
        out = m.update(d(lam), d(Q), d(np.zeros((n, 6))), d(E), torch.zeros((S, n), dtype=torch.float64, device=DEV))
        st_o, sig_o, C_o, it_o, stat_o, _ = oracle.update(tree, lam, Q, np.zeros((n, 6)), E, np.zeros((S, n)),
                                                          max_iter=1)
        stat = out["status"].cpu().numpy()
        np.testing.assert_array_equal(stat, stat_o)
        assert stat[5] == dmn.STATUS_NONFINITE and stat[0] == dmn.STATUS_MAXITER and stat[7] == dmn.STATUS_OK
        assert np.isnan(out["stress"][5].cpu().numpy()).all() and np.isnan(out["state_out"][:, 5].cpu().numpy()).all()
        assert (out["iters"].cpu().numpy()[stat == 1] == 1).all()
        assert np.abs(out["stress"][7].cpu().numpy()).max() == 0.0 and out["iters"][7].item() == 0
        fine = stat != 2
        if prec == "f64":   # status MAXITER: outputs of the last iterate, as in the oracle
            assert rel(out["stress"].cpu().numpy()[fine], sig_o[fine]).max() < 1e-10
        m.close()
    m = dmn.DMN(tree)
    out = m.update(d(lam[:0]), d(Q[:0]), d(np.zeros((0, 6))), d(np.zeros((0, 6))),
                   torch.zeros((S, 0), dtype=torch.float64, device=DEV))
    assert out["stress"].shape == (0, 6)
    with pytest.raises(RuntimeError, match="must differ"):
        st = torch.zeros((S, n), dtype=torch.float64, device=DEV)
        m.update(d(lam), d(Q), d(E), d(E), st, out=dict(m.alloc_outputs(n, DEV), state_out=st))
    m.close()


def test_interp_orientation_against_oracle():
    n = 4099
    A2, lam_in, Q_in = W.orientation_field(n, seed=90)
    m = dmn.DMN(W.tree_d10_fit(2, seed=1))
    lam, Q = m.interp_orientation(d(A2))
    lam, Q = lam.cpu().numpy(), Q.cpu().numpy().reshape(n, 3, 3)
    lo, Qo = oracle.interp_orientation(A2)
    np.testing.assert_allclose(lam, lo, atol=1e-13)
    Qo = Qo.reshape(n, 3, 3)
    np.testing.assert_allclose(np.einsum("nki,nkj->nij", Q, Q), np.broadcast_to(np.eye(3), (n, 3, 3)), atol=1e-13)
    np.testing.assert_allclose(np.linalg.det(Q), 1.0, atol=1e-13)
    l3 = np.stack([lam[:, 0], lam[:, 1], A2[:, :3].sum(1) - lam.sum(1)], 1)
    A = np.einsum("nij,nj,nkj->nik", Q, l3, Q)
    np.testing.assert_allclose(A[:, [0, 1, 2, 1, 0, 0], [0, 1, 2, 2, 2, 1]], A2, atol=1e-13)
    gap = np.minimum(lo[:, 0] - lo[:, 1], lo[:, 1] - l3[:, 2])
    good = gap > 1e-5      # eigenvectors are well defined: same frame as the oracle's
    assert good.mean() > 0.99
    np.testing.assert_allclose(Q[good], Qo[good], atol=1e-9)
    m.close()


def test_interp_orientation_at_the_triangle_corners():
    """Orientation tensors with repeated eigenvalues: the corners UD (1, 0, 0), ISO (1/3, 1/3, 1/3) and
    PI (1/2, 1/2, 0) of the triangle and points 1e-9 and 1e-12 away, unrotated and in random frames.
    The eigenvalues are unique and must match the oracle's; the eigenframe within a repeated
    eigenvalue is not, so Q must be a right-handed orthonormal frame that reproduces A2.  The update
    on the GPU's (lam, Q) must then match the oracle's on the same (lam, Q)."""
    rng = np.random.default_rng(92)
    spectra = [(1.0, 0.0, 0.0), (1 / 3, 1 / 3, 1 / 3), (0.5, 0.5, 0.0), (1 - 2e-9, 1e-9, 1e-9),
               (0.5 + 1e-12, 0.5 - 1e-12, 0.0)]
    R = np.concatenate([np.eye(3)[None], W.haar_rotations(rng, 24)])
    A = np.einsum("rik,sk,rjk->srij", R, np.array(spectra), R).reshape(-1, 3, 3)
    A2 = np.ascontiguousarray(A[:, [0, 1, 2, 1, 0, 0], [0, 1, 2, 2, 2, 1]])
    n = A2.shape[0]
    m = dmn.DMN(W.tree_d10_fit(2, seed=1))
    lam_g, Q_g = m.interp_orientation(d(A2))
    m.close()
    lam, Q = lam_g.cpu().numpy(), Q_g.cpu().numpy()
    assert np.isfinite(lam).all() and np.isfinite(Q).all()
    lo, _ = oracle.interp_orientation(A2)
    np.testing.assert_allclose(lam, lo, atol=1e-13)
    Qm = Q.reshape(n, 3, 3)
    np.testing.assert_allclose(np.einsum("nki,nkj->nij", Qm, Qm), np.broadcast_to(np.eye(3), (n, 3, 3)), atol=1e-13)
    np.testing.assert_allclose(np.linalg.det(Qm), 1.0, atol=1e-13)
    l3 = np.stack([lam[:, 0], lam[:, 1], A2[:, :3].sum(1) - lam.sum(1)], 1)
    np.testing.assert_allclose(np.einsum("nij,nj,nkj->nik", Qm, l3, Qm), A, atol=1e-13)
    tree = W.tree_d10_fit(4, seed=93)
    Ef = W.random6_path_final(n, 0.025, seed=94)
    worst, _, _ = run_path(tree, lam, Q, Ef, 4, "f64")
    assert worst["stress"] <= 1e-10 and worst["tangent"] <= 1e-10, worst
    assert worst["iters_mismatch"] <= 0.005 * n * 4, worst


@pytest.mark.parametrize("prec", ["f64", "mixed"])
def test_points_are_independent_of_the_batch(prec):
    """Every point's update depends on that point alone: 65,537 points at depth 6 (more than one
    point per lane of the persistent kernel) give bit for bit the results of the same points
    updated as two uneven parts in the reverse order, in the thread-per-point organisation (the
    warp organisation, which small calls get by default, rounds differently)."""
    K, n, cut = 6, 65537, 40001
    tree = W.tree_d10_fit(K, seed=97)
    A2, lam, Q = W.orientation_field(n, seed=98)
    Ef = W.random6_path_final(n, 0.03, seed=99)
    m = dmn.DMN(tree, precision=prec, warp_per_point=-1)
    lam_d, Q_d = d(lam), d(Q)
    st = torch.zeros((m.state_size, n), dtype=torch.float64, device=DEV)
    for s in range(1, 4):
        En, dE = W.proportional_increment(Ef, s, 20)
        En_d, dE_d = d(En), d(dE)
        whole = m.update(lam_d, Q_d, En_d, dE_d, st)
        parts = {}
        for a, b in ((cut, n), (0, cut)):
            o = m.update(lam_d[a:b], Q_d[a:b], En_d[a:b], dE_d[a:b], st[:, a:b].contiguous())
            for k, v in o.items():
                parts.setdefault(k, [None, None])[0 if a == 0 else 1] = v
        for k, (lo, hi) in parts.items():
            joined = torch.cat([lo, hi], dim=1 if k == "state_out" else 0)
            assert torch.equal(joined, whole[k]), (prec, s, k)
        assert (whole["status"] == 0).all()
        st = whole["state_out"]
    m.close()


def test_repeatable_bitwise():
    K, n = 6, 500
    tree = W.tree_d10_fit(K, seed=95)
    A2, lam, Q = W.orientation_field(n, seed=96)
    Ef = W.random6_path_final(n, 0.03, seed=97)
    for prec in ("f64", "mixed"):
        a = run_path(tree, lam, Q, Ef, 3, prec, compare=False)[1]
        b = run_path(tree, lam, Q, Ef, 3, prec, compare=False)[1]
        for k in a:
            assert torch.equal(a[k], b[k]), (prec, k)
