"""The all-FP32 first Newton stage (the mixed forms' default, the FP64 form's option), through the C ABI,
against the oracle.

The stage runs Sec. 3.2's Newton iteration with every quantity in FP32 until its own residual is
small, and the FP64-residual iteration of the mixed forms continues from its jumps to the FP64
criterion.  So the results must meet the mixed forms' tolerances against the FP64 oracle (stress
<= 1e-6, tangent <= 1e-6 with the FP64 final sweep) on plastic paths, on full and compressed trees,
and agree with the same forms without the stage to the accuracy the common FP64 criterion leaves.
The pass counters must show the FP64-residual passes that the stage saves.
"""
import numpy as np
import pytest
import torch

from paper_2103_08253_gb300 import dmn, workloads as W
from test_gpu_parity import d, rel, run_path

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda:0")


@pytest.mark.parametrize("prec,matrix", [("mixed", "linear"), ("mixed-f32-tangent", "linear"), ("mixed", "explin")])
def test_first_stage_matches_the_oracle_at_depth_8(prec, matrix):
    phases = (W.FIBER, W.MATRIX_EXPLIN if matrix == "explin" else W.MATRIX)
    tree = W.tree_d10_fit(8, seed=301, phases=phases)
    n = 192
    A2, lam, Q = W.orientation_field(n, seed=302)
    Ef = W.random6_path_final(n, 0.03, seed=303)
    worst, out, _ = run_path(tree, lam, Q, Ef, 20, prec, upto=8, first_stage=True)
    assert worst["stress"] <= 1e-6
    assert worst["tangent"] <= (1e-6 if prec == "mixed" else 1e-4)
    assert worst["state"] <= 1e-5


def test_first_stage_on_a_compressed_tree():
    tree = W.tree_with_zero_weights(7, seed=311)
    n = 160
    A2, lam, Q = W.orientation_field(n, seed=312)
    Ef = W.random6_path_final(n, 0.03, seed=313)
    S = W.state_size(tree.K, tree.phases)
    m_on = dmn.DMN(tree, precision="mixed")
    m_off = dmn.DMN(tree, precision="mixed", first_stage=False)
    assert m_on.first_stage and not m_off.first_stage
    import oracle
    S = oracle.state_size(tree.K, tree.phases, tree.w)
    st_on = torch.zeros((m_on.state_size, n), dtype=torch.float64, device=DEV)
    st_off = st_on.clone()
    st_o = np.zeros((S, n))
    for s in range(1, 9):
        En, dE = W.proportional_increment(Ef, s, 20)
        a = m_on.update(d(lam), d(Q), d(En), d(dE), st_on)
        b = m_off.update(d(lam), d(Q), d(En), d(dE), st_off)
        st_o, sig_o, C_o, it_o, stat_o, gap = oracle.update(tree, lam, Q, En, dE, st_o)
        st_on, st_off = a["state_out"], b["state_out"]
        ok = (stat_o == 0) & (a["status"].cpu().numpy() == 0)
        assert ok.mean() > 0.95
        assert rel(a["stress"].cpu().numpy()[ok], sig_o[ok]).max() <= 1e-6
        tie = gap < 1e-9
        assert rel(a["tangent"].cpu().numpy()[ok & ~tie], C_o[ok & ~tie]).max() <= 1e-6
        # the same fixed point as the mixed iteration without the stage, to its stopping criterion
        assert rel(a["stress"].cpu().numpy()[ok], b["stress"].cpu().numpy()[ok]).max() <= 1e-8
    m_on.close()
    m_off.close()


def test_first_stage_saves_fp64_passes_and_the_counters_add_up():
    """Profiling counters: with the stage the Newton kernel runs fewer FP64-residual passes; the stage's
    and the Newton kernel's passes per point are each (corrections + 1), their corrections add up to
    the iteration counts; without the stage (or in the FP64 form by default) the stage counter stays zero."""
    tree = W.tree_d10_fit(8, seed=321)
    n = 4096
    A2, lam, Q = W.orientation_field(n, seed=322)
    Ef = W.random6_path_final(n, 0.03, seed=323)
    res = {}
    for key, prec, stage in (("on", "mixed", True), ("off", "mixed", False), ("f64", "f64", None)):
        m = dmn.DMN(tree, precision=prec, first_stage=stage)
        st = torch.zeros((m.state_size, n), dtype=torch.float64, device=DEV)
        for s in range(1, 6):
            En, dE = W.proportional_increment(Ef, s, 20)
            st = m.update(d(lam), d(Q), d(En), d(dE), st)["state_out"]
        En, dE = W.proportional_increment(Ef, 6, 20)
        m.profile(True)
        out = m.update(d(lam), d(Q), d(En), d(dE), st)
        ms, passes, upd = m.profile_read_stages()
        m.profile(False)
        assert upd == 1
        assert (out["status"] == 0).all()
        it = int(out["iters"].to(torch.int64).sum().item())
        if key == "on":
            assert ms["stage"] > 0.0 and passes["stage"] >= n
            # corrections of both kernels = the reported iterations
            assert (passes["stage"] - n) + (passes["newton"] - n) == it
        else:
            assert passes["stage"] == 0
            assert passes["newton"] - n == it
        res[key] = (passes, it, out["stress"].cpu().numpy())
        m.close()
    assert res["on"][0]["newton"] < 0.75 * res["off"][0]["newton"]
    assert rel(res["on"][2], res["f64"][2]).max() <= 1e-8


def test_first_stage_within_max_iter():
    """With a small max_iter the stage's corrections count against it: no point reports more."""
    tree = W.tree_d10_fit(6, seed=331)
    n = 512
    A2, lam, Q = W.orientation_field(n, seed=332)
    Ef = W.random6_path_final(n, 0.03, seed=333)
    m = dmn.DMN(tree, precision="mixed", max_iter=3)
    st = torch.zeros((m.state_size, n), dtype=torch.float64, device=DEV)
    for s in range(1, 5):
        En, dE = W.proportional_increment(Ef, s, 20)
        out = m.update(d(lam), d(Q), d(En), d(dE), st)
        st = out["state_out"]
        it = out["iters"].cpu().numpy()
        stat = out["status"].cpu().numpy()
        assert it.max() <= 3
        assert set(np.unique(stat)) <= {dmn.STATUS_OK, dmn.STATUS_MAXITER}
        assert (it[stat == dmn.STATUS_MAXITER] == 3).all()
    m.close()


def test_fp64_form_after_the_first_stage():
    """The FP64 form with the first stage on request: at least one FP64 Newton step after the stage, the
    FP64 criterion, FP64 tangent.  It stops at the same criterion as the oracle from another start, so it
    agrees with the oracle to that criterion's reach (||A^T W sigma|| <= 1e-12 x 255 ||sigma_bar|| leaves
    some 1e-9 of the stress open at depth 8; the oracle itself moves that much when converged further),
    not to rounding as the plain FP64 form does; and it needs far fewer FP64 passes."""
    import oracle
    tree = W.tree_d10_fit(8, seed=341)
    n = 256
    A2, lam, Q = W.orientation_field(n, seed=342)
    Ef = W.random6_path_final(n, 0.03, seed=343)
    S = W.state_size(8, tree.phases)
    m = dmn.DMN(tree, precision="f64", first_stage=True)
    plain = dmn.DMN(tree, precision="f64")
    assert m.first_stage and not plain.first_stage
    st, st_p = (torch.zeros((S, n), dtype=torch.float64, device=DEV) for _ in range(2))
    st_o = np.zeros((S, n))
    for s in range(1, 7):
        En, dE = W.proportional_increment(Ef, s, 20)
        m.profile(True)
        plain.profile(True)
        out = m.update(d(lam), d(Q), d(En), d(dE), st)
        ref = plain.update(d(lam), d(Q), d(En), d(dE), st_p)
        _, ps, _ = m.profile_read_stages()
        _, pp, _ = plain.profile_read_stages()
        st, st_p = out["state_out"], ref["state_out"]
        st_o, sig_o, C_o, it_o, stat_o, gap = oracle.update(tree, lam, Q, En, dE, st_o)
        assert (out["status"] == 0).all() and (stat_o == 0).all()
        tie = gap < 1e-9
        assert rel(out["stress"].cpu().numpy(), sig_o).max() <= 1e-8
        assert rel(out["tangent"].cpu().numpy()[~tie], C_o[~tie]).max() <= 1e-8
        assert ps["stage"] >= n and pp["stage"] == 0
        assert ps["newton"] >= 2 * n            # one FP64 step at least: two FP64 passes per point
        if s > 1:
            assert ps["newton"] < 0.7 * pp["newton"]
    m.close()
    plain.close()


@pytest.mark.parametrize("prec", ["mixed", "mixed-f32-tangent"])
def test_first_stage_ragged_sizes_and_depths(prec):
    """The stage at depths 1..8 and batch sizes that are not multiples of a warp or a CTA (one point
    included), against the oracle; and no launch at all for an empty batch."""
    for K, n in ((1, 1), (2, 33), (3, 129), (5, 257), (8, 37)):
        tree = W.tree_d10_fit(K, seed=350 + K)
        A2, lam, Q = W.orientation_field(n, seed=360 + K)
        Ef = W.random6_path_final(n, 0.025, seed=370 + K)
        worst, out, _ = run_path(tree, lam, Q, Ef, 4, prec, first_stage=True)
        assert worst["stress"] <= 1e-6, (K, n, worst)
        assert worst["tangent"] <= (1e-6 if prec == "mixed" else 1e-4), (K, n, worst)
    tree = W.tree_d10_fit(4, seed=380)
    m = dmn.DMN(tree, precision=prec)
    S = m.state_size
    m.profile(True)
    out = m.update(d(np.zeros((0, 2))), d(np.zeros((0, 9))), d(np.zeros((0, 6))), d(np.zeros((0, 6))),
                   torch.zeros((S, 0), dtype=torch.float64, device=DEV))
    assert out["stress"].shape == (0, 6)
    _, passes, upd = m.profile_read_stages()
    assert passes == {"stage": 0, "newton": 0} and upd == 0
    m.close()
