"""The autotuner times candidate launch shapes through the C ABI and caches the fastest."""
import json

import numpy as np
import pytest
import torch

from paper_2103_08253_gb300 import autotune, dmn, workloads as W

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda:0")


def test_autotune_picks_a_candidate_and_caches_it(tmp_path, monkeypatch):
    monkeypatch.setattr(autotune, "CACHE", str(tmp_path / "autotune.json"))
    K, n = 5, 4096
    tree = W.tree_d10_fit(K, seed=3)
    A2, lam, Q = W.orientation_field(n, seed=4)
    Ef = W.random6_path_final(n, 0.03, seed=5)
    En, dE = W.proportional_increment(Ef, 10, 20)
    d = lambda x: torch.from_numpy(np.ascontiguousarray(x)).to(DEV)
    st = torch.zeros((W.state_size(K), n), dtype=torch.float64, device=DEV)
    cands = ((128, 2), (64, 4))
    res = autotune.tune(tree, "mixed", d(lam), d(Q), d(En), d(dE), st, reps=1, candidates=cands)
    assert (res["block"], res["ctas_per_sm"]) in cands
    assert len(res["table"]) == 2 and all(r["newton_ms"] > 0 for r in res["table"])
    assert autotune.cached(tree, "mixed", DEV) == (res["block"], res["ctas_per_sm"])
    data = json.load(open(autotune.CACHE))
    assert len(data) == 1
    # a tuned handle computes the same result as a default one, bit for bit (the launch shape is the
    # thread-per-point kernel's; at this size the default would take the warp kernel)
    a = dmn.DMN(tree, precision="f64", warp_per_point=-1).update(d(lam), d(Q), d(En), d(dE), st)
    b = dmn.DMN(tree, precision="f64", block=64, ctas_per_sm=6, warp_per_point=-1).update(d(lam), d(Q), d(En),
                                                                                         d(dE), st)
    for k in a:
        assert torch.equal(a[k], b[k]), k


def test_autotune_of_a_handle_with_several_trees(tmp_path, monkeypatch):
    """The mixed-depth batch (trees of depths 5 to 8 in one handle, points selected by tree_id):
    the tuner times the candidates on that handle and caches them under the handle's own key,
    apart from any single tree's."""
    monkeypatch.setattr(autotune, "CACHE", str(tmp_path / "autotune.json"))
    n = 8192
    depths = (5, 6, 7, 8)
    trees = [W.tree_d10_fit(K, seed=40 + K) for K in depths]
    tid, elastic = W.mixed_depth_batch(n, 41, depths)
    A2, lam, Q = W.orientation_field(n, seed=42)
    Ef = W.random6_path_final(n, 0.02, seed=43)
    En, dE = W.proportional_increment(Ef, 3, 10)
    d = lambda x: torch.from_numpy(np.ascontiguousarray(x)).to(DEV)
    m = dmn.DMN(trees)
    st = torch.zeros((m.state_size, n), dtype=torch.float64, device=DEV)
    m.close()
    cands = ((128, 2), (64, 6))
    res = autotune.tune(trees, "f64", d(lam), d(Q), d(En), d(dE), st, reps=1, candidates=cands, tree_id=d(tid))
    assert (res["block"], res["ctas_per_sm"]) in cands and len(res["table"]) == 2
    assert autotune.cached(trees, "f64", DEV) == (res["block"], res["ctas_per_sm"])
    assert autotune.cached(trees[0], "f64", DEV) is None


def test_stage_shape_tuner(tmp_path, monkeypatch):
    """The first stage's launch shape: the tuner times the candidates and picks one.  Each shape is its
    own instantiation (register cap), so the FP32 stage's rounding may differ between shapes; the FP64
    iteration then ends at the same criterion, and the results agree to that criterion's reach."""
    monkeypatch.setattr(autotune, "CACHE", str(tmp_path / "autotune.json"))
    K, n = 6, 3000
    tree = W.tree_d10_fit(K, seed=13)
    A2, lam, Q = W.orientation_field(n, seed=14)
    Ef = W.random6_path_final(n, 0.03, seed=15)
    En, dE = W.proportional_increment(Ef, 8, 20)
    d = lambda x: torch.from_numpy(np.ascontiguousarray(x)).to(DEV)
    st = torch.zeros((W.state_size(K), n), dtype=torch.float64, device=DEV)
    res = autotune.tune_stage(tree, "mixed-f32-tangent", d(lam), d(Q), d(En), d(dE), st, candidates=(2, 4, 8))
    assert res["stage_ctas_per_sm"] in (2, 4, 8)
    assert len(res["table"]) == 3 and all(r["stage_ms"] > 0 for r in res["table"])
    outs = [dmn.DMN(tree, precision="mixed", stage_ctas_per_sm=c).update(d(lam), d(Q), d(En), d(dE), st)
            for c in (2, 8)]
    assert torch.equal(outs[0]["status"], outs[1]["status"])
    ok = (outs[0]["status"] == 0).cpu().numpy()
    assert ok.mean() > 0.9      # one increment to 40 % of the path from the virgin state: a few points end at MAXITER
    for k in ("stress", "tangent"):
        a, b = (o[k].reshape(n, -1).cpu().numpy()[ok] for o in outs)
        assert (np.linalg.norm(a - b, axis=1) / np.linalg.norm(b, axis=1)).max() <= 1e-8, k
