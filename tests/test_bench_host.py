"""Host-side arithmetic of the benchmark: the algorithmic flop counts behind the
roofline fraction.

The per-laminate and per-leaf counts are constants counted from the kernels'
arithmetic.  These tests pin what follows from them and from the tree's
structure: the per-pass totals of the full depth-8 tree (31,548 FP64 and
168,499 condensation flops) and of the benchmark's compressed tree (178
laminates), the structure of compressed trees against the oracle's own
compression, whose state holds 6 values per inelastic leaf and 3 per laminate,
and the roofline arithmetic of the JSON line (flops per launch, achieved rate,
derived FP64 peak, the mixed forms' F64/P64 + F32/P32 bound).
"""
import numpy as np

import bench
import oracle
from paper_2103_08253_gb300 import workloads as W


def test_full_tree_counts_and_flops_per_pass():
    for K in range(1, 9):
        L = 1 << K
        assert bench.tree_counts(np.ones(L)) == dict(N=L - 1, pairs=L // 2, inner=L // 2 - 1, single=0,
                                                     el=L // 2, j2=L // 2)
    # 255 x (39 + 44) + 128 x 13 + 128 x 68 + 15; 127 x (678 + 39) + 128 x (353 + 121): the bottom
    # laminates' elastic fiber leaves carry no rank-one tangent terms
    assert bench.pass_flops(8) == (31548, 151731)
    # the FP32 condensation of the mixed forms keeps the fiber's rank-one terms: 128 x (353 + 2 x 121)
    assert bench.pass_flops(8, t_is_f64=False) == (31548, 127 * 717 + 128 * 595)
    assert bench.corr_flops(8) == (255 * 3, 255 * 39)


def test_compressed_tree_structure_against_the_oracle():
    rng = np.random.default_rng(7)
    phases = (W.FIBER, W.MATRIX)
    for _ in range(300):
        K = int(rng.integers(1, 9))
        L = 1 << K
        w = rng.dirichlet(np.ones(L))
        w[rng.random(L) < rng.uniform(0.0, 0.9)] = 0.0
        if not (w > 0).any():
            w[rng.integers(L)] = 1.0
        c = bench.tree_counts(w)
        leaves = int((w > 0).sum())
        assert c["el"] + c["j2"] == leaves
        assert c["N"] == leaves - 1                      # a full binary tree over the remaining leaves
        assert c["pairs"] + c["inner"] == c["N"]
        if c["N"] > 0:                                   # each leaf hangs below one laminate
            assert 2 * c["pairs"] + c["single"] == leaves
        assert oracle.state_size(K, phases, w) == 6 * c["j2"] + 3 * c["N"], (K, w)


def test_benchmark_compressed_tree():
    tree = W.tree_with_zero_weights(bench.K_DEPTH, seed=bench.SEED_TREE)
    c = bench.tree_counts(tree.w)
    assert c["N"] == 178
    f64, ft = bench.pass_flops(bench.K_DEPTH, tree.w)
    assert round(f64 / 100) == 218 and round(ft / 100) == 1081     # 21.8 k + 108.1 k per pass


def test_roofline_arithmetic():
    """The FP64 line's roofline from its parts: flops per launch = (corrections + points) x flops per
    pass + corrections x flops per correction; achieved = flops / Newton time; the peak is
    152 SMs x 4 SMSPs x 0.5 DFMA per clock x 2 flops x 2.07 GHz.  With the figures of a 2^20-point run
    (3.6615 corrections per update, 1245.6 ms per launch) that is 9.370e11 flops and 0.598 of the peak."""
    n, steps = 1 << 20, 10
    iters = 3.661489200592041 * n * steps
    r = {"iters_sum": iters, "kms": {"newton": 1245.6054931640624 * steps, "final": 22.67 * steps}}
    line = bench.roofline_f64(r, n, steps)
    per_launch = ((iters / steps + n) * (31548 + 151731) + iters / steps * (255 * 3 + 255 * 39))
    assert abs(line["flops_per_launch"] - per_launch) <= 1e-9 * per_launch
    assert abs(line["flops_per_launch"] - 9.3697357e+11) <= 1e-6 * 9.3697357e+11
    peak = 152 * 4 * 0.5 * 2 * 2.07
    assert line["peak"] == peak and abs(line["frac"] - line["achieved"] / peak) <= 1e-12
    assert abs(line["achieved"] - per_launch / 1.2456054931640624 / 1e9) <= 1e-9 * line["achieved"]
    assert round(line["frac"], 3) == 0.598
    # the mixed forms: the Newton kernel against F64/P64 + F32/P32
    mx = bench.roofline_mixed(r, n, steps, sweep=True)
    f64 = (iters / steps + n) * 31548 + iters / steps * 255 * 3
    f32 = (iters / steps + n) * (127 * 717 + 128 * 595) + iters / steps * 255 * 39
    t_bound = f64 / (peak * 1e9) + f32 / (152 * 128 * 2 * 2.07 * 1e9)
    assert abs(mx["frac"] - t_bound / 1.2456054931640624) <= 1e-9 * mx["frac"]
    # with the all-FP32 first stage: the Newton kernel's corrections from its pass counter, the stage's
    # flops (every part of its passes in FP32) against the FP32 peak
    rs = dict(r, passes={"stage": int(3.4 * n * steps), "newton": int(2.4 * n * steps)},
              kms={"newton": 600.0 * steps, "stage": 80.0 * steps, "final": 22.67 * steps})
    ms = bench.roofline_mixed(rs, n, steps, sweep=True)
    cn = 1.4 * n
    f64 = (cn + n) * 31548 + cn * 255 * 3
    f32 = (cn + n) * (127 * 717 + 128 * 595) + cn * 255 * 39
    t_bound = f64 / (peak * 1e9) + f32 / (152 * 128 * 2 * 2.07 * 1e9)
    assert abs(ms["frac"] - t_bound / 0.6) <= 1e-6 * ms["frac"]
    assert abs(ms["passes_per_update"] - 2.4) <= 1e-9
    cs = 2.4 * n
    fs = (cs + n) * (31548 + 127 * 717 + 128 * 595) + cs * (255 * 3 + 255 * 39)
    st = ms["stage_kernel"]
    assert abs(st["flops_per_launch"] - fs) <= 1e-6 * fs
    assert st["peak"] == 152 * 128 * 2 * 2.07 and abs(st["achieved"] - fs / 0.08 / 1e9) <= 1e-6 * st["achieved"]
    assert bench.form_stage("mixed") and not bench.form_stage("mixed/no-stage")
    assert not bench.form_stage("f64") and not bench.form_stage("mixed/extrap")


def test_roofline_names_the_warp_kernel(monkeypatch):
    """A call that ran one warp per point is reported as k_newton_warp, with the same algorithmic flops,
    and looks up its own DRAM figure, never the thread kernel's."""
    keys = []
    monkeypatch.setattr(bench, "ncu_traffic", lambda k, n: keys.append(k))
    n, steps = 4096, 10
    r = {"iters_sum": 3.5 * n * steps, "kms": {"newton": 9.0 * steps, "final": 0.2 * steps}}
    thread = bench.roofline_f64(r, n, steps)
    warp = bench.roofline_f64(dict(r, warp=True), n, steps)
    assert thread["kernel"] == "k_newton<double>" and warp["kernel"] == "k_newton_warp<double>"
    assert warp["flops_per_launch"] == thread["flops_per_launch"]
    mw = bench.roofline_mixed(dict(r, warp=True), n, steps)
    assert mw["kernel"] == "k_newton_warp<float>"
    assert keys == ["k_newton_f64", "k_newton_warp_f64", "k_newton_warp_mixed"]


def test_form_options_and_l2_flush_rule():
    """Forms name the start, the first stage and the organisation; a step whose state fits twice into
    the L2 gets an L2 flush (depth 8: 1533 fields, so 4096 points do and 2^20 do not)."""
    assert bench.form_opts("f64/thread") == ("f64", False) and bench.form_warp_option("f64/thread") == (-1, 0)
    assert bench.form_warp_option("mixed") == (0, 0) and bench.form_stage_option("mixed") is None
    assert bench.form_warp_option("f64/w8") == (1, 8) and bench.form_warp_option("mixed/w16") == (1, 16)
    assert bench.form_stage_option("f64/stage") is True and bench.form_stage_option("mixed/no-stage") is False
    tree = W.tree_d10_fit(8, seed=0)
    S = bench.state_fields(tree)
    assert S == 1533
    assert bench.l2_flush_needed(S, 4096) and not bench.l2_flush_needed(S, 1 << 20)


def test_source_hash_ignores_comments_only():
    """The key of the committed DRAM figures changes with the code, not with comments or blank lines."""
    a = "int f(int x) {  // the square\n  return x * x;\n}\n"
    b = "/* squares */\nint f(int x) {\n\n  return x * x;   // as before\n}\n"
    c = "int f(int x) {\n  return x * x + 1;\n}\n"
    assert bench.code_only(a) == bench.code_only(b) != bench.code_only(c)
    assert len(bench.src_hash()) == 16
