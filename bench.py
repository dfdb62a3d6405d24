#!/usr/bin/env python
"""DMN Gauss-point updates/s at depth 8 on one GB300, FP64 and mixed forms.

The JSON line's value is the FP64 form; next to it, value_mixed and
value_mixed_f32_tangent give the mixed form (FP32 condensation, FP64 residual
and final sweep) and the mixed form with an FP32 tangent (no final sweep), each
with its roofline and its error against the oracle (roofline_*, parity_*);
"forms" holds every form's full record.  The rooflines divide by the FMA peaks
measured on the same GPU at the start of the run (dmn_peak_gflops, "peaks").

Workload (one "step" = one increment of the load path over the whole batch:
orientation set-up + material-point update, all through the C ABI):
  * K = 8 DMN (256 leaves, 255 laminates), linear angle interpolation fitted to
    seeded angles at the ten D10 points of the orientation triangle,
    Dirichlet(1) leaf weights; glass fiber (E 72 GPa, nu 0.22) and a J2 matrix
    (E 3 GPa, nu 0.35, sigma0 40 MPa, H 300 MPa);
  * 2^20 Gauss points per GPU whose orientation eigenvalues are uniform over
    the triangle, Haar-random principal frames;
  * random proportional 6-component macro strain paths reaching 3 %
    equivalent strain after 50 increments; step s of the run is increment s.
The state (12.9 GB per buffer at 2^20 points) is far larger than L2, so no
flush is needed between steps.

Prints one JSON line (rank 0).  ``--impl reference`` times the CPU oracle on a
bounded sample of the same workload instead.

The oracle runs only in the CPU-baseline leg (N = 1): timed on a bounded sample
(``cpu_baseline``) and, untimed, on --parity-points sampled points of the timed
batch, whose results it compares with the GPU's (each form's
``parity_vs_oracle``).  No result of the GPU path comes from it.
"""
from __future__ import annotations

import argparse
import hashlib
import re
import json
import os
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from paper_2103_08253_gb300 import workloads as W  # noqa: E402

METRIC = "DMN Gauss-point updates/s at depth 8 on 1 GB300 (FP64 vs mixed) at stated stress error"
UNIT = "GP-updates/s"
K_DEPTH = 8
N_INCREMENTS = 50
EPS_EQ = 0.03
SEED_TREE, SEED_ORI, SEED_PATH = 2103, 8253, 1208
WORKLOAD = "K=8 D10-interpolated DMN, 2^20 points/GPU, random 6-comp paths, 50 increments to 3% eq. strain"
SHAPE_NOTE = {3: "linear (M = 3), coefficients fitted at the D10 points", 4: "tri-linear (M = 4), seeded nodal angles",
              6: "quadratic (M = 6), seeded nodal angles"}
MATRIX_NOTE = {"linear": "J2, linear hardening 40 + 300 a MPa (E 3 GPa, nu 0.35)",
               "explin": "J2, exponential-linear hardening of the paper's polyamide (E 2.1 GPa, nu 0.3, s0 29, "
                         "s_inf 61.7 MPa, k0 10.6 GPa, k_inf 139 MPa); flop counts exclude its scalar Newton"}
WORKLOAD_CMP = ("K=8 D10-interpolated DMN compressed to 70% of its leaves (weights of zero, 178 of 255 laminates "
                "left), 2^20 points/GPU, random 6-comp paths, 50 increments to 3% eq. strain")

# FP64 peak: 152 SMs x 4 sub-partitions x 0.5 DFMA/clk x 2 flop x 2.07 GHz
PEAK_F64_GFLOPS = 152 * 4 * 0.5 * 2 * 2.07
# FP32 peak: 152 SMs x 128 FFMA/clk x 2 flop x 2.07 GHz
PEAK_F32_GFLOPS = 152 * 128 * 2 * 2.07
# The rooflines use the peaks measured on the GPU at the start of the run (dmn_peak_gflops: a sustained
# FMA loop on every SM); the derived figures above are kept beside them as a cross-check.
PEAKS_DERIVED = {"f64": PEAK_F64_GFLOPS, "f32": PEAK_F32_GFLOPS,
                 "note": "derived: 152 SM x 4 SMSP x 0.5 DFMA/clk x 2 flop x 2.07 GHz (FP64); "
                         "152 SM x 128 FFMA/clk x 2 flop x 2.07 GHz (FP32)"}


def measure_peaks(seconds_f64=1.0, seconds_f32=0.3):
    """Sustained FP64 and FP32 FMA throughput of this GPU through the library's own kernel."""
    from paper_2103_08253_gb300 import dmn
    g64, ms64 = dmn.peak_gflops("fp64", seconds_f64)
    g32, ms32 = dmn.peak_gflops("fp32", seconds_f32)
    return {"f64": g64, "f32": g32,
            "note": "measured: dmn_peak_gflops, sustained FMA loop on every SM (%.2f s FP64, %.2f s FP32); "
                    "derived cross-check %.1f / %.1f GFLOP/s" % (ms64 * 1e-3, ms32 * 1e-3, PEAK_F64_GFLOPS,
                                                                PEAK_F32_GFLOPS)}

# ---------------------------------------------------------------------------------------------
# Algorithmic flop counts (add/sub/mul/div/sqrt/rsqrt = 1, fma = 2) of the tree-condensed Newton
# method, counted from the arithmetic of csrc/dmn_device.cuh.  T = FP64 in the FP64 form, FP32
# in the mixed form.
#   per laminate, every pass:  N a and the children's strains 39 (FP64); residual share and
#                              plain stress average 44 (FP64); condensation 678 (T), or, for a bottom
#                              laminate (leaf tangents D = lam 1(x)1 + 2 mu I - c m(x)m), 353 (T) plus
#                              121 (T) for each leaf of an inelastic phase (an elastic leaf has c = 0
#                              in every pass and the FP64 condensation skips its rank-one terms; the
#                              FP32 one computes them)
#   per inner laminate:        children's strain corrections 39 (T)
#   per laminate, per Newton correction: da = g + H d_eps 39 (T), a += da 3 (FP64)
#   per leaf:                  elastic stress 13; J2 stress 56 + tangent scalars 12 (FP64)
#   per pass:                  convergence test 15 (FP64)
F_NODE_F64, F_RES, F_COND, F_COND_BOTTOM, F_COND_LEAF, F_DEPS, F_DA, F_A = 39, 44, 678, 353, 121, 39, 39, 3
F_LEAF_EL, F_LEAF_J2, F_TEST = 13, 56 + 12, 15
F_ROTATE = 1150         # per point: stress and tangent back to the global frame (k_final)
F_STATE_NODE = 39       # state pass: per laminate (strains from the jumps)
F_STATE_J2 = 68         # state pass: per J2 leaf (return mapping and new state)


F_LEAF_SUB = 84         # a leaf whose sibling is a laminate: its 21 tangent entries as a subtree (T)


def tree_counts(w):
    """Laminates and leaves of the tree with leaf weights w after compression (leaves of weight
    zero removed, laminates with one weightless side passed through): dict(N = laminates,
    pairs = laminates whose children are two leaves, inner = the other laminates, single =
    leaves whose sibling is a laminate, el / j2 = remaining fiber (odd) / matrix (even) leaves)."""
    w = np.asarray(w, dtype=np.float64)
    L = w.size
    Wh = np.zeros(2 * L)
    Wh[L:] = w
    for h in range(L - 1, 0, -1):
        Wh[h] = Wh[2 * h] + Wh[2 * h + 1]

    def kind(h):        # 'leaf', 'lam' or None after compression
        if Wh[h] <= 0:
            return None
        if h >= L:
            return "leaf"
        if Wh[2 * h] > 0 and Wh[2 * h + 1] > 0:
            return "lam"
        return kind(2 * h if Wh[2 * h] > 0 else 2 * h + 1)

    def child(h):       # the compressed node standing for heap node h
        while h < L and not (Wh[2 * h] > 0 and Wh[2 * h + 1] > 0):
            h = 2 * h if Wh[2 * h] > 0 else 2 * h + 1
        return h

    c = dict(N=0, pairs=0, inner=0, single=0, el=int((w[0::2] > 0).sum()), j2=int((w[1::2] > 0).sum()))
    for h in range(1, L):
        if not (Wh[2 * h] > 0 and Wh[2 * h + 1] > 0):
            continue
        c["N"] += 1
        kl, kr = kind(child(2 * h)), kind(child(2 * h + 1))
        if kl == "leaf" and kr == "leaf":
            c["pairs"] += 1
        else:
            c["inner"] += 1
            c["single"] += (kl == "leaf") + (kr == "leaf")
    return c


def pass_flops(K, w=None, t_is_f64=True):
    """(FP64 flops, T flops) of one Newton pass without the jump correction (w: leaf weights of
    a compressed tree; None: the full tree).  Phases of the benchmark: an elastic fiber on the
    left leaf of every laminate pair, a J2 matrix on the right one.  The FP64 condensation skips
    the fiber's rank-one terms; the FP32 one (t_is_f64 False) computes them (with c = 0)."""
    c = tree_counts(np.ones(1 << K) if w is None else w)
    f64 = c["N"] * (F_NODE_F64 + F_RES) + c["el"] * F_LEAF_EL + c["j2"] * F_LEAF_J2 + F_TEST
    ft = (c["inner"] * (F_COND + F_DEPS) + c["pairs"] * (F_COND_BOTTOM + (1 if t_is_f64 else 2) * F_COND_LEAF)
          + c["single"] * F_LEAF_SUB)
    return f64, ft


def corr_flops(K, w=None):
    """(FP64 flops, T flops) of one jump correction of all laminates."""
    N = tree_counts(np.ones(1 << K) if w is None else w)["N"]
    return N * F_A, N * F_DA


def newton_flops(K, iters_sum, npts, mixed, w=None):
    """(FP64, FP32) flops of the Newton kernel over npts points with iters_sum corrections:
    one pass per point evaluates the starting jumps, one more per correction."""
    f64, ft = pass_flops(K, w, t_is_f64=not mixed)
    c64, ct = corr_flops(K, w)
    passes = iters_sum + npts
    F64 = passes * f64 + iters_sum * c64
    FT = passes * ft + iters_sum * ct
    return (F64, FT) if mixed else (F64 + FT, 0.0)


def final_flops(K, npts, sweep, w=None):
    """FP64 flops of the final kernel (state pass and rotation; mixed form: plus one FP64 pass)."""
    c = tree_counts(np.ones(1 << K) if w is None else w)
    f = npts * (F_ROTATE + c["N"] * F_STATE_NODE + c["j2"] * F_STATE_J2)
    if sweep:
        f64, ft = pass_flops(K, w)
        f += npts * (f64 + ft)
    return f


# ---------------------------------------------------------------------------------------------
SRC_FILES = ("paper_2103_08253_gb300/csrc/dmn.cu", "paper_2103_08253_gb300/csrc/dmn_device.cuh",
             "paper_2103_08253_gb300/csrc/dmn_warp.cu", "paper_2103_08253_gb300/csrc/dmn_launch.cuh")


def code_only(text):
    """A CUDA source without its comments and blank lines, each line stripped: what a change must touch
    for the compiled kernels (and so their DRAM figures) to change."""
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    lines = (re.sub(r"//.*", "", line).strip() for line in text.split("\n"))
    return "\n".join(line for line in lines if line)


def src_hash():
    """Hash of the DMN kernels' sources, comments and layout left out (the key of profiles/traffic.json)."""
    h = hashlib.sha256()
    for f in SRC_FILES:
        h.update(code_only(open(os.path.join(ROOT, f)).read()).encode())
    return h.hexdigest()[:16]


def ncu_traffic(kernel, npts_launch):
    """DRAM bytes per launch from a committed ncu summary of the same sources: the capture of this
    batch size ("kernel@points") if there is one, else the kernel's (scaled by points)."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        d = json.load(open(path))
    except (OSError, ValueError):
        return None
    e = d.get("%s@%d" % (kernel, npts_launch)) or d.get(kernel)
    if not e or e.get("src_hash") != src_hash():
        return None
    return e["dram_bytes_per_point"] * npts_launch


class ClockSampler:
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_id):
        self.proc = None
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(gpu_id), "--query-gpu=" + self.FIELDS,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
            out, _ = self.proc.communicate()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in out.strip().splitlines():
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 7:
                continue
            try:
                sm.append(float(f[0]))
                smax.append(float(f[1]))
            except ValueError:
                continue
            for nm, v in zip(names, f[3:7]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ---------------------------------------------------------------------------------------------
def max_over_ranks(t_ms, dist, device):
    """The largest of the ranks' times (all ranks get it); t_ms itself without a process group."""
    if not dist:
        return t_ms
    import torch
    t = torch.tensor([float(t_ms)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_value(world, n, steps, t_ms):
    """Whole-job throughput: the units all ranks processed over the slowest rank's time."""
    return world * n * steps / (t_ms * 1e-3)


def make_workload(n, rank, compressed=False, matrix="linear", shape=3):
    phases = (W.FIBER, W.MATRIX_EXPLIN if matrix == "explin" else W.MATRIX)
    if compressed:
        tree = W.tree_with_zero_weights(K_DEPTH, seed=SEED_TREE, phases=phases)
    elif shape != 3:
        tree = W.tree_nodal_angles(K_DEPTH, shape, seed=SEED_TREE, phases=phases)
    else:
        tree = W.tree_d10_fit(K_DEPTH, seed=SEED_TREE, phases=phases)
    A2, lam, Q = W.orientation_field(n, seed=SEED_ORI + 1000 * rank)
    Ef = W.random6_path_final(n, EPS_EQ, seed=SEED_PATH + 1000 * rank)
    return tree, A2, lam, Q, Ef


def oracle_baseline(tree, A2, Ef, idx, warmup, steps, threads):
    """Time the oracle (as it stands) on the points idx over increments warmup+1..warmup+steps."""
    import oracle
    A2s = A2[idx]
    lam, Q = oracle.interp_orientation(A2s)
    S = oracle.state_size(tree.K, tree.phases, tree.w)
    st = np.zeros((S, len(idx)))
    for s in range(1, warmup + 1):
        En, dE = W.proportional_increment(Ef[idx], s, N_INCREMENTS)
        st = oracle.update(tree, lam, Q, En, dE, st, nthreads=threads)[0]
    t0 = time.perf_counter()
    for s in range(warmup + 1, warmup + steps + 1):
        lam, Q = oracle.interp_orientation(A2s)
        En, dE = W.proportional_increment(Ef[idx], s, N_INCREMENTS)
        st = oracle.update(tree, lam, Q, En, dE, st, nthreads=threads)[0]
    return time.perf_counter() - t0


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    tree, A2, lam, Q, Ef = make_workload(args.points, 0, args.workload == "k8-compressed", args.matrix, args.shape)
    cores = os.cpu_count() or 1
    m = args.ref_points
    idx = np.arange(m)
    t = oracle_baseline(tree, A2, Ef, idx, args.warmup, args.steps, cores)
    v = m * args.steps / t
    line = {"metric": METRIC, "value": v, "unit": UNIT, "impl": "reference", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * t / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD_CMP if args.workload == "k8-compressed" else WORKLOAD, "K": K_DEPTH,
                       "points_per_step": m,
                       "increments": [args.warmup + 1, args.warmup + args.steps]},
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": "first %d points of the workload, increments %d..%d (after %d untimed)"
                                       % (m, args.warmup + 1, args.warmup + args.steps, args.warmup)},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def rel_rows(a, b):
    a = a.reshape(a.shape[0], -1)
    b = b.reshape(b.shape[0], -1)
    return np.linalg.norm(a - b, axis=1) / np.maximum(np.linalg.norm(b, axis=1), 1e-300)


def form_opts(form):
    """(precision, extrapolated start) of a form name such as "f64", "mixed-f32-tangent/extrap",
    "mixed/no-stage" (the mixed iteration without its all-FP32 first stage), "f64/stage" (the FP64
    iteration after that stage), "f64/thread" (one point per thread whatever the batch size) or
    "f64/w8" (the warp organisation with 8, 16 or 32 lanes per point whatever the batch size)."""
    prec, _, start = form.partition("/")
    if start not in ("", "extrap", "no-stage", "stage", "thread", "w8", "w16", "w32"):
        raise ValueError("unknown start in form %r" % form)
    return prec, start == "extrap"


def form_stage(form):
    """Whether the form runs the all-FP32 first stage (the mixed forms' default; "/stage" in the FP64 form)."""
    prec, pred = form_opts(form)
    if pred or form.endswith("/no-stage"):
        return False
    return prec != "f64" or form.endswith("/stage")


def form_stage_option(form):
    """The handle's first_stage argument for the form: explicit only where the form names it ("/stage",
    "/no-stage"), else the library default (on in the mixed forms; a small call, which runs one warp
    per point, goes without it)."""
    return True if form.endswith("/stage") else False if form.endswith("/no-stage") else None


L2_BYTES = 126 << 20


def state_fields(tree):
    """Doubles of state per point (leaf states of the inelastic leaves, jumps) of a tree's handle."""
    c = tree_counts(tree.w)
    return 6 * c["j2"] + 3 * c["N"]


def l2_flush_needed(S, n):
    """Whether one step's state (read and written) and strains fit twice into the L2."""
    return 8 * n * (2 * S + 12 + 11) < 2 * L2_BYTES


def form_warp_option(form):
    """The handle's (warp_per_point, warp_lanes) arguments: (-1, 0) for "/thread", (1, lanes) for "/w8",
    "/w16", "/w32", else the library default (the warp organisation for small calls, its lanes by size)."""
    start = form.partition("/")[2]
    if start == "thread":
        return -1, 0
    if start in ("w8", "w16", "w32"):
        return 1, int(start[1:])
    return 0, 0


def tune_shape(form, ctx, args):
    """Launch shape of the Newton kernel from the autotuner, tuned on the first 2^18 points at the
    first timed increment (after the warm-up increments).  Forms that differ only in the start
    share the kernel and its shape."""
    import torch
    from paper_2103_08253_gb300 import autotune, dmn
    form, _ = form_opts(form)
    cache = ctx.setdefault("shapes", {})
    if form in cache:
        return cache[form]
    dev = ctx["dev"]
    m = min(ctx["n"], 1 << 18)
    A2 = ctx["A2"][:m].contiguous()
    h = dmn.DMN(ctx["tree"], precision=form)
    lam, Q = h.interp_orientation(A2)
    st = torch.zeros((h.state_size, m), dtype=torch.float64, device=dev)
    for s in range(1, args.warmup + 1):
        st = h.update(lam, Q, ctx["En"][s - 1][:m].contiguous(), ctx["dE"][s - 1][:m].contiguous(), st)["state_out"]
    h.close()
    s = args.warmup + 1
    res = autotune.tune(ctx["tree"], form, lam, Q, ctx["En"][s - 1][:m].contiguous(),
                        ctx["dE"][s - 1][:m].contiguous(), st, reps=1)
    # the first stage's own launch shape, at the Newton kernel's tuned one
    ts = autotune.tune_stage(ctx["tree"], form, lam, Q, ctx["En"][s - 1][:m].contiguous(),
                             ctx["dE"][s - 1][:m].contiguous(), st, block=res["block"], ctas_per_sm=res["ctas_per_sm"])
    res["stage_ctas_per_sm"], res["stage_table"] = ts["stage_ctas_per_sm"], ts["table"]
    del st
    torch.cuda.empty_cache()
    cache[form] = res
    return res


def run_form(form, ctx, args, dist):
    """Warm-up increments, then the timed increments; returns timings and the last outputs."""
    import torch
    from paper_2103_08253_gb300 import dmn
    dev, n = ctx["dev"], ctx["n"]
    shape = tune_shape(form, ctx, args) if args.autotune else None
    prec, pred = form_opts(form)
    m = dmn.DMN(ctx["tree"], precision=prec, block=shape["block"] if shape else 0,
                ctas_per_sm=shape["ctas_per_sm"] if shape else 0, predictor=pred,
                first_stage=form_stage_option(form), warp_per_point=form_warp_option(form)[0],
                warp_lanes=form_warp_option(form)[1],
                stage_ctas_per_sm=shape["stage_ctas_per_sm"] if shape else 0)
    assert m.first_stage == form_stage(form)
    S = m.state_size
    st = [torch.zeros((S, n), dtype=torch.float64, device=dev), torch.zeros((S, n), dtype=torch.float64, device=dev)]
    lam = torch.empty((n, 2), dtype=torch.float64, device=dev)
    Q = torch.empty((n, 9), dtype=torch.float64, device=dev)
    out = m.alloc_outputs(n, dev)
    iters_steps = torch.zeros((args.steps, n), dtype=torch.int32, device=dev)
    cur = 0
    # a step's inputs and state smaller than twice the L2: overwrite the L2 (a 256 MB fill) before
    # every step, inside the timed region (about 0.05 ms a step)
    flush = torch.empty(1 << 25, dtype=torch.float64, device=dev) if l2_flush_needed(S, n) else None

    def step(s, cur, iters_buf=None):
        if flush is not None:
            flush.fill_(float(s))
        m.interp_orientation(ctx["A2"], lam, Q)
        out["state_out"] = st[1 - cur]
        if iters_buf is not None:
            out["iters"] = iters_buf
        m.update(lam, Q, ctx["En"][s - 1], ctx["dE"][s - 1], st[cur], out=out)
        return 1 - cur

    for s in range(1, args.warmup + 1):
        cur = step(s, cur)
    torch.cuda.synchronize()
    host_state = None
    if form == "f64" and args.e2e_steps != 0:
        # the host state an application would hold: written by the CPU, then pinned (a copy-engine
        # write into freshly pinned pages gave a 4x slower host-to-device rate on the box)
        host_state = st[cur].cpu().pin_memory()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    clocks = ClockSampler(ctx["smi_id"]) if ctx["rank"] == 0 else None
    m.profile(True)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for j, s in enumerate(range(args.warmup + 1, args.warmup + args.steps + 1)):
        cur = step(s, cur, iters_steps[j])
    e1.record()
    torch.cuda.synchronize()
    t_ms = max_over_ranks(e0.elapsed_time(e1), dist, dev)
    if dist:
        dist.barrier()
    clk = clocks.stop() if clocks else None
    kms, passes, cnt = m.profile_read_stages()
    m.profile(False)
    lanes = m.lanes_per_point(n)   # a small call runs the warp organisation, without the first stage
    warp = lanes > 1
    if not form_stage(form) or warp:
        kms.pop("stage")
    its = iters_steps.to(torch.int64).sum().item()
    hist = torch.bincount(iters_steps.reshape(-1).to(torch.int64), minlength=1).cpu().numpy()
    res = dict(t_ms=t_ms, kms=kms, updates=cnt, clocks=clk, iters_sum=int(its), iters_hist=hist.tolist(),
               passes=passes, warp=warp,
               launch=("%d lanes per point (k_newton_warp, 2 CTAs of 4 warps per SM)" % lanes if warp else
                       dict(block=shape["block"], ctas_per_sm=shape["ctas_per_sm"], tuned_on_points=shape["points"],
                            table=shape["table"], stage_ctas_per_sm=shape["stage_ctas_per_sm"],
                            stage_table=shape["stage_table"]) if shape else "defaults"),
               stress=out["stress"], tangent=out["tangent"], status=out["status"], state=st[cur],
               host_state=host_state, m=m, lam=lam, Q=Q, S=S, st=st)
    return res


def parity_sample(form, r, ctx, args, pidx):
    """CPU-baseline leg, untimed part: the oracle on the sampled points through increments
    1..warmup+steps, compared with the GPU's results there (the form's error statement)."""
    import oracle
    tree, A2, Ef = ctx["tree"], ctx["A2_np"], ctx["Ef_np"]
    _, pred = form_opts(form)
    cache = ctx.setdefault("oracle_runs", {})   # the oracle's results depend only on the start
    if pred not in cache:
        lam, Q = oracle.interp_orientation(A2[pidx])
        S0, J = oracle.jump_fields(tree)
        st = np.zeros((S0 + J + 6 if pred else S0, len(pidx)))
        for s in range(1, args.warmup + args.steps + 1):
            En, dE = W.proportional_increment(Ef[pidx], s, N_INCREMENTS)
            st, sig, C, it, stat, gap = oracle.update(tree, lam, Q, En, dE, st, predictor=pred)
        cache[pred] = (st, sig, C, stat, gap)
    st, sig, C, stat, gap = cache[pred]
    sig_g = r["stress"][pidx].cpu().numpy()
    C_g = r["tangent"][pidx].cpu().numpy()
    st_g = r["state"][:, pidx].cpu().numpy()
    ok = (stat == 0) & (r["status"][pidx].cpu().numpy() == 0)
    tie = ok & (gap < 1e-9)    # yield decision within rounding: the tangent may take either branch
    scale = np.abs(st).max(axis=1, keepdims=True) + 1e-300
    return {"points": int(len(pidx)), "max_rel_stress": float(rel_rows(sig_g[ok], sig[ok]).max(initial=0)),
            "max_rel_tangent": float(rel_rows(C_g[ok & ~tie], C[ok & ~tie]).max(initial=0)),
            "tangent_ties_excluded": int(tie.sum()),
            "max_rel_state": float((np.abs(st_g - st) / scale).max()), "status_ok": int(ok.sum())}


def run_e2e(r, ctx, args, dist):
    """Same increments through the public API with host buffers (dmn_update_host, FP64 form): every
    step copies its inputs (orientation, strains, state) from pinned host memory and its results
    (stress, tangent, iterations, status, state) back; the chunked pipeline of the library overlaps
    those copies with the updates.  Wall-clock time of the blocking calls."""
    import torch
    n, S = ctx["n"], r["S"]
    m = r["m"]
    steps = args.steps if args.e2e_steps < 0 else min(args.e2e_steps, args.steps)
    lam_h = r["lam"].cpu().pin_memory()
    Q_h = r["Q"].cpu().pin_memory()
    En_h = [ctx["En"][s - 1].cpu().pin_memory() for s in range(args.warmup + 1, args.warmup + steps + 1)]
    dE_h = [ctx["dE"][s - 1].cpu().pin_memory() for s in range(args.warmup + 1, args.warmup + steps + 1)]
    st_h = r["host_state"]                        # state after the warm-up increments, updated in place
    out_h = m.alloc_host_outputs(n)
    # untimed call (its own state_out): allocates the library's stage buffers and second work set
    m.update_host(lam_h, Q_h, En_h[0], dE_h[0], st_h, out=out_h, chunk=args.e2e_chunk)
    out_h["state_out"] = st_h
    # copy bandwidth of this process's pinned state buffer (up to 1 GiB each way), for the record;
    # the device-to-host copy writes back the bytes the host-to-device copy just read
    cnt = min(1 << 27, st_h.numel())
    probe = torch.empty(cnt, dtype=torch.float64, device=ctx["dev"])
    flat = st_h.view(-1)[:cnt]
    bw = {}
    for name, dst, src in (("h2d_GBps", probe, flat), ("d2h_GBps", flat, probe)):
        torch.cuda.synchronize()
        c0 = time.perf_counter()
        dst.copy_(src, non_blocking=True)
        torch.cuda.synchronize()
        bw[name] = round(8 * cnt / (time.perf_counter() - c0) / 1e9, 1)
    del probe
    h2d = lam_h.nbytes + Q_h.nbytes + En_h[0].nbytes + dE_h[0].nbytes + st_h.nbytes
    d2h = (out_h["stress"].nbytes + out_h["tangent"].nbytes + st_h.nbytes + out_h["iters"].nbytes
           + out_h["status"].nbytes)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    t0 = time.perf_counter()
    for j in range(steps):
        m.update_host(lam_h, Q_h, En_h[j], dE_h[j], st_h, out=out_h, chunk=args.e2e_chunk)
    t_ms = max_over_ranks(1e3 * (time.perf_counter() - t0), dist, ctx["dev"])
    world = dist.get_world_size() if dist else 1
    return {"value": job_value(world, n, steps, t_ms), "unit": UNIT, "h2d_bytes_per_step": int(h2d),
            "d2h_bytes_per_step": int(d2h), "steps": steps, "form": "f64", "ms_per_step": t_ms / steps,
            "api": "dmn_update_host", "chunk": args.e2e_chunk or "default", "pinned_copy": bw,
            "status_ok": int((out_h["status"] == 0).sum().item())}


def stage_roofline(r, n, steps, w, P32):
    """The all-FP32 first stage against the FP32 peak, from its pass counter and event time."""
    npts = n * steps
    Fs = stage_flops(K_DEPTH, r["passes"]["stage"], npts, w=w)
    ts = r["kms"]["stage"] * 1e-3
    return {"kernel": "k_stage32", "achieved": Fs / ts / 1e9, "peak": P32, "unit": "GFLOP/s (FP32)",
            "frac": Fs / ts / 1e9 / P32, "flops_per_launch": Fs / steps, "launch_ms": r["kms"]["stage"] / steps,
            "passes_per_update": r["passes"]["stage"] / npts}


def roofline_f64(r, n, steps, w=None, peaks=None):
    pk = peaks or PEAKS_DERIVED
    P64 = pk["f64"]
    npts = n * steps
    passes = r.get("passes") or {}
    corr = passes["newton"] - npts if passes.get("newton") else r["iters_sum"]
    F, _ = newton_flops(K_DEPTH, corr, npts, mixed=False, w=w)
    t = r["kms"]["newton"] * 1e-3
    ach = F / t / 1e9
    cmp = "_compressed" if w is not None and (np.asarray(w) == 0).any() else ""
    org = "_warp" if r.get("warp") else ""
    tr = ncu_traffic("k_newton" + org + "_f64" + cmp + ("_stage" if "stage" in r["kms"] else ""), n)
    out = {"bound": "alu", "kernel": "k_newton_warp<double>" if org else "k_newton<double>", "achieved": ach,
           "peak": P64,
           "unit": "GFLOP/s (FP64)", "frac": ach / P64, "traffic": tr,
           "flops_per_launch": F / steps, "launch_ms": r["kms"]["newton"] / steps,
           "frac_of_derived_peak": ach / PEAK_F64_GFLOPS, "peak_note": pk["note"],
           "passes_per_update": (corr + npts) / npts}
    if "stage" in r["kms"]:
        out["stage_kernel"] = stage_roofline(r, n, steps, w, pk["f32"])
        out["stage_kernel"]["traffic"] = ncu_traffic("k_stage32" + cmp, n)
    return out


def stage_flops(K, passes, npts, w=None):
    """FP32 flops of the all-FP32 first stage over npts points and `passes` tree passes: the Newton
    pass's FP64 and FP32 parts, and the jump corrections, all in FP32."""
    f64, ft = pass_flops(K, w, t_is_f64=False)
    c64, ct = corr_flops(K, w)
    corr = passes - npts
    return passes * (f64 + ft) + corr * (c64 + ct)


def roofline_mixed(r, n, steps, w=None, sweep=True, peaks=None):
    """Mixed forms: the Newton kernel against F64/P64 + F32/P32; the first stage (all FP32) against the
    FP32 peak; the final kernel (with the FP64 sweep, or only the state pass and rotation in the form
    with an FP32 tangent) against the FP64 peak.  Pass counts come from the kernels' counters."""
    pk = peaks or PEAKS_DERIVED
    P64, P32 = pk["f64"], pk["f32"]
    npts = n * steps
    passes = r.get("passes") or {}
    newton_corr = passes["newton"] - npts if passes.get("newton") else r["iters_sum"]
    F64, F32 = newton_flops(K_DEPTH, newton_corr, npts, mixed=True, w=w)
    t = r["kms"]["newton"] * 1e-3
    tb = F64 / (P64 * 1e9) + F32 / (P32 * 1e9)
    Ff = final_flops(K_DEPTH, n * steps, sweep=sweep, w=w)
    tf = r["kms"]["final"] * 1e-3
    fin = {"kernel": "k_final<sweep>" if sweep else "k_final", "achieved": Ff / tf / 1e9, "peak": P64,
           "unit": "GFLOP/s (FP64)", "frac": Ff / tf / 1e9 / P64, "launch_ms": r["kms"]["final"] / steps}
    cmp = "_compressed" if w is not None and (np.asarray(w) == 0).any() else ""
    stg = "stage" in r["kms"]
    org = "_warp" if r.get("warp") else ""
    out = {"bound": "alu", "kernel": "k_newton_warp<float>" if org else "k_newton<float>", "achieved": tb / t * P64,
           "peak": P64, "unit": "GFLOP/s (FP64-equivalent: F64/P64 + F32/P32)", "frac": tb / t, "peak_note": pk["note"],
           "traffic": ncu_traffic("k_newton" + org + "_mixed" + cmp + ("_stage" if stg else ""), n),
           "flops_f64_per_launch": F64 / steps,
           "flops_f32_per_launch": F32 / steps, "launch_ms": r["kms"]["newton"] / steps,
           "passes_per_update": (newton_corr + npts) / npts, "final_kernel": fin}
    if stg:
        out["stage_kernel"] = stage_roofline(r, n, steps, w, P32)
        out["stage_kernel"]["traffic"] = ncu_traffic("k_stage32" + cmp, n)
    return out


# ---------------------------------------------------------------------------------------------
# Mixed-depth batch: 4M points, depths 5/6/7/8 (25 % each), half loaded in the elastic range
# (proportional ramp to 0.1 % equivalent strain), half cyclic +-2 % (one triangle period over
# 40 increments), shuffled; one persistent launch per increment, a CUDA graph over a block of
# increments, autotuned launch shape.  A secondary measurement (not the headline line).
MD_DEPTHS = (5, 6, 7, 8)
MD_INCREMENTS = 40


def run_mixed_depth(args):
    import torch
    from paper_2103_08253_gb300 import autotune, dmn
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    n = args.points
    trees = [W.tree_d10_fit(K, seed=SEED_TREE + K) for K in MD_DEPTHS]
    tid, elastic = W.mixed_depth_batch(n, SEED_ORI + 7, MD_DEPTHS)
    A2, lam_np, Q_np = W.orientation_field(n, seed=SEED_ORI + 8)
    Edir = W.random6_path_final(n, 1.0, seed=SEED_PATH + 9)
    amp = np.where(elastic, 0.001, 0.02)[:, None] * Edir
    G = args.steps                      # increments per graph replay
    first = args.warmup + 1
    inc = list(range(first, first + G))

    def inputs(k):
        En_c, dE_c = W.cyclic_increment(amp, k, MD_INCREMENTS)
        En_r, dE_r = W.proportional_increment(amp, k, MD_INCREMENTS)
        e = elastic[:, None]
        return (torch.from_numpy(np.where(e, En_r, En_c)).to(dev), torch.from_numpy(np.where(e, dE_r, dE_c)).to(dev))

    A2_d, tid_d = torch.from_numpy(A2).to(dev), torch.from_numpy(tid).to(dev)
    line = {"metric": "DMN Gauss-point updates/s, mixed depths 5-8, cyclic + elastic-range batch", "unit": UNIT,
            "n_gpus": 1, "steps": G, "warmup": args.warmup, "higher_is_better": True, "data": "synthetic",
            "config": {"workload": "4M points, depths 5/6/7/8 x 25%%, half elastic-range 0.1%%, half cyclic +-2%% over "
                                   "%d increments, shuffled" % MD_INCREMENTS, "points": n,
                       "timed_increments": [inc[0], inc[-1]], "graph": "one CUDA graph of %d increments" % G},
            "forms": {}}
    for form in [f for f in args.forms.split(",") if f]:
        # autotuned shape on 2^18 points of the batch at the first timed increment
        prec, pred = form_opts(form)
        stage = form_stage_option(form)
        m0 = dmn.DMN(trees, precision=prec, first_stage=stage)
        msub = min(n, 1 << 18)
        lam_s, Q_s = m0.interp_orientation(A2_d[:msub].contiguous())
        st = torch.zeros((m0.state_size, msub), dtype=torch.float64, device=dev)
        for k in range(1, first):
            En, dE = inputs(k)
            st = m0.update(lam_s, Q_s, En[:msub].contiguous(), dE[:msub].contiguous(), st,
                           tree_id=tid_d[:msub].contiguous())["state_out"]
        m0.close()
        # the project's autotuner on the handle of four trees, on this sub-batch
        En, dE = inputs(first)
        tuned = autotune.tune(trees, prec, lam_s, Q_s, En[:msub].contiguous(), dE[:msub].contiguous(), st, reps=1,
                              tree_id=tid_d[:msub].contiguous(), first_stage=stage)
        best = (tuned["block"], tuned["ctas_per_sm"], tuned["newton_ms"])
        del st
        torch.cuda.empty_cache()
        m = dmn.DMN(trees, precision=prec, block=best[0], ctas_per_sm=best[1], predictor=pred, first_stage=stage)
        lam, Q = m.interp_orientation(A2_d)
        S = m.state_size
        bufs = [torch.zeros((S, n), dtype=torch.float64, device=dev) for _ in range(2)]
        outs = [None] * G
        for j in range(G):
            outs[j] = dict(stress=torch.empty((n, 6), dtype=torch.float64, device=dev),
                           tangent=torch.empty((n, 6, 6), dtype=torch.float64, device=dev),
                           iters=torch.empty(n, dtype=torch.int32, device=dev),
                           status=torch.empty(n, dtype=torch.int32, device=dev))
        for k in range(1, first):       # warm-up increments, eager
            En, dE = inputs(k)
            o = dict(outs[0], state_out=bufs[k % 2])
            m.update(lam, Q, En, dE, bufs[(k - 1) % 2], out=o, tree_id=tid_d)
        En_all, dE_all = zip(*[inputs(k) for k in inc])
        base = (first - 1) % 2
        for j in range(G):
            outs[j]["state_out"] = bufs[(base + j + 1) % 2]
        # the graph: increments first .. first+G-1, state ping-pong between the two buffers
        torch.cuda.synchronize()
        g = torch.cuda.CUDAGraph()
        side = torch.cuda.Stream()
        side.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(side):
            with torch.cuda.graph(g, stream=side):
                for j in range(G):
                    m.update(lam, Q, En_all[j], dE_all[j], bufs[(base + j) % 2], out=outs[j], tree_id=tid_d)
        torch.cuda.current_stream().wait_stream(side)
        torch.cuda.synchronize()
        clocks = ClockSampler("0")
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        g.replay()
        e1.record()
        torch.cuda.synchronize()
        clk = clocks.stop()
        t_ms = e0.elapsed_time(e1)
        its = torch.stack([o["iters"] for o in outs]).to(torch.int64)
        stat = torch.stack([o["status"] for o in outs])
        el = torch.from_numpy(elastic).to(dev)
        line["forms"][form] = {
            "value": n * G / (t_ms * 1e-3), "unit": UNIT, "ms_per_step": t_ms / G,
            "launch": {"block": best[0], "ctas_per_sm": best[1], "autotuner_table": tuned["table"]},
            "iters_elastic_half": torch.bincount(its[:, el].reshape(-1)).cpu().tolist(),
            "iters_cyclic_half": torch.bincount(its[:, ~el].reshape(-1)).cpu().tolist(),
            "status_counts": torch.bincount(stat.reshape(-1).to(torch.int64)).cpu().tolist(),
            "clocks": clk}
        del g, outs, bufs, En_all, dE_all
        m.close()
        torch.cuda.empty_cache()
    main_form = "f64" if "f64" in line["forms"] else next(iter(line["forms"]))
    line["value"] = line["forms"][main_form]["value"]
    line["dtype"] = "f64" if form_opts(main_form)[0] == "f64" else "f32+f64"
    print(json.dumps(line), flush=True)
    return 0


# ---------------------------------------------------------------------------------------------
# FE-coupled plate: a plate with a central hole (O-grid, 48 x 4 columns around the hole, 98
# elements radially, 8 through the half thickness: 150,528 hexahedra x 8 Gauss points =
# 1,204,224 DMN points at depth 8), tension to 1.5 % in 30 increments, macro Newton with
# Jacobi-PCG.  A secondary measurement (not the headline line).
PLATE = dict(n_t=48, n_r=98, n_z=8, R=5.0, H=25.0, T=4.0)
PLATE_INCREMENTS = 30
PLATE_STRAIN = 0.015


def run_plate(args):
    import torch
    from paper_2103_08253_gb300 import fe
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    mesh = W.plate_with_hole_mesh(PLATE["n_t"], PLATE["n_r"], PLATE["n_z"], R=PLATE["R"], H=PLATE["H"],
                                  T=PLATE["T"])
    A2 = W.plate_orientation_field(mesh.centroid, mesh.R, mesh.H, mesh.T, seed=SEED_ORI + 21)
    tree = W.tree_d10_fit(K_DEPTH, seed=SEED_TREE)
    n_inc = min(args.steps, PLATE_INCREMENTS)
    n_gp = 8 * mesh.conn.shape[0]
    line = {"metric": "FE-DMN plate with hole: DMN Gauss-point updates/s inside the macro Newton loop",
            "unit": UNIT, "n_gpus": 1, "steps": n_inc, "warmup": 0, "higher_is_better": True, "data": "synthetic",
            "config": {"workload": "plate with hole, %d hexahedra x 8 Gauss points = %d DMN points (K=8), tension "
                                   "to %.1f%% in %d increments (first %d run)"
                                   % (mesh.conn.shape[0], n_gp, 100 * PLATE_STRAIN, PLATE_INCREMENTS, n_inc),
                       "dofs": int(mesh.xyz.size), "newton_rtol": 1e-6, "cg_rtol": 1e-6,
                       "cg_operator": "FP32 products, FP64 vectors (fe_pcg_f32)", "mesh": PLATE,
                       "dmn_line_search": True, "predictor": "uniform strain, then extrapolated increments"},
            "forms": {}}
    for form in [f for f in args.forms.split(",") if f]:
        prec, pred = form_opts(form)
        run = fe.FEDMN(mesh, tree, A2, precision=prec, newton_rtol=1e-6, cg_rtol=1e-6, cg_f32=True, predictor=pred)
        clocks = ClockSampler("0")
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        incs = []
        for k in range(1, n_inc + 1):
            delta = PLATE_STRAIN * 2 * mesh.H * k / PLATE_INCREMENTS
            r = run.increment(delta)
            incs.append(dict(k=k, newton=r["newton"], cg=r["cg_iters"], reaction=r["reaction"],
                             converged=bool(r["converged"]), bad=r["dmn_status_bad"]))
        torch.cuda.synchronize()
        wall = time.perf_counter() - t0
        clk = clocks.stop()
        tm = run.timing
        line["forms"][form] = {
            "value": n_gp * tm["dmn_calls"] / tm["dmn_s"], "unit": UNIT,
            "wall_s": wall, "ms_per_increment": 1e3 * wall / n_inc, "dmn_s": tm["dmn_s"], "fe_s": tm["fe_s"],
            "dmn_calls": tm["dmn_calls"], "cg_iters": tm["cg_iters"],
            "macro_newton_per_increment": [x["newton"] for x in incs],
            "all_converged": all(x["converged"] for x in incs), "dmn_status_bad": sum(x["bad"] for x in incs),
            "reaction_N": [round(x["reaction"], 6) for x in incs], "clocks": clk}
        print(json.dumps({"form": form, "partial": line["forms"][form]}), file=sys.stderr, flush=True)
        run.close()
        del run
        torch.cuda.empty_cache()
    main_form = "f64" if "f64" in line["forms"] else next(iter(line["forms"]))
    line["value"] = line["forms"][main_form]["value"]
    line["ms_per_step"] = line["forms"][main_form]["ms_per_increment"]
    line["dtype"] = "f64" if form_opts(main_form)[0] == "f64" else "f32+f64"
    print(json.dumps(line), flush=True)
    return 0


# ---------------------------------------------------------------------------------------------
# Offline training (differentiation workload): a depth-8 DMN with trainable angle coefficients
# and leaf weights fitted to a seeded target DMN on 4096 elastic stiffness samples (relative
# error in the Sec. 3.1 loss, p = 1, q = 10, penalty 1e3) plus 4096 stresses of one
# elastoplastic increment from the virgin state (1-3 % equivalent strain); AMSGrad with the
# schedule of Sec. 4.4.  Forward: dmn_update (6 unit strains per stiffness sample), backward:
# dmn_grad.  A secondary measurement (not the headline line).
TRAIN_SAMPLES = 4096


def run_train(args):
    import torch
    from paper_2103_08253_gb300 import training
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    target = W.tree_d10_fit(K_DEPTH, seed=SEED_TREE + 31)
    tr = training.Trainer(K_DEPTH, target, TRAIN_SAMPLES, seed=SEED_TREE + 32, elastic_matrix=W.Phase(0, 3000.0, 0.35),
                          plastic=W.MATRIX, n_plastic=TRAIN_SAMPLES, plastic_precision=args.train_plastic,
                          elastic_precision=args.train_elastic, stiffness_method=args.train_stiffness)
    tr.train(args.warmup)
    clocks = ClockSampler("0")
    t = tr.train(args.steps)
    clk = clocks.stop()
    hist = tr.history
    six = tr.stiff_method == "stress" or (tr.stiff_method is None and args.train_elastic == "mixed-f32-tangent")
    # updates per epoch (forward), each with its adjoint: per stiffness sample one (tangent seed) or six
    n_upd = TRAIN_SAMPLES * (6 if six else 1) + TRAIN_SAMPLES
    line = {"metric": "DMN offline training: samples/s (forward + adjoint) at depth 8", "unit": "samples/s",
            "value": 2 * TRAIN_SAMPLES * args.steps / t, "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * t / args.steps, "higher_is_better": True, "dtype": "f64" if args.train_plastic == args.train_elastic == "f64" else "f32+f64", "data": "synthetic",
            "config": {"workload": "K=8, %d stiffness samples (elastic phases) + %d stress samples (one J2 increment),"
                                   " target = seeded DMN, AMSGrad + cosine schedule (Sec. 4.4); step = epoch"
                                   % (TRAIN_SAMPLES, TRAIN_SAMPLES),
                       "dmn_updates_per_epoch": n_upd,
                       "plastic_samples_precision": args.train_plastic,
                       "stiffness_samples_precision": args.train_elastic,
                       "stiffness_gradient": "six stress adjoints" if six else "tangent-seeded adjoint"},
            "gp_updates_per_s": n_upd * args.steps / t,
            "compression": {"handle_rebuilds": tr.rebuilds, "leaves_left": int(tr.pattern.sum()),
                            "leaves": 1 << K_DEPTH},
            "loss": [round(h[0], 6) for h in hist], "mean_stiffness_error": [round(h[2], 6) for h in hist],
            "clocks": clk}
    tr.close()
    print(json.dumps(line), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--points", type=int, default=1 << 20)
    ap.add_argument("--forms", default="f64,mixed,mixed-f32-tangent,f64/stage",
                    help="precisions, each optionally with /extrap: the Newton iteration starts from the last "
                         "update's jumps extrapolated along the strain increment instead of the paper's a^n")
    ap.add_argument("--e2e-chunk", type=int, default=0,
                    help="points per chunk of dmn_update_host (0: the library's default)")
    ap.add_argument("--e2e-steps", type=int, default=-1,
                    help="increments timed through dmn_update_host (-1: the same increments as the device timing)")
    ap.add_argument("--ref-points", type=int, default=1024)
    ap.add_argument("--cpu-points", type=int, default=1024)
    ap.add_argument("--parity-points", type=int, default=256,
                    help="points of the timed batch recomputed by the oracle for the error statement")
    ap.add_argument("--matrix", default="linear", choices=["linear", "explin"],
                    help="matrix law of the k8 workloads: linear hardening (default) or the paper's exp-linear")
    ap.add_argument("--train-plastic", default="mixed-f32-tangent", choices=["f64", "mixed", "mixed-f32-tangent"],
                    help="precision of the training workload's plastic forward solves (the adjoint is FP64)")
    ap.add_argument("--train-stiffness", default=None, choices=["tangent", "stress"],
                    help="training workload: stiffness gradients by tangent seeds or six stress adjoints")
    ap.add_argument("--train-elastic", default="mixed", choices=["f64", "mixed", "mixed-f32-tangent"],
                    help="precision of the training workload's stiffness-sample forward solves")
    ap.add_argument("--shape", type=int, default=3, choices=[3, 4, 6],
                    help="shape functions of the angle interpolation: 3 linear (default, D10 fit), 4 tri-linear, "
                         "6 quadratic (seeded nodal angles)")
    ap.add_argument("--no-autotune", dest="autotune", action="store_false",
                    help="use the library's default launch shape instead of autotuning it")
    ap.add_argument("--workload", default="k8", choices=["k8", "k8-compressed", "mixed-depth", "plate", "train"],
                    help="k8: the headline depth-8 batch; mixed-depth: 4M points of depths 5-8; plate: the "
                         "FE-coupled plate with a hole (both secondary)")
    args = ap.parse_args()
    if args.workload == "plate":
        return run_plate(args)
    if args.workload == "train":
        return run_train(args)
    if args.workload == "mixed-depth":
        if args.points == 1 << 20:
            args.points = 1 << 22
        return run_mixed_depth(args)
    if args.warmup < 3:
        raise SystemExit("--warmup must be >= 3")
    if args.warmup + args.steps > N_INCREMENTS:
        raise SystemExit("warmup + steps must not exceed the %d increments of the load path" % N_INCREMENTS)
    if args.impl == "reference":
        return run_reference(args)
    return run_gpu(args)


def run_gpu(args):
    import torch
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        import torch.distributed as tdist
        tdist.init_process_group("nccl")
        dist = tdist
    from paper_2103_08253_gb300 import dmn
    dmn.load_library()
    peaks = measure_peaks()
    n = args.points
    cmp = args.workload == "k8-compressed"
    tree, A2, lam_np, Q_np, Ef = make_workload(n, rank, cmp, args.matrix, args.shape)
    try:
        smi_id = "GPU-" + str(torch.cuda.get_device_properties(dev).uuid)
    except Exception:
        smi_id = str(local)
    A2_d = torch.from_numpy(A2).to(dev)
    Ef_d = torch.from_numpy(Ef).to(dev)
    total = args.warmup + args.steps
    En = [Ef_d * ((s - 1) / N_INCREMENTS) for s in range(1, total + 1)]
    dE = [Ef_d * (s / N_INCREMENTS) - En[s - 1] for s in range(1, total + 1)]
    ctx = dict(dev=dev, n=n, tree=tree, A2=A2_d, En=En, dE=dE, smi_id=smi_id, rank=rank, A2_np=A2, Ef_np=Ef)
    forms = [f for f in args.forms.split(",") if f]
    rng = np.random.default_rng(7)
    pidx = np.sort(rng.choice(n, size=min(args.parity_points, n), replace=False))
    results, e2e = {}, None
    for form in forms:
        r = run_form(form, ctx, args, dist)
        if world == 1 and args.parity_points > 0:     # the CPU-baseline leg: N = 1 only
            r["parity"] = parity_sample(form, r, ctx, args, pidx)
        if form == "f64" and args.e2e_steps != 0:
            e2e = run_e2e(r, ctx, args, dist)
        r["m"].close()
        for k in ("stress", "tangent", "status", "state", "host_state", "st", "lam", "Q", "m"):
            r.pop(k, None)
        torch.cuda.empty_cache()
        results[form] = r
    if rank != 0:
        return 0
    steps = args.steps
    forms_out = {}
    for form, r in results.items():
        v = job_value(world, n, steps, r["t_ms"])
        forms_out[form] = {"value": v, "unit": UNIT, "ms_per_step": r["t_ms"] / steps,
                           "kernel_ms_per_step": {k: x / steps for k, x in r["kms"].items()},
                           "newton_iters_per_update": r["iters_sum"] / (n * steps), "iters_hist": r["iters_hist"],
                           "roofline": (roofline_f64(r, n, steps, tree.w, peaks) if form_opts(form)[0] == "f64"
                                        else roofline_mixed(r, n, steps, tree.w,
                                                            sweep=form_opts(form)[0] == "mixed", peaks=peaks)),
                           "launch": r["launch"],
                           "parity_vs_oracle": r.get("parity"), "clocks": r["clocks"]}
    main_form = "f64" if "f64" in results else forms[0]
    mr = results[main_form]
    cpu = None
    if world == 1 and args.cpu_points > 0:
        cores = os.cpu_count() or 1
        idx = np.arange(min(args.cpu_points, n))
        t = oracle_baseline(tree, A2, Ef, idx, args.warmup, min(3, steps), cores)
        cpu = {"value": len(idx) * min(3, steps) / t, "unit": UNIT, "cores": cores, "kind": "oracle",
               "sample": "first %d points, increments %d..%d after %d untimed, orientation set-up included"
                         % (len(idx), args.warmup + 1, args.warmup + min(3, steps), args.warmup)}
    line = {"metric": METRIC, "value": forms_out[main_form]["value"], "unit": UNIT, "n_gpus": world,
            "steps": steps, "warmup": args.warmup, "ms_per_step": mr["t_ms"] / steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64" if form_opts(main_form)[0] == "f64" else "f32+f64",
            "data": "synthetic",
            "config": {"workload": WORKLOAD_CMP if cmp else WORKLOAD, "K": K_DEPTH, "points_per_gpu": n,
                       "increments": N_INCREMENTS, "matrix": MATRIX_NOTE[args.matrix],
                       "shape_functions": SHAPE_NOTE[args.shape],
                       "timed_increments": [args.warmup + 1, args.warmup + steps],
                       "l2": ("flushed before every step (256 MB fill, in the timed region): per-step state "
                              "%.1f MB" if l2_flush_needed(state_fields(tree), n) else
                              "no flush: per-step inputs (state %.1f MB) exceed L2")
                             % (state_fields(tree) * n * 8e-6),
                       "parallelism": "independent point shards per GPU, no collective"},
            "roofline": forms_out[main_form]["roofline"], "cpu_baseline": cpu, "e2e": e2e,
            "gpu_launches": (4 + ("stage" in mr["kms"]) + (bool(mr.get("warp")) and main_form.split("/")[0] == "mixed"))
                            * steps, "clocks": mr["clocks"],
            "peaks": {"fp64_gflops": peaks["f64"], "fp32_gflops": peaks["f32"], "note": peaks["note"]}}
    # the other forms side by side with the headline: value, roofline and error against the oracle
    for form in ("mixed", "mixed-f32-tangent", "f64/stage"):
        if form in forms_out and form != main_form:
            key = form.replace("-", "_").replace("/", "_")
            line["value_" + key] = forms_out[form]["value"]
            line["roofline_" + key] = forms_out[form]["roofline"]
            line["parity_" + key] = forms_out[form]["parity_vs_oracle"]
    if main_form in forms_out:
        line["parity"] = forms_out[main_form]["parity_vs_oracle"]
    line["forms"] = forms_out
    print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
