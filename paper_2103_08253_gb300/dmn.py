"""Python binding of the DMN C ABI (include/dmn.h).

Argument marshalling only: every step of the update runs in the CUDA library
``_build/libdmn.so``.  PyTorch provides device memory and the current stream.
There is no CPU fallback: if the library or a CUDA device is missing, the calls
raise.
"""
from __future__ import annotations

import ctypes
import os
import sys

from . import build as _build

_lib = None

# ABI symbols declared in include/dmn.h
EXPORTS = ("dmn_create", "dmn_destroy", "dmn_state_size", "dmn_update_lanes_per_point", "dmn_interp_orientation",
           "dmn_update",
           "dmn_set_params", "dmn_grad", "dmn_profile_enable", "dmn_profile_read", "dmn_profile_read_stages",
           "dmn_update_noalloc",
           "dmn_update_host", "dmn_last_error")

PHASE_ELASTIC, PHASE_J2_LINEAR, PHASE_J2_EXPLIN = 0, 1, 2
PREC_F64 = 0
PREC_MIXED = 1
PREC_MIXED_F32_TANGENT = 2
PRECISIONS = {"f64": PREC_F64, "mixed": PREC_MIXED, "mixed-f32-tangent": PREC_MIXED_F32_TANGENT}
STATUS_OK, STATUS_MAXITER, STATUS_NONFINITE, STATUS_LINESEARCH, STATUS_BAD_TREE = 0, 1, 2, 3, 4
MAX_TREES = 8


class Phase_(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("E", ctypes.c_double), ("nu", ctypes.c_double),
                ("sigma0", ctypes.c_double), ("H", ctypes.c_double), ("sigma_inf", ctypes.c_double),
                ("k0", ctypes.c_double)]


class TreeDesc_(ctypes.Structure):
    _fields_ = [("K", ctypes.c_int32), ("M", ctypes.c_int32), ("p", ctypes.POINTER(ctypes.c_double)),
                ("q", ctypes.POINTER(ctypes.c_double)), ("w", ctypes.POINTER(ctypes.c_double)),
                ("phase", Phase_ * 2)]


class Options_(ctypes.Structure):
    _fields_ = [("tol", ctypes.c_double), ("max_iter", ctypes.c_int32), ("precision", ctypes.c_int32),
                ("block", ctypes.c_int32), ("ctas_per_sm", ctypes.c_int32), ("line_search", ctypes.c_int32),
                ("predictor", ctypes.c_int32), ("first_stage", ctypes.c_int32),
                ("stage_ctas_per_sm", ctypes.c_int32), ("warp_per_point", ctypes.c_int32),
                ("warp_lanes", ctypes.c_int32)]


def library_path() -> str:
    return _build.LIB


def load_library(build_if_missing: bool = True):
    """Load the CUDA library (building it first if it is missing or stale)."""
    global _lib
    if _lib is not None:
        return _lib
    path = _build.LIB
    if build_if_missing:
        path = _build.build()
    if not os.path.exists(path):
        raise RuntimeError("DMN CUDA library not built: run __graft_entry__.build() or "
                           "python -m paper_2103_08253_gb300.build")
    lib = ctypes.CDLL(path)
    vp, i64, i32 = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32
    lib.dmn_create.argtypes = [ctypes.POINTER(TreeDesc_), i32, ctypes.POINTER(Options_), ctypes.POINTER(vp)]
    lib.dmn_create.restype = ctypes.c_int
    lib.dmn_destroy.argtypes = [vp]
    lib.dmn_destroy.restype = None
    lib.dmn_state_size.argtypes = [vp, i32]
    lib.dmn_state_size.restype = i64
    lib.dmn_update_lanes_per_point.restype = ctypes.c_int
    lib.dmn_update_lanes_per_point.argtypes = [ctypes.c_void_p, i64]
    lib.dmn_interp_orientation.argtypes = [vp, i64, vp, vp, vp, vp]
    lib.dmn_interp_orientation.restype = ctypes.c_int
    lib.dmn_update.argtypes = [vp, i64, vp, vp, vp, vp, vp, vp, vp, vp, vp, vp, vp, vp]
    lib.dmn_update.restype = ctypes.c_int
    lib.dmn_update_host.argtypes = [vp, i64, vp, vp, vp, vp, vp, vp, vp, vp, vp, vp, vp, i64, vp]
    lib.dmn_update_host.restype = ctypes.c_int
    lib.dmn_set_params.argtypes = [vp, i32, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double),
                                   ctypes.POINTER(ctypes.c_double)]
    lib.dmn_set_params.restype = ctypes.c_int
    lib.dmn_grad.argtypes = [vp, i64, vp, vp, vp, vp, vp, vp, vp, vp, vp, vp, vp, vp, vp, vp]
    lib.dmn_grad.restype = ctypes.c_int
    lib.dmn_profile_enable.argtypes = [vp, i32]
    lib.dmn_profile_enable.restype = ctypes.c_int
    lib.dmn_profile_read.argtypes = [vp, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(i64)]
    lib.dmn_profile_read.restype = ctypes.c_int
    lib.dmn_profile_read_stages.argtypes = [vp, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(i64),
                                            ctypes.POINTER(i64)]
    lib.dmn_profile_read_stages.restype = ctypes.c_int
    lib.dmn_update_noalloc.argtypes = [ctypes.POINTER(TreeDesc_), ctypes.POINTER(Options_), i64,
                                       vp, vp, vp, vp, vp, vp, vp, vp, vp, vp, vp]
    lib.dmn_update_noalloc.restype = ctypes.c_int
    lib.dmn_last_error.argtypes = [vp]
    lib.dmn_last_error.restype = ctypes.c_char_p
    lib.dmn_peak_gflops.argtypes = [i32, ctypes.c_double, ctypes.POINTER(ctypes.c_double),
                                    ctypes.POINTER(ctypes.c_double), vp]
    lib.dmn_peak_gflops.restype = ctypes.c_int
    lib.dmn_fma_throughput.argtypes = [i32, i32, i32, i32, ctypes.c_double, ctypes.POINTER(ctypes.c_double),
                                       ctypes.POINTER(ctypes.c_double), vp]
    lib.dmn_fma_throughput.restype = ctypes.c_int
    _lib = lib
    return lib


# include/dmn_peak.h
PEAK_EXPORTS = ("dmn_peak_gflops", "dmn_fma_throughput")
PEAK_FP64_FMA, PEAK_FP32_FMA = 0, 1


def peak_gflops(kind: str = "fp64", seconds: float = 1.0):
    """Sustained FMA throughput (GFLOP/s) of the current CUDA device over about `seconds`
    (dmn_peak_gflops, on torch's current stream); returns (gflops, measured ms)."""
    import torch
    lib = load_library()
    k = {"fp64": PEAK_FP64_FMA, "fp32": PEAK_FP32_FMA}[kind]
    g, ms = ctypes.c_double(), ctypes.c_double()
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    rc = lib.dmn_peak_gflops(k, float(seconds), ctypes.byref(g), ctypes.byref(ms), stream)
    if rc != 0:
        raise RuntimeError(lib.dmn_last_error(None).decode())
    return g.value, ms.value


def fma_throughput(kind: str = "fp64", warps_per_sm: int = 64, chains: int = 8, active_lanes: int = 32,
                   seconds: float = 0.2):
    """dmn_fma_throughput: FMA GFLOP/s of the active lanes at a chosen occupancy, number of independent
    chains per thread and number of active lanes per warp; returns (gflops, measured ms)."""
    import torch
    lib = load_library()
    k = {"fp64": PEAK_FP64_FMA, "fp32": PEAK_FP32_FMA}[kind]
    g, ms = ctypes.c_double(), ctypes.c_double()
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    rc = lib.dmn_fma_throughput(k, int(warps_per_sm), int(chains), int(active_lanes), float(seconds), ctypes.byref(g),
                                ctypes.byref(ms), stream)
    if rc != 0:
        raise RuntimeError(lib.dmn_last_error(None).decode())
    return g.value, ms.value


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else None


def _check_dev(name, t, dtype, shape, device=None):
    """Raise unless t is a contiguous CUDA tensor of dtype, of shape `shape` (a tuple, or a list of
    accepted tuples), on `device` if given (the device whose memory the library's kernels read)."""
    import torch
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError("%s must be a CUDA tensor" % name)
    if device is not None and t.device != device:
        raise ValueError("%s is on %s, the handle on %s" % (name, t.device, device))
    if t.dtype != dtype:
        raise TypeError("%s must be %s" % (name, dtype))
    if not t.is_contiguous():
        raise ValueError("%s must be contiguous" % name)
    shapes = shape if isinstance(shape, list) else [shape]
    if tuple(t.shape) not in [tuple(x) for x in shapes]:
        raise ValueError("%s has shape %s, expected %s" % (name, tuple(t.shape), " or ".join(str(tuple(x)) for x in shapes)))


def _check_host(name, t, dtype, shape):
    import torch
    if not isinstance(t, torch.Tensor) or t.device.type != "cpu":
        raise TypeError("%s must be a CPU tensor" % name)
    if t.dtype != dtype:
        raise TypeError("%s must be %s" % (name, dtype))
    if not t.is_contiguous():
        raise ValueError("%s must be contiguous" % name)
    if tuple(t.shape) != tuple(shape):
        raise ValueError("%s has shape %s, expected %s" % (name, tuple(t.shape), tuple(shape)))


def _fill_desc(d, tr):
    """Fill the dmn_tree_desc d from a tree object; returns the arrays d points into (keep them alive)."""
    import numpy as np
    dp = ctypes.POINTER(ctypes.c_double)
    keep = [np.ascontiguousarray(x, dtype=np.float64).reshape(-1) for x in (tr.p, tr.q, tr.w)]
    d.K, d.M = int(tr.K), int(tr.M)
    d.p, d.q, d.w = (a.ctypes.data_as(dp) for a in keep)
    for f, ph in enumerate(tr.phases):
        d.phase[f] = Phase_(int(ph.kind), float(ph.E), float(ph.nu), float(ph.sigma0), float(ph.H),
                            float(getattr(ph, "sigma_inf", 0.0)), float(getattr(ph, "k0", 0.0)))
    return keep


def update_noalloc(tree, lam, Q, E_n, dE, state_in, out=None, tol=1e-12, max_iter=50):
    """dmn_update_noalloc: the FP64 update of one uncompressed tree with no handle, the library allocating
    no device memory (its work space is a static 64 MiB array; calls that overlap on the GPU race).
    Arrays as in DMN.update, on lam's device, state [6 (inelastic leaves) + 3 (2^K - 1)][n]; `out`
    (a dict like DMN.alloc_outputs) is allocated by torch if None.  Returns out."""
    import torch
    lib = load_library()
    n = lam.shape[0]
    dev = lam.device
    K = int(tree.K)
    n_inel = sum(int(ph.kind) != PHASE_ELASTIC for ph in tree.phases)
    S = 6 * n_inel * (1 << (K - 1)) + 3 * ((1 << K) - 1)
    if out is None:
        out = dict(state_out=torch.empty((S, n), dtype=torch.float64, device=dev),
                   stress=torch.empty((n, 6), dtype=torch.float64, device=dev),
                   tangent=torch.empty((n, 6, 6), dtype=torch.float64, device=dev),
                   iters=torch.empty(n, dtype=torch.int32, device=dev),
                   status=torch.empty(n, dtype=torch.int32, device=dev))
    for name, t, dtype, shape in (("lam", lam, torch.float64, (n, 2)), ("Q", Q, torch.float64, (n, 9)),
                                  ("E_n", E_n, torch.float64, (n, 6)), ("dE", dE, torch.float64, (n, 6)),
                                  ("state_in", state_in, torch.float64, (S, n)),
                                  ("state_out", out["state_out"], torch.float64, (S, n)),
                                  ("stress", out["stress"], torch.float64, (n, 6)),
                                  ("tangent", out["tangent"], torch.float64, (n, 6, 6)),
                                  ("iters", out["iters"], torch.int32, (n,)),
                                  ("status", out["status"], torch.int32, (n,))):
        _check_dev(name, t, dtype, shape, dev)
    d = TreeDesc_()
    keep = _fill_desc(d, tree)
    opt = Options_(float(tol), int(max_iter), PREC_F64, 0, 0, 0, 0)
    with torch.cuda.device(dev):
        s = torch.cuda.current_stream(dev).cuda_stream
        rc = lib.dmn_update_noalloc(ctypes.byref(d), ctypes.byref(opt), n, _ptr(lam), _ptr(Q), _ptr(E_n), _ptr(dE),
                                    _ptr(state_in), _ptr(out["state_out"]), _ptr(out["stress"]),
                                    _ptr(out["tangent"]), _ptr(out["iters"]), _ptr(out["status"]),
                                    ctypes.c_void_p(s))
    del keep   # the library copied the parameters during the call
    if rc != 0:
        raise RuntimeError("dmn_update_noalloc failed (%d): %s" % (rc, lib.dmn_last_error(None).decode()))
    return out


class DMN:
    """One or several DMNs (up to 8, e.g. of different depths) on the current CUDA device.

    tree: an object with K, M, p [N, M], q [N, M], w [2^K] (numpy, paper
    ordering) and phases (two objects with kind, E, nu, sigma0, H), or a list
    of such objects (tree i is selected by tree_id == i in update()).
    precision: "f64"; "mixed" (FP32 condensation, FP64 residual and final
    sweep); "mixed-f32-tangent" (the mixed iteration, tangent from its last
    FP32 condensation).  predictor: start each Newton iteration from the last update's jumps
    extrapolated along the new strain increment (the state then holds the last jump change
    and strain increment too).  first_stage: True starts every point with the all-FP32 Newton
    stage, False goes straight to the iteration of the chosen precision; None (default) runs it
    in the mixed forms only.  warp_per_point: 0 (default) the warp organisation for calls of at most
    1024 points per SM in the FP64 form, 256 in the mixed forms; 1 always, -1 never (the paper's
    start); warp_lanes: lanes per point there (32, 16, 8; 0 chooses by the call's size).  The other options are those of dmn_options."""

    def __init__(self, tree, precision: str = "f64", tol: float = 1e-12, max_iter: int = 50, block: int = 0,
                 ctas_per_sm: int = 0, line_search: bool = False, predictor: bool = False,
                 first_stage=None, stage_ctas_per_sm: int = 0, warp_per_point: int = 0, warp_lanes: int = 0):
        import torch
        self._lib = load_library()
        if not torch.cuda.is_available():
            raise RuntimeError("dmn.DMN needs a CUDA device; the library has no CPU path")
        # the handle's parameters and scratch live on this device; every call runs there
        self.device = torch.device("cuda", torch.cuda.current_device())
        trees = list(tree) if isinstance(tree, (list, tuple)) else [tree]
        self.n_trees = len(trees)
        self.K, self.M = int(trees[0].K), int(trees[0].M)
        self._Ks = [int(tr.K) for tr in trees]
        self._Ms = [int(tr.M) for tr in trees]
        self.phases = tuple(trees[0].phases)
        descs = (TreeDesc_ * len(trees))()
        self._keep = []
        for k, tr in enumerate(trees):
            self._keep += _fill_desc(descs[k], tr)
        if precision not in PRECISIONS:
            raise ValueError("precision must be one of %s" % (tuple(PRECISIONS),))
        opt = Options_(float(tol), int(max_iter), PRECISIONS[precision], int(block),
                       int(ctas_per_sm), int(bool(line_search)), int(bool(predictor)),
                       0 if first_stage is None else (1 if first_stage else -1), int(stage_ctas_per_sm),
                       int(warp_per_point), int(warp_lanes))
        self.precision = precision
        want = precision != "f64" if first_stage is None else bool(first_stage)
        self.first_stage = want and not line_search and not predictor
        self.predictor = bool(predictor)
        h = ctypes.c_void_p()
        rc = self._lib.dmn_create(descs, len(trees), ctypes.byref(opt), ctypes.byref(h))
        if rc != 0:
            raise ValueError("dmn_create failed (%d): %s" % (rc, self._lib.dmn_last_error(None).decode()))
        self._h = h
        # state fields of the arrays passed to update(); tree i uses the first tree_state_sizes[i]
        self.state_size = int(self._lib.dmn_state_size(h, -1))
        self.tree_state_sizes = [int(self._lib.dmn_state_size(h, k)) for k in range(len(trees))]

    def lanes_per_point(self, n: int) -> int:
        """dmn_update_lanes_per_point: the organisation of a call of n points, as lanes per point (1
        one point per thread of the persistent kernel; 32, 16 or 8 the warp organisation)."""
        r = self._lib.dmn_update_lanes_per_point(self._h, int(n))
        if r < 0:
            raise ValueError("lanes_per_point: n must be >= 0 on an open handle")
        return int(r)

    def close(self):
        if getattr(self, "_h", None):
            with self._on_device():
                self._lib.dmn_destroy(self._h)
            self._h = None

    def _on_device(self):
        import torch
        return torch.cuda.device(self.device)

    def _check(self, name, t, dtype, shape):
        _check_dev(name, t, dtype, shape, self.device)

    def __del__(self):
        # at interpreter exit the CUDA runtime may already be torn down; the
        # process releases the device memory anyway
        if sys is None or sys.is_finalizing():
            return
        try:
            self.close()
        except Exception:
            pass

    def _err(self, what, rc):
        msg = self._lib.dmn_last_error(self._h).decode()
        raise RuntimeError("%s failed (%d): %s" % (what, rc, msg))

    def interp_orientation(self, A2, lam=None, Q=None):
        """A2 [n, 6] float64 CUDA -> (lam [n, 2], Q [n, 9])."""
        import torch
        n = A2.shape[0]
        self._check("A2", A2, torch.float64, (n, 6))
        lam = torch.empty((n, 2), dtype=torch.float64, device=A2.device) if lam is None else lam
        Q = torch.empty((n, 9), dtype=torch.float64, device=A2.device) if Q is None else Q
        self._check("lam", lam, torch.float64, (n, 2))
        self._check("Q", Q, torch.float64, (n, 9))
        with self._on_device():
            s = torch.cuda.current_stream(self.device).cuda_stream
            rc = self._lib.dmn_interp_orientation(self._h, n, _ptr(A2), _ptr(lam), _ptr(Q), ctypes.c_void_p(s))
        if rc != 0:
            self._err("dmn_interp_orientation", rc)
        return lam, Q

    def set_params(self, p, q, w, tree_id: int = 0):
        """Replace p, q, w of one tree (numpy or CPU tensors, paper ordering)."""
        import numpy as np
        arrs = [np.ascontiguousarray(np.asarray(x, dtype=np.float64)).reshape(-1) for x in (p, q, w)]
        dp = ctypes.POINTER(ctypes.c_double)
        tr = int(tree_id)
        if not 0 <= tr < self.n_trees:
            raise ValueError("tree_id must be in 0..%d" % (self.n_trees - 1))
        K = self._Ks[tr]
        N = (1 << K) - 1
        for name, a, size in (("p", arrs[0], N * self._Ms[tr]), ("q", arrs[1], N * self._Ms[tr]), ("w", arrs[2], 1 << K)):
            if a.size != size:
                raise ValueError("%s has %d entries, expected %d" % (name, a.size, size))
        with self._on_device():
            rc = self._lib.dmn_set_params(self._h, tr, *(a.ctypes.data_as(dp) for a in arrs))
        if rc != 0:
            self._err("dmn_set_params", rc)

    def grad(self, lam, Q, E_n, dE, state_in, state_out, g_stress, g_p=None, g_q=None, g_w=None, want_E=True,
             g_tangent=None):
        """Adjoint of a converged update: returns (g_p [N, M], g_q [N, M], g_w [2^K], g_E [n, 6] or None),
        with g_p, g_q, g_w accumulated into the given tensors if passed.  g_stress [n, 6] and/or
        g_tangent [n, 6, 6] (trees of elastic phases) are the seeds; with g_stress None, E_n, dE and
        the states may be None too."""
        import torch
        n = lam.shape[0]
        dev = lam.device
        N = (1 << self.K) - 1
        checks = [("lam", lam, (n, 2)), ("Q", Q, (n, 9))]
        if g_stress is not None:
            checks += [("E_n", E_n, (n, 6)), ("dE", dE, (n, 6)), ("state_in", state_in, (self.state_size, n)),
                       ("state_out", state_out, (self.state_size, n)), ("g_stress", g_stress, (n, 6))]
        if g_tangent is not None:
            g_tangent = g_tangent.reshape(n, 36) if g_tangent.dim() == 3 and g_tangent.is_contiguous() else g_tangent
            checks.append(("g_tangent", g_tangent, (n, 36)))
        if g_stress is None and g_tangent is None:
            raise ValueError("grad: g_stress and g_tangent are both None")
        for name, t, shape in checks:
            self._check(name, t, torch.float64, shape)
        z = lambda *sh: torch.zeros(sh, dtype=torch.float64, device=dev)
        g_p = z(N, self.M) if g_p is None else g_p
        g_q = z(N, self.M) if g_q is None else g_q
        g_w = z(1 << self.K) if g_w is None else g_w
        # the library adds into these: their size bounds its writes
        self._check("g_p", g_p, torch.float64, (N, self.M))
        self._check("g_q", g_q, torch.float64, (N, self.M))
        self._check("g_w", g_w, torch.float64, (1 << self.K,))
        g_E = torch.empty((n, 6), dtype=torch.float64, device=dev) if want_E else None
        with self._on_device():
            s = torch.cuda.current_stream(self.device).cuda_stream
            rc = self._lib.dmn_grad(self._h, n, None, _ptr(lam), _ptr(Q), _ptr(E_n), _ptr(dE), _ptr(state_in),
                                    _ptr(state_out), _ptr(g_stress), _ptr(g_tangent), _ptr(g_p), _ptr(g_q),
                                    _ptr(g_w), _ptr(g_E), ctypes.c_void_p(s))
        if rc != 0:
            self._err("dmn_grad", rc)
        return g_p, g_q, g_w, g_E

    def profile(self, enable: bool):
        """Start (clearing the totals) or stop per-kernel event timing of update()."""
        with self._on_device():
            rc = self._lib.dmn_profile_enable(self._h, 1 if enable else 0)
        if rc != 0:
            self._err("dmn_profile_enable", rc)

    def profile_read(self):
        """(ms of the normals, Newton and final kernels summed over the timed updates, number of updates)."""
        ms = (ctypes.c_double * 3)()
        cnt = ctypes.c_int64()
        with self._on_device():
            rc = self._lib.dmn_profile_read(self._h, ms, ctypes.byref(cnt))
        if rc != 0:
            self._err("dmn_profile_read", rc)
        return dict(normals=ms[0], newton=ms[1], final=ms[2]), int(cnt.value)

    def profile_read_stages(self):
        """(ms of the normals, first-stage, Newton and final kernels, tree passes of the first stage and of
        the Newton kernel, number of updates), summed over the timed updates."""
        ms = (ctypes.c_double * 4)()
        ps = (ctypes.c_int64 * 2)()
        cnt = ctypes.c_int64()
        with self._on_device():
            rc = self._lib.dmn_profile_read_stages(self._h, ms, ps, ctypes.byref(cnt))
        if rc != 0:
            self._err("dmn_profile_read_stages", rc)
        return (dict(normals=ms[0], stage=ms[1], newton=ms[2], final=ms[3]),
                dict(stage=int(ps[0]), newton=int(ps[1])), int(cnt.value))

    def alloc_outputs(self, n, device):
        import torch
        return dict(state_out=torch.empty((self.state_size, n), dtype=torch.float64, device=device),
                    stress=torch.empty((n, 6), dtype=torch.float64, device=device),
                    tangent=torch.empty((n, 6, 6), dtype=torch.float64, device=device),
                    iters=torch.empty(n, dtype=torch.int32, device=device),
                    status=torch.empty(n, dtype=torch.int32, device=device))

    def update(self, lam, Q, E_n, dE, state_in, out=None, tree_id=None):
        """One material-point update; returns dict(state_out, stress, tangent, iters, status).
        tree_id: int32 CUDA tensor [n] selecting each point's tree, or None (tree 0)."""
        import torch
        n = lam.shape[0]
        dev = lam.device
        if tree_id is not None:
            self._check("tree_id", tree_id, torch.int32, (n,))
        self._check("lam", lam, torch.float64, (n, 2))
        self._check("Q", Q, torch.float64, (n, 9))
        self._check("E_n", E_n, torch.float64, (n, 6))
        self._check("dE", dE, torch.float64, (n, 6))
        self._check("state_in", state_in, torch.float64, (self.state_size, n))
        out = self.alloc_outputs(n, dev) if out is None else out
        self._check("state_out", out["state_out"], torch.float64, (self.state_size, n))
        self._check("stress", out["stress"], torch.float64, (n, 6))
        self._check("tangent", out["tangent"], torch.float64, (n, 6, 6))
        self._check("iters", out["iters"], torch.int32, (n,))
        self._check("status", out["status"], torch.int32, (n,))
        with self._on_device():
            s = torch.cuda.current_stream(self.device).cuda_stream
            rc = self._lib.dmn_update(self._h, n, _ptr(tree_id), _ptr(lam), _ptr(Q), _ptr(E_n), _ptr(dE),
                                      _ptr(state_in), _ptr(out["state_out"]), _ptr(out["stress"]),
                                      _ptr(out["tangent"]), _ptr(out["iters"]), _ptr(out["status"]),
                                      ctypes.c_void_p(s))
        if rc != 0:
            self._err("dmn_update", rc)
        return out

    def alloc_host_outputs(self, n, pin=True):
        """Output arrays of update_host in (pinned) host memory."""
        import torch
        return dict(state_out=torch.empty((self.state_size, n), dtype=torch.float64, pin_memory=pin),
                    stress=torch.empty((n, 6), dtype=torch.float64, pin_memory=pin),
                    tangent=torch.empty((n, 6, 6), dtype=torch.float64, pin_memory=pin),
                    iters=torch.empty(n, dtype=torch.int32, pin_memory=pin),
                    status=torch.empty(n, dtype=torch.int32, pin_memory=pin))

    def update_host(self, lam, Q, E_n, dE, state_in, out=None, tree_id=None, chunk=0):
        """dmn_update_host: the update of `update` with every array in host memory (CPU tensors, pinned
        for overlapped copies).  out["state_out"] may be state_in itself.  Blocks until the results are
        in the host arrays; returns out."""
        import torch
        n = lam.shape[0]
        if tree_id is not None:
            _check_host("tree_id", tree_id, torch.int32, (n,))
        _check_host("lam", lam, torch.float64, (n, 2))
        _check_host("Q", Q, torch.float64, (n, 9))
        _check_host("E_n", E_n, torch.float64, (n, 6))
        _check_host("dE", dE, torch.float64, (n, 6))
        _check_host("state_in", state_in, torch.float64, (self.state_size, n))
        out = self.alloc_host_outputs(n) if out is None else out
        _check_host("state_out", out["state_out"], torch.float64, (self.state_size, n))
        _check_host("stress", out["stress"], torch.float64, (n, 6))
        _check_host("tangent", out["tangent"], torch.float64, (n, 6, 6))
        _check_host("iters", out["iters"], torch.int32, (n,))
        _check_host("status", out["status"], torch.int32, (n,))
        with self._on_device():
            s = torch.cuda.current_stream(self.device).cuda_stream
            rc = self._lib.dmn_update_host(self._h, n, _ptr(tree_id), _ptr(lam), _ptr(Q), _ptr(E_n), _ptr(dE),
                                           _ptr(state_in), _ptr(out["state_out"]), _ptr(out["stress"]),
                                           _ptr(out["tangent"]), _ptr(out["iters"]), _ptr(out["status"]),
                                           int(chunk), ctypes.c_void_p(s))
        if rc != 0:
            self._err("dmn_update_host", rc)
        return out
