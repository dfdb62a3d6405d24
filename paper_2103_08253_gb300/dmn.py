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
EXPORTS = ("dmn_create", "dmn_destroy", "dmn_state_size", "dmn_interp_orientation", "dmn_update",
           "dmn_set_params", "dmn_grad", "dmn_profile_enable", "dmn_profile_read", "dmn_update_noalloc",
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
                ("predictor", ctypes.c_int32)]


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
    lib.dmn_interp_orientation.argtypes = [vp, i64, vp, vp, vp, vp]
    lib.dmn_interp_orientation.restype = ctypes.c_int
    lib.dmn_update.argtypes = [vp, i64, vp, vp, vp, vp, vp, vp, vp, vp, vp, vp, vp, vp]
    lib.dmn_update.restype = ctypes.c_int
    lib.dmn_update_host.argtypes = [vp, i64, vp, vp, vp, vp, vp, vp, vp, vp, vp, vp, vp, i64, vp]
    lib.dmn_update_host.restype = ctypes.c_int
    lib.dmn_set_params.argtypes = [vp, i32, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double),
                                   ctypes.POINTER(ctypes.c_double)]
    lib.dmn_set_params.restype = ctypes.c_int
    lib.dmn_grad.argtypes = [vp, i64, vp, vp, vp, vp, vp, vp, vp, vp, vp, vp, vp, vp, vp]
    lib.dmn_grad.restype = ctypes.c_int
    lib.dmn_profile_enable.argtypes = [vp, i32]
    lib.dmn_profile_enable.restype = ctypes.c_int
    lib.dmn_profile_read.argtypes = [vp, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(i64)]
    lib.dmn_profile_read.restype = ctypes.c_int
    lib.dmn_last_error.argtypes = [vp]
    lib.dmn_last_error.restype = ctypes.c_char_p
    _lib = lib
    return lib


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else None


def _check_dev(name, t, dtype, shape):
    import torch
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError("%s must be a CUDA tensor" % name)
    if t.dtype != dtype:
        raise TypeError("%s must be %s" % (name, dtype))
    if not t.is_contiguous():
        raise ValueError("%s must be contiguous" % name)
    if tuple(t.shape) != tuple(shape):
        raise ValueError("%s has shape %s, expected %s" % (name, tuple(t.shape), tuple(shape)))


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


class DMN:
    """One or several DMNs (up to 8, e.g. of different depths) on the current CUDA device.

    tree: an object with K, M, p [N, M], q [N, M], w [2^K] (numpy, paper
    ordering) and phases (two objects with kind, E, nu, sigma0, H), or a list
    of such objects (tree i is selected by tree_id == i in update()).
    precision: "f64"; "mixed" (FP32 condensation, FP64 residual and final
    sweep); "mixed-f32-tangent" (the mixed iteration, tangent from its last
    FP32 condensation).  predictor: start each Newton iteration from the last update's jumps
    extrapolated along the new strain increment (the state then holds the last jump change
    and strain increment too).  The other options are those of dmn_options."""

    def __init__(self, tree, precision: str = "f64", tol: float = 1e-12, max_iter: int = 50, block: int = 0,
                 ctas_per_sm: int = 0, line_search: bool = False, predictor: bool = False):
        import numpy as np
        self._lib = load_library()
        trees = list(tree) if isinstance(tree, (list, tuple)) else [tree]
        self.n_trees = len(trees)
        self.K, self.M = int(trees[0].K), int(trees[0].M)
        self.phases = tuple(trees[0].phases)
        dp = ctypes.POINTER(ctypes.c_double)
        descs = (TreeDesc_ * len(trees))()
        self._keep = []
        for k, tr in enumerate(trees):
            p = np.ascontiguousarray(tr.p, dtype=np.float64).reshape(-1)
            q = np.ascontiguousarray(tr.q, dtype=np.float64).reshape(-1)
            w = np.ascontiguousarray(tr.w, dtype=np.float64).reshape(-1)
            self._keep += [p, q, w]
            descs[k].K, descs[k].M = int(tr.K), int(tr.M)
            descs[k].p, descs[k].q, descs[k].w = p.ctypes.data_as(dp), q.ctypes.data_as(dp), w.ctypes.data_as(dp)
            for f, ph in enumerate(tr.phases):
                descs[k].phase[f] = Phase_(int(ph.kind), float(ph.E), float(ph.nu), float(ph.sigma0), float(ph.H),
                                           float(getattr(ph, "sigma_inf", 0.0)), float(getattr(ph, "k0", 0.0)))
        if precision not in PRECISIONS:
            raise ValueError("precision must be one of %s" % (tuple(PRECISIONS),))
        opt = Options_(float(tol), int(max_iter), PRECISIONS[precision], int(block),
                       int(ctas_per_sm), int(bool(line_search)), int(bool(predictor)))
        self.precision = precision
        self.predictor = bool(predictor)
        h = ctypes.c_void_p()
        rc = self._lib.dmn_create(descs, len(trees), ctypes.byref(opt), ctypes.byref(h))
        if rc != 0:
            raise ValueError("dmn_create failed (%d): %s" % (rc, self._lib.dmn_last_error(None).decode()))
        self._h = h
        # state fields of the arrays passed to update(); tree i uses the first tree_state_sizes[i]
        self.state_size = int(self._lib.dmn_state_size(h, -1))
        self.tree_state_sizes = [int(self._lib.dmn_state_size(h, k)) for k in range(len(trees))]

    def close(self):
        if getattr(self, "_h", None):
            self._lib.dmn_destroy(self._h)
            self._h = None

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
        _check_dev("A2", A2, torch.float64, (n, 6))
        lam = torch.empty((n, 2), dtype=torch.float64, device=A2.device) if lam is None else lam
        Q = torch.empty((n, 9), dtype=torch.float64, device=A2.device) if Q is None else Q
        _check_dev("lam", lam, torch.float64, (n, 2))
        _check_dev("Q", Q, torch.float64, (n, 9))
        s = torch.cuda.current_stream(A2.device).cuda_stream
        rc = self._lib.dmn_interp_orientation(self._h, n, _ptr(A2), _ptr(lam), _ptr(Q), ctypes.c_void_p(s))
        if rc != 0:
            self._err("dmn_interp_orientation", rc)
        return lam, Q

    def set_params(self, p, q, w, tree_id: int = 0):
        """Replace p, q, w of one tree (numpy or CPU tensors, paper ordering)."""
        import numpy as np
        arrs = [np.ascontiguousarray(np.asarray(x, dtype=np.float64)).reshape(-1) for x in (p, q, w)]
        dp = ctypes.POINTER(ctypes.c_double)
        rc = self._lib.dmn_set_params(self._h, int(tree_id), *(a.ctypes.data_as(dp) for a in arrs))
        if rc != 0:
            self._err("dmn_set_params", rc)

    def grad(self, lam, Q, E_n, dE, state_in, state_out, g_stress, g_p=None, g_q=None, g_w=None, want_E=True):
        """Adjoint of a converged update: returns (g_p [N, M], g_q [N, M], g_w [2^K], g_E [n, 6] or None),
        with g_p, g_q, g_w accumulated into the given tensors if passed."""
        import torch
        n = lam.shape[0]
        dev = lam.device
        N = (1 << self.K) - 1
        for name, t, shape in (("lam", lam, (n, 2)), ("Q", Q, (n, 9)), ("E_n", E_n, (n, 6)), ("dE", dE, (n, 6)),
                               ("state_in", state_in, (self.state_size, n)),
                               ("state_out", state_out, (self.state_size, n)), ("g_stress", g_stress, (n, 6))):
            _check_dev(name, t, torch.float64, shape)
        z = lambda *sh: torch.zeros(sh, dtype=torch.float64, device=dev)
        g_p = z(N, self.M) if g_p is None else g_p
        g_q = z(N, self.M) if g_q is None else g_q
        g_w = z(1 << self.K) if g_w is None else g_w
        g_E = torch.empty((n, 6), dtype=torch.float64, device=dev) if want_E else None
        s = torch.cuda.current_stream(dev).cuda_stream
        rc = self._lib.dmn_grad(self._h, n, None, _ptr(lam), _ptr(Q), _ptr(E_n), _ptr(dE), _ptr(state_in),
                                _ptr(state_out), _ptr(g_stress), _ptr(g_p), _ptr(g_q), _ptr(g_w), _ptr(g_E),
                                ctypes.c_void_p(s))
        if rc != 0:
            self._err("dmn_grad", rc)
        return g_p, g_q, g_w, g_E

    def profile(self, enable: bool):
        """Start (clearing the totals) or stop per-kernel event timing of update()."""
        rc = self._lib.dmn_profile_enable(self._h, 1 if enable else 0)
        if rc != 0:
            self._err("dmn_profile_enable", rc)

    def profile_read(self):
        """(ms of the normals, Newton and final kernels summed over the timed updates, number of updates)."""
        ms = (ctypes.c_double * 3)()
        cnt = ctypes.c_int64()
        rc = self._lib.dmn_profile_read(self._h, ms, ctypes.byref(cnt))
        if rc != 0:
            self._err("dmn_profile_read", rc)
        return dict(normals=ms[0], newton=ms[1], final=ms[2]), int(cnt.value)

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
            _check_dev("tree_id", tree_id, torch.int32, (n,))
        _check_dev("lam", lam, torch.float64, (n, 2))
        _check_dev("Q", Q, torch.float64, (n, 9))
        _check_dev("E_n", E_n, torch.float64, (n, 6))
        _check_dev("dE", dE, torch.float64, (n, 6))
        _check_dev("state_in", state_in, torch.float64, (self.state_size, n))
        out = self.alloc_outputs(n, dev) if out is None else out
        _check_dev("state_out", out["state_out"], torch.float64, (self.state_size, n))
        _check_dev("stress", out["stress"], torch.float64, (n, 6))
        _check_dev("tangent", out["tangent"], torch.float64, (n, 6, 6))
        _check_dev("iters", out["iters"], torch.int32, (n,))
        _check_dev("status", out["status"], torch.int32, (n,))
        s = torch.cuda.current_stream(dev).cuda_stream
        rc = self._lib.dmn_update(self._h, n, _ptr(tree_id), _ptr(lam), _ptr(Q), _ptr(E_n), _ptr(dE), _ptr(state_in),
                                  _ptr(out["state_out"]), _ptr(out["stress"]), _ptr(out["tangent"]),
                                  _ptr(out["iters"]), _ptr(out["status"]), ctypes.c_void_p(s))
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
        s = torch.cuda.current_stream().cuda_stream
        rc = self._lib.dmn_update_host(self._h, n, _ptr(tree_id), _ptr(lam), _ptr(Q), _ptr(E_n), _ptr(dE),
                                       _ptr(state_in), _ptr(out["state_out"]), _ptr(out["stress"]),
                                       _ptr(out["tangent"]), _ptr(out["iters"]), _ptr(out["status"]),
                                       int(chunk), ctypes.c_void_p(s))
        if rc != 0:
            self._err("dmn_update_host", rc)
        return out
