"""Python binding of the FE operator ABI (include/fe.h) and the FE-DMN driver.

The binding only marshals arguments: strains, internal forces, the tangent
operator, its diagonal, the preconditioned CG and the reductions all run in the
CUDA library, and every Gauss point's stress and tangent come from dmn_update.
PyTorch holds the device arrays.

`FEDMN` runs a displacement-controlled structural computation the way an FE
code drives its material routine (Sec. 5): per macroscopic Newton iteration,
the strains of the current displacement go to the DMN (from the state of the
last converged increment), the DMN's stresses give the internal forces and
its algorithmic tangents the linearised system, solved by Jacobi-PCG.
"""
from __future__ import annotations

import ctypes
import time

from . import dmn as _dmn

FE_EXPORTS = ("fe_mesh_create", "fe_mesh_destroy", "fe_num_gauss_points", "fe_num_dofs", "fe_volume",
              "fe_strain", "fe_internal_force", "fe_apply_tangent", "fe_tangent_diagonal", "fe_pcg", "fe_pcg_f32",
              "fe_dot", "fe_axpy", "fe_last_error")

_ready = False


def load_library():
    global _ready
    lib = _dmn.load_library()
    if not _ready:
        vp, i64, i32, dbl = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32, ctypes.c_double
        lib.fe_mesh_create.argtypes = [i64, i64, vp, vp, ctypes.POINTER(vp)]
        lib.fe_mesh_create.restype = ctypes.c_int
        lib.fe_mesh_destroy.argtypes = [vp]
        lib.fe_mesh_destroy.restype = None
        lib.fe_num_gauss_points.argtypes = [vp]
        lib.fe_num_gauss_points.restype = i64
        lib.fe_num_dofs.argtypes = [vp]
        lib.fe_num_dofs.restype = i64
        lib.fe_volume.argtypes = [vp]
        lib.fe_volume.restype = dbl
        for name in ("fe_strain", "fe_internal_force", "fe_tangent_diagonal"):
            getattr(lib, name).argtypes = [vp, vp, vp, vp]
            getattr(lib, name).restype = ctypes.c_int
        lib.fe_apply_tangent.argtypes = [vp, vp, vp, vp, vp]
        lib.fe_apply_tangent.restype = ctypes.c_int
        for name in ("fe_pcg", "fe_pcg_f32"):
            getattr(lib, name).argtypes = [vp, vp, vp, vp, vp, vp, dbl, i32, ctypes.POINTER(i32), ctypes.POINTER(dbl), vp]
            getattr(lib, name).restype = ctypes.c_int
        lib.fe_dot.argtypes = [vp, vp, vp, vp, ctypes.POINTER(dbl), vp]
        lib.fe_dot.restype = ctypes.c_int
        lib.fe_axpy.argtypes = [vp, dbl, vp, vp, vp, vp]
        lib.fe_axpy.restype = ctypes.c_int
        lib.fe_last_error.argtypes = [vp]
        lib.fe_last_error.restype = ctypes.c_char_p
        _ready = True
    return lib


def _p(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else None


def _stream(device):
    import torch
    return ctypes.c_void_p(torch.cuda.current_stream(device).cuda_stream)


class Hex8Mesh:
    """A hexahedral mesh on the current CUDA device (fe_mesh_create)."""

    def __init__(self, xyz, conn):
        import numpy as np
        import torch
        self._lib = load_library()
        if not torch.cuda.is_available():
            raise RuntimeError("fe.Hex8Mesh needs a CUDA device; the library has no CPU path")
        self.device = torch.device("cuda", torch.cuda.current_device())
        xyz = np.ascontiguousarray(xyz, dtype=np.float64)
        conn = np.ascontiguousarray(conn, dtype=np.int32)
        if xyz.ndim != 2 or xyz.shape[1] != 3 or conn.ndim != 2 or conn.shape[1] != 8:
            raise ValueError("xyz must be [n_nodes, 3] and conn [n_elem, 8]")
        h = ctypes.c_void_p()
        with torch.cuda.device(self.device):
            rc = self._lib.fe_mesh_create(xyz.shape[0], conn.shape[0], xyz.ctypes.data_as(ctypes.c_void_p),
                                          conn.ctypes.data_as(ctypes.c_void_p), ctypes.byref(h))
        if rc != 0:
            raise ValueError("fe_mesh_create failed (%d): %s" % (rc, self._lib.fe_last_error(None).decode()))
        self._h = h
        self.n_gp = int(self._lib.fe_num_gauss_points(h))
        self.n_dofs = int(self._lib.fe_num_dofs(h))
        self.volume = float(self._lib.fe_volume(h))

    def _check(self, name, rc):
        if rc != 0:
            raise RuntimeError("%s failed (%d): %s" % (name, rc, self._lib.fe_last_error(self._h).decode()))

    def _args(self, **arrays):
        """Check the arrays of one call against the layouts of fe.h (FP64, contiguous, on the mesh's
        device): u-like names are [n_dofs], E/sigma [n_gp, 6], C [n_gp, 6, 6] or [n_gp, 36]; None
        (an optional `free`) is passed through."""
        import torch
        shapes = {"vec": (self.n_dofs,), "gp6": (self.n_gp, 6), "C": [(self.n_gp, 6, 6), (self.n_gp, 36)]}
        for name, (t, kind) in arrays.items():
            if t is not None:
                _dmn._check_dev(name, t, torch.float64, shapes[kind], self.device)

    def _call(self, name, *args):
        import torch
        with torch.cuda.device(self.device):
            self._check(name, getattr(self._lib, name)(self._h, *args, _stream(self.device)))

    def _vec(self):
        import torch
        return torch.empty(self.n_dofs, dtype=torch.float64, device=self.device)

    def strain(self, u, out=None):
        import torch
        out = torch.empty((self.n_gp, 6), dtype=torch.float64, device=self.device) if out is None else out
        self._args(u=(u, "vec"), E=(out, "gp6"))
        self._call("fe_strain", _p(u), _p(out))
        return out

    def internal_force(self, sigma, out=None):
        out = self._vec() if out is None else out
        self._args(sigma=(sigma, "gp6"), f=(out, "vec"))
        self._call("fe_internal_force", _p(sigma), _p(out))
        return out

    def apply_tangent(self, C, v, out=None):
        out = self._vec() if out is None else out
        self._args(C=(C, "C"), v=(v, "vec"), Kv=(out, "vec"))
        self._call("fe_apply_tangent", _p(C), _p(v), _p(out))
        return out

    def tangent_diagonal(self, C, out=None):
        out = self._vec() if out is None else out
        self._args(C=(C, "C"), diag=(out, "vec"))
        self._call("fe_tangent_diagonal", _p(C), _p(out))
        return out

    def pcg(self, C, free, diag, b, x, rtol=1e-8, max_iter=20000, f32=False):
        """Jacobi-PCG on the free dofs (f32: products K p in FP32, fe_pcg_f32); returns
        (iterations, relative residual)."""
        self._args(C=(C, "C"), free=(free, "vec"), diag=(diag, "vec"), b=(b, "vec"), x=(x, "vec"))
        it = ctypes.c_int32()
        rr = ctypes.c_double()
        self._call("fe_pcg_f32" if f32 else "fe_pcg", _p(C), _p(free), _p(diag), _p(b), _p(x), float(rtol),
                   int(max_iter), ctypes.byref(it), ctypes.byref(rr))
        return it.value, rr.value

    def dot(self, a, b, free=None):
        self._args(a=(a, "vec"), b=(b, "vec"), free=(free, "vec"))
        out = ctypes.c_double()
        self._call("fe_dot", _p(a), _p(b), _p(free), ctypes.byref(out))
        return out.value

    def axpy(self, alpha, x, y, free=None):
        self._args(x=(x, "vec"), y=(y, "vec"), free=(free, "vec"))
        self._call("fe_axpy", float(alpha), _p(x), _p(free), _p(y))

    def close(self):
        if getattr(self, "_h", None):
            import torch
            with torch.cuda.device(self.device):
                self._lib.fe_mesh_destroy(self._h)
            self._h = None

    def __del__(self):
        import sys
        if sys is None or sys.is_finalizing():
            return
        try:
            self.close()
        except Exception:
            pass


class FEDMN:
    """Displacement-controlled FE-DMN computation on one GPU.

    mesh: object with xyz [n_nodes, 3], conn [n_elem, 8], fixed [n_dofs] bool, pull [n_dofs]
    (the prescribed displacement of a fixed dof is delta * pull); A2 [n_elem, 6] fiber
    orientation per element (all 8 Gauss points share it); tree: DMN parameters.
    predictor: the DMN's extrapolated start (every macro Newton iteration of an increment
    extrapolates from the last committed increment)."""

    def __init__(self, mesh, tree, A2, precision="f64", newton_rtol=1e-6, max_newton=20, cg_rtol=1e-8,
                 cg_max_iter=50000, line_search=True, block=0, ctas_per_sm=0, cg_f32=False, predictor=False):
        import numpy as np
        import torch
        self.dev = torch.device("cuda", torch.cuda.current_device())
        self.mesh = Hex8Mesh(mesh.xyz, mesh.conn)
        self.m = _dmn.DMN(tree, precision=precision, block=block, ctas_per_sm=ctas_per_sm, line_search=line_search,
                          predictor=predictor)
        n, dev = self.mesh.n_gp, self.dev
        A2g = torch.from_numpy(np.ascontiguousarray(np.repeat(np.asarray(A2, dtype=np.float64), 8, axis=0))).to(dev)
        self.lam, self.Q = self.m.interp_orientation(A2g)
        S = self.m.state_size
        self.state = torch.zeros((S, n), dtype=torch.float64, device=dev)
        self.E_n = torch.zeros((n, 6), dtype=torch.float64, device=dev)
        self.E = torch.empty_like(self.E_n)
        self.dE = torch.empty_like(self.E_n)
        self.out = self.m.alloc_outputs(n, dev)
        nd = self.mesh.n_dofs
        self.free = torch.from_numpy((~np.asarray(mesh.fixed, dtype=bool)).astype(np.float64)).to(dev)
        self.pull = torch.from_numpy(np.asarray(mesh.pull, dtype=np.float64)).to(dev)
        affine = getattr(mesh, "affine", None)
        self.affine = None if affine is None else torch.from_numpy(np.asarray(affine, dtype=np.float64)).to(dev)
        self.u = torch.zeros(nd, dtype=torch.float64, device=dev)
        self.u_last_inc = torch.zeros(nd, dtype=torch.float64, device=dev)   # u_n - u_{n-1}
        self.delta_n, self.ddelta_n = 0.0, 0.0
        self.f = torch.empty(nd, dtype=torch.float64, device=dev)
        self.du = torch.empty(nd, dtype=torch.float64, device=dev)
        self.diag = torch.empty(nd, dtype=torch.float64, device=dev)
        self.newton_rtol, self.max_newton = newton_rtol, max_newton
        self.cg_rtol, self.cg_max_iter, self.cg_f32 = cg_rtol, cg_max_iter, cg_f32
        self.timing = dict(dmn_s=0.0, fe_s=0.0, dmn_calls=0, cg_iters=0)

    def increment(self, delta):
        """Prescribe delta on the loaded face and iterate to equilibrium; commits the DMN state.
        Returns dict(newton, cg_iters, residual, reaction, dmn_status_bad)."""
        import torch
        u_n = self.u.clone()
        # starting point: extrapolate the last increment, or for the first one a field that meets the
        # boundary conditions with uniform strain; then the prescribed values on the fixed dofs
        if self.ddelta_n > 0.0:
            self.mesh.axpy((delta - self.delta_n) / self.ddelta_n, self.u_last_inc, self.u)
        elif self.affine is not None:
            self.u.zero_()
            self.mesh.axpy(delta, self.affine, self.u)
        fx = 1.0 - self.free
        self.u.mul_(self.free).add_(fx * self.pull * delta)
        cg_total, hist = 0, []
        for it in range(self.max_newton + 1):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            self.mesh.strain(self.u, self.E)
            torch.sub(self.E, self.E_n, out=self.dE)
            self.m.update(self.lam, self.Q, self.E_n, self.dE, self.state, out=self.out)
            torch.cuda.synchronize()
            t1 = time.perf_counter()
            self.timing["dmn_s"] += t1 - t0
            self.timing["dmn_calls"] += 1
            self.mesh.internal_force(self.out["stress"], self.f)
            rn = self.mesh.dot(self.f, self.f, self.free) ** 0.5
            fn = self.mesh.dot(self.f, self.f) ** 0.5
            hist.append(rn / fn if fn > 0 else 0.0)
            if rn <= self.newton_rtol * fn or it == self.max_newton:
                self.timing["fe_s"] += time.perf_counter() - t1
                break
            self.mesh.tangent_diagonal(self.out["tangent"], self.diag)
            k, _ = self.mesh.pcg(self.out["tangent"], self.free, self.diag, self.f, self.du, self.cg_rtol,
                                 self.cg_max_iter, f32=self.cg_f32)
            cg_total += k
            self.mesh.axpy(-1.0, self.du, self.u, self.free)
            torch.cuda.synchronize()
            self.timing["fe_s"] += time.perf_counter() - t1
        self.timing["cg_iters"] += cg_total
        bad = int((self.out["status"] != 0).sum().item())
        reaction = self.mesh.dot(self.f, self.pull)
        # commit: the converged strain and state become those of the next increment's start
        self.u_last_inc.copy_(self.u)
        self.mesh.axpy(-1.0, u_n, self.u_last_inc)
        self.ddelta_n, self.delta_n = delta - self.delta_n, delta
        self.E_n.copy_(self.E)
        self.state, self.out["state_out"] = self.out["state_out"], self.state
        return dict(newton=it, cg_iters=cg_total, residual=hist, reaction=reaction, dmn_status_bad=bad,
                    converged=hist[-1] <= self.newton_rtol)

    def close(self):
        self.m.close()
        self.mesh.close()
