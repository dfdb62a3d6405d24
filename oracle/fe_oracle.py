"""Plain CPU oracle of the FE-DMN coupling: small-strain 8-node hexahedra,
2 x 2 x 2 Gauss points, a global sparse tangent assembled explicitly and
solved directly, Newton's method on the macroscopic equilibrium, every Gauss
point's stress and tangent from the DMN oracle (oracle.update).

TEST INFRASTRUCTURE: only the tests, the smoke check and the bench's CPU
baseline use this module.  It shares no code with the CUDA path.

The paper couples its DMN to an FE code through the material-subroutine
interface (Sec. 5): per Gauss point the FE code passes the strain increment
and the stored state and receives stress and algorithmic tangent.  The FE side
here is the textbook displacement method (virtual work with B matrices), written
out without any blocking or matrix-free tricks so that it can be checked by eye.

Conventions (those of the CUDA FE operator's header): dofs [n_nodes][3];
element nodes in the order (-,-,-), (+,-,-), (+,+,-), (-,+,-), then +zeta;
Gauss point g = gx + 2 gy + 4 gz at -1/sqrt(3), +1/sqrt(3), weight 1;
strain as the Mandel vector (11, 22, 33, sqrt2 23, sqrt2 13, sqrt2 12).
"""
from __future__ import annotations

import math

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

import oracle

NODE_SIGNS = np.array([[-1, -1, -1], [1, -1, -1], [1, 1, -1], [-1, 1, -1],
                       [-1, -1, 1], [1, -1, 1], [1, 1, 1], [-1, 1, 1]], dtype=np.float64)


def gauss_points():
    g = 1.0 / math.sqrt(3.0)
    return np.array([[(-g, g)[k & 1], (-g, g)[(k >> 1) & 1], (-g, g)[(k >> 2) & 1]] for k in range(8)])


def shape_derivatives(xi):
    """dN_a / dxi_k [8, 3] of the trilinear shape functions N_a = prod_k (1 + s_ak xi_k) / 8."""
    out = np.empty((8, 3))
    for a in range(8):
        f = 1.0 + NODE_SIGNS[a] * xi
        out[a, 0] = NODE_SIGNS[a, 0] * f[1] * f[2] / 8.0
        out[a, 1] = NODE_SIGNS[a, 1] * f[0] * f[2] / 8.0
        out[a, 2] = NODE_SIGNS[a, 2] * f[0] * f[1] / 8.0
    return out


def b_matrix(dNdx):
    """Mandel strain-displacement matrix [6, 24] (columns: node a, component i -> 3a + i)."""
    s = 1.0 / math.sqrt(2.0)
    B = np.zeros((6, 24))
    for a in range(8):
        gx, gy, gz = dNdx[a]
        B[0, 3 * a + 0] = gx
        B[1, 3 * a + 1] = gy
        B[2, 3 * a + 2] = gz
        B[3, 3 * a + 1] = s * gz; B[3, 3 * a + 2] = s * gy     # (u2,3 + u3,2) / sqrt2
        B[4, 3 * a + 0] = s * gz; B[4, 3 * a + 2] = s * gx     # (u1,3 + u3,1) / sqrt2
        B[5, 3 * a + 0] = s * gy; B[5, 3 * a + 1] = s * gx     # (u1,2 + u2,1) / sqrt2
    return B


class Mesh:
    """B matrices and integration weights of every Gauss point (index 8 e + g)."""

    def __init__(self, xyz, conn):
        self.xyz = np.asarray(xyz, dtype=np.float64)
        self.conn = np.asarray(conn, dtype=np.int64)
        ne = self.conn.shape[0]
        self.n_nodes = self.xyz.shape[0]
        self.n_dofs = 3 * self.n_nodes
        self.n_gp = 8 * ne
        dN = [shape_derivatives(xi) for xi in gauss_points()]
        self.B = np.empty((self.n_gp, 6, 24))
        self.w = np.empty(self.n_gp)
        for e in range(ne):
            X = self.xyz[self.conn[e]]                 # [8, 3]
            for g in range(8):
                J = X.T @ dN[g]                        # J[i, k] = dx_i / dxi_k
                det = np.linalg.det(J)
                if not det > 0:
                    raise ValueError("element %d: det(J) = %g" % (e, det))
                dNdx = dN[g] @ np.linalg.inv(J)        # dN_a/dx_i = dN_a/dxi_k dxi_k/dx_i
                self.B[8 * e + g] = b_matrix(dNdx)
                self.w[8 * e + g] = det
        self.dofs = (3 * self.conn[:, :, None] + np.arange(3)[None, None, :]).reshape(ne, 24)

    def volume(self):
        return float(self.w.sum())

    def gp_dofs(self, k):
        return self.dofs[k // 8]

    def strain(self, u):
        """[n_gp, 6]"""
        ue = u[self.dofs]                              # [ne, 24]
        return np.einsum("gij,gj->gi", self.B, np.repeat(ue, 8, axis=0))

    def internal_force(self, sig):
        f = np.zeros(self.n_dofs)
        fe = np.einsum("gji,gj,g->gi", self.B, sig, self.w)   # B^T sigma w, [n_gp, 24]
        np.add.at(f, np.repeat(self.dofs, 8, axis=0), fe)
        return f

    def stiffness(self, C):
        """Global sparse K = sum B^T C B w (C [n_gp, 6, 6])."""
        ke = np.einsum("gki,gkl,glj,g->gij", self.B, C, self.B, self.w)   # [n_gp, 24, 24]
        d = np.repeat(self.dofs, 8, axis=0)
        rows = np.repeat(d[:, :, None], 24, axis=2).ravel()
        cols = np.repeat(d[:, None, :], 24, axis=1).ravel()
        return sp.csr_matrix((ke.ravel(), (rows, cols)), shape=(self.n_dofs, self.n_dofs))


def solve_free(K, rhs, fixed):
    """x with x_fixed = 0 and K_ff x_f = rhs_f (sparse direct)."""
    free = ~fixed
    x = np.zeros(K.shape[0])
    Kff = K[free][:, free].tocsc()
    x[free] = spla.spsolve(Kff, rhs[free])
    return x


def run_fe_dmn(mesh, tree, lam, Q, fixed, pull, deltas, affine=None, rtol=1e-8, max_newton=20, line_search=True):
    """Displacement-controlled FE-DMN run: for each prescribed displacement delta of the
    loaded face, Newton's method on f_int(u) = 0 at the free dofs, the DMN oracle at every
    Gauss point (E_n and state committed at each converged increment).

    Starting point of each increment: the first from delta * affine (a displacement field
    meeting the boundary conditions, if given), later ones by extrapolating the last
    increment, u_n + (d delta_k / d delta_{k-1}) (u_n - u_{n-1}); the prescribed dofs then
    take delta * pull.  The DMN's own Newton uses the backtracking line search by default.
    Returns a list of per-increment dicts (u, reaction, newton iterations, stress)."""
    n = mesh.n_gp
    S = oracle.state_size(tree.K, tree.phases)
    state = np.zeros((S, n))
    E_n = np.zeros((n, 6))
    u = np.zeros(mesh.n_dofs)
    u_prev = u.copy()
    d_prev, dd_prev = 0.0, 0.0
    out = []
    for delta in deltas:
        if dd_prev > 0.0:
            u_start = u + (delta - d_prev) / dd_prev * (u - u_prev)
        elif affine is not None:
            u_start = delta * np.asarray(affine, dtype=np.float64)
        else:
            u_start = u.copy()
        u_prev = u
        u = np.where(fixed, delta * pull, u_start)
        for it in range(max_newton + 1):
            E = mesh.strain(u)
            st_new, sig, C, dit, stat, _ = oracle.update(tree, lam, Q, E_n, E - E_n, state, line_search=line_search)
            if (stat != 0).any():
                raise RuntimeError("DMN oracle did not converge at %d points" % int((stat != 0).sum()))
            f = mesh.internal_force(sig)
            rn = np.linalg.norm(f[~fixed])
            if rn <= rtol * np.linalg.norm(f):
                break
            if it == max_newton:
                raise RuntimeError("FE Newton did not converge")
            K = mesh.stiffness(C)
            u = u - solve_free(K, f, fixed)
        state, E_n = st_new, E
        dd_prev, d_prev = delta - d_prev, delta
        out.append(dict(u=u.copy(), reaction=float(f @ pull), newton=it, stress=sig.copy()))
    return out
