"""Plain FP64 CPU oracle of the DMN material-point update (test infrastructure).

Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  It shares no code with the CUDA path.
The arithmetic lives in ``dmn_oracle.c`` (plain C + OpenMP over points); this
module builds it with gcc and marshals numpy arrays through ctypes.

Every function states the passage of the paper it follows in the C source.
Parity is pinned by the ``-m "not gpu"`` tests in ``tests/test_oracle_*.py``
against closed forms, textbook routines and the depth-3 operator printed in the
paper.  Pinned-status of each function is listed in the module docstring of
those tests; nothing here is "parity unpinned".
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import sys

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "dmn_oracle.c")
_LIB = os.path.join(_HERE, "_build", "liboracle_dmn.so")
_lib = None

_D = ctypes.POINTER(ctypes.c_double)
_I = ctypes.POINTER(ctypes.c_int)


def build(force: bool = False) -> str:
    """Compile the oracle with the host gcc (-O2, OpenMP); returns the .so path."""
    os.makedirs(os.path.dirname(_LIB), exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + ".tmp%d" % os.getpid()
        cmd = ["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-std=c11", "-o", tmp, _SRC, "-lm"]
        subprocess.check_call(cmd)
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        lib.oracle_update.argtypes = [ctypes.c_int, ctypes.c_int, _D, _D, _D, _D, ctypes.c_double, ctypes.c_int,
                                      ctypes.c_int, ctypes.c_long, _D, _D, _D, _D, _D, _D, _D, _D, _I, _I, _D,
                                      ctypes.c_int]
        lib.oracle_normals.argtypes = [ctypes.c_int, ctypes.c_int, _D, _D, ctypes.c_double, ctypes.c_double, _D]
        lib.oracle_barycentric.argtypes = [ctypes.c_double, ctypes.c_double, _D]
        lib.oracle_gradient_operator.argtypes = [ctypes.c_int, ctypes.c_int, _D, _D, _D, ctypes.c_double,
                                                 ctypes.c_double, _D]
        lib.oracle_newton_system.argtypes = [ctypes.c_int, ctypes.c_int, _D, _D, _D, _D, ctypes.c_double,
                                             ctypes.c_double, _D, _D, _D, _D, _D, _D, _D, _D, _D]
        lib.oracle_phase_law.argtypes = [_D, _D, _D, _D, _D, _D]
        lib.oracle_rotate.argtypes = [_D, _D, _D, _D, _D]
        lib.oracle_interp_orientation.argtypes = [ctypes.c_long, _D, _D, _D]
        lib.oracle_state_size.argtypes = [ctypes.c_int, _D]
        lib.oracle_state_size_w.argtypes = [ctypes.c_int, _D, _D]
        lib.oracle_eval_dual.argtypes = [ctypes.c_int, ctypes.c_int, _D, _D, _D, _D, _D, _D, _D, ctypes.c_double,
                                         ctypes.c_double, _D, _D, _D, _D, _D, ctypes.c_int, _D, _D, _D, _D, _D, _D]
        lib.oracle_gradient.argtypes = [ctypes.c_int, ctypes.c_int, _D, _D, _D, _D, ctypes.c_double,
                                        ctypes.c_double, _D, _D, _D, _D, _D, _D, _D, _D, _D]
        _lib = lib
    return _lib


def _p(a):
    return a.ctypes.data_as(_D)


def _f64(a, shape=None):
    a = np.ascontiguousarray(np.asarray(a, dtype=np.float64))
    if shape is not None:
        a = a.reshape(shape)
    return a


def phases_array(phases) -> np.ndarray:
    """(kind, E, nu, sigma0, H, sigma_inf, k0) of phase 1 then phase 2."""
    return np.array([_phase_row(ph) for ph in phases], dtype=np.float64).reshape(14)


def _phase_row(ph):
    return [ph.kind, ph.E, ph.nu, ph.sigma0, ph.H, getattr(ph, "sigma_inf", 0.0), getattr(ph, "k0", 0.0)]


def state_size(K: int, phases, w=None) -> int:
    """Doubles of state per point; with leaf weights w, of the compressed tree (weightless
    leaves and the laminates without weight on both sides carry no state)."""
    m = phases_array(phases)
    if w is None:
        return int(_load().oracle_state_size(K, _p(m)))
    return int(_load().oracle_state_size_w(K, _p(m), _p(_f64(w))))


PRED_TRIES = 6   # corrections from the extrapolated start before a restart from a^n


def jump_fields(tree):
    """(S0, J): state fields of the tree (its compressed form when weights are zero) and
    how many of them, the last ones, are laminate jumps (3 per remaining laminate).  The
    others are 6 per remaining inelastic leaf."""
    S0 = state_size(tree.K, tree.phases, tree.w)
    w = np.asarray(tree.w, dtype=np.float64)
    inel = [int(ph.kind) != 0 for ph in tree.phases]
    nz = sum(1 for leaf in range(w.size) if w[leaf] > 0 and inel[leaf % 2])
    return S0, S0 - 6 * nz


def update(tree, lam, Q, E_n, dE, state_in, tol=1e-12, max_iter=50, line_search=False, nthreads=None,
           predictor=False):
    """One material-point update of n points (Sec. 3.2): returns
    (state_out, stress [n,6], tangent [n,6,6], iters [n], status [n], yield_gap [n]).

    state_in is field-major [S, n]; stress/tangent are in the global frame.  The Newton
    iteration starts from the jumps held in state_in (Sec. 4.7: the last converged ones).

    predictor: the extrapolated start of this library (the paper has none).  state_in then
    carries J more fields (the last update's jump change) and 6 (its strain increment
    dE_prev) after the S0 of the tree, J and S0 as given by jump_fields.  The iteration
    starts from a^n + rho (jump change), rho = (dE . dE_prev) / (dE_prev . dE_prev)
    clipped to [0, 1], or 0 when dE_prev = 0 or the ratio is not finite.  A point with
    rho > 0 gets PRED_TRIES corrections; if it has not converged by then (any status but
    0), it starts again from a^n with max_iter corrections, and its iteration count is the
    sum of both attempts.  state_out carries this update's jump change and dE in the same
    places."""
    if predictor:
        S0, J = jump_fields(tree)
        state_in = _f64(state_in)
        assert state_in.shape[0] == S0 + J + 6, (state_in.shape, S0, J)
        a_n = state_in[S0 - J:S0]
        change = state_in[S0:S0 + J]
        dE_prev = state_in[S0 + J:]
        dE = _f64(dE)
        num = np.einsum("ni,in->n", dE, dE_prev)
        den = (dE_prev * dE_prev).sum(axis=0)
        with np.errstate(all="ignore"):
            r = num / den
            rho = np.where((den > 0) & np.isfinite(r), np.clip(r, 0.0, 1.0), 0.0)
        paper = np.array(state_in[:S0])
        start = paper.copy()
        start[S0 - J:] = a_n + rho[None, :] * change
        ext = rho > 0
        lam = _f64(lam); Q = _f64(Q); E_n = _f64(E_n)
        res = list(update(tree, lam, Q, E_n, dE, paper, tol, max_iter, line_search, nthreads))
        if ext.any():   # the extrapolated attempts, and restarts of those that failed
            x = np.nonzero(ext)[0]
            r1 = update(tree, lam[x], Q[x], E_n[x], dE[x], start[:, x], tol, PRED_TRIES, line_search, nthreads)
            fail = x[r1[4] != 0]
            keep = r1[4] == 0
            for k, v in enumerate(r1):
                if v.ndim == 2 and v.shape[0] != len(x):      # field-major state
                    res[k][:, x[keep]] = v[:, keep]
                else:
                    res[k][x[keep]] = v[keep]
            if fail.size:
                r2 = update(tree, lam[fail], Q[fail], E_n[fail], dE[fail], paper[:, fail], tol, max_iter,
                            line_search, nthreads)
                for k, v in enumerate(r2):
                    if v.ndim == 2 and v.shape[0] != len(fail):
                        res[k][:, fail] = v
                    else:
                        res[k][fail] = v
                res[3][fail] += r1[3][r1[4] != 0]
        st = res[0]
        return (np.vstack([st, st[S0 - J:] - a_n, dE.T]),) + tuple(res[1:])
    lib = _load()
    lam = _f64(lam); Q = _f64(Q); E_n = _f64(E_n); dE = _f64(dE); state_in = _f64(state_in)
    n = lam.shape[0]
    S = state_size(tree.K, tree.phases, tree.w)
    assert state_in.shape == (S, n), (state_in.shape, S, n)
    p = _f64(tree.p); q = _f64(tree.q); w = _f64(tree.w); m = phases_array(tree.phases)
    state_out = np.empty_like(state_in)
    stress = np.empty((n, 6)); tangent = np.empty((n, 6, 6))
    iters = np.empty(n, dtype=np.int32); status = np.empty(n, dtype=np.int32); gap = np.empty(n)
    if nthreads is None:
        nthreads = os.cpu_count() or 1
    rc = lib.oracle_update(tree.K, tree.M, _p(p), _p(q), _p(w), _p(m), float(tol), int(max_iter),
                           int(bool(line_search)), n, _p(lam), _p(Q), _p(E_n), _p(dE), _p(state_in),
                           _p(state_out), _p(stress), _p(tangent), iters.ctypes.data_as(_I),
                           status.ctypes.data_as(_I), _p(gap), int(nthreads))
    if rc != 0:
        raise ValueError("oracle_update rejected its arguments (rc=%d)" % rc)
    return state_out, stress, tangent, iters, status, gap


def normals(tree, lam1, lam2):
    """Normals of all laminates [N, 3] in the paper's ordering (Sec. 2.3)."""
    N = (1 << tree.K) - 1
    out = np.empty((N, 3))
    p = _f64(tree.p); q = _f64(tree.q)
    rc = _load().oracle_normals(tree.K, tree.M, _p(p), _p(q), float(lam1), float(lam2), _p(out))
    assert rc == 0
    return out


def barycentric(lam1, lam2):
    out = np.empty(3)
    _load().oracle_barycentric(float(lam1), float(lam2), _p(out))
    return out


def gradient_operator(tree, lam1, lam2):
    """Dense A [6 * 2^K, 3 * (2^K - 1)] (Sec. 3.2)."""
    L = 1 << tree.K
    N = L - 1
    A = np.empty((6 * L, 3 * N))
    p = _f64(tree.p); q = _f64(tree.q); w = _f64(tree.w)
    rc = _load().oracle_gradient_operator(tree.K, tree.M, _p(p), _p(q), _p(w), float(lam1), float(lam2), _p(A))
    assert rc == 0
    return A


def newton_system(tree, lam1, lam2, E_loc, a, z_n):
    """J (dense), R, da = -J^{-1} R (oracle's Cholesky), leaf eps, sigma and
    sigma_bar at one iterate.  z_n: [2^K, 7] per leaf (alpha_bar, ep6); a: the jumps of
    the (compressed) tree's laminates, as in the state."""
    L = 1 << tree.K
    n_a = np.asarray(a).size
    J = np.empty((n_a, n_a)); R = np.empty(n_a); da = np.empty(n_a)
    eps = np.empty((L, 6)); sig = np.empty((L, 6)); sbar = np.empty(6)
    p = _f64(tree.p); q = _f64(tree.q); w = _f64(tree.w); m = phases_array(tree.phases)
    rc = _load().oracle_newton_system(tree.K, tree.M, _p(p), _p(q), _p(w), _p(m), float(lam1), float(lam2),
                                      _p(_f64(E_loc)), _p(_f64(a)), _p(_f64(z_n)), _p(J), _p(R), _p(da),
                                      _p(eps), _p(sig), _p(sbar))
    return dict(J=J, R=R, da=da, eps=eps, sig=sig, sbar=sbar, rc=rc)


def phase_law(phase, eps, z_n=None):
    """One leaf: (sigma [6], D [6,6], z_new [7]); z = (alpha_bar, ep6 Mandel)."""
    ph = np.array(_phase_row(phase), dtype=np.float64)
    z = np.zeros(7) if z_n is None else _f64(z_n)
    sig = np.empty(6); D = np.empty((6, 6)); zn = np.empty(7)
    _load().oracle_phase_law(_p(ph), _p(_f64(eps)), _p(z), _p(sig), _p(D), _p(zn))
    return sig, D, zn


def rotate(Q, C_loc, v_loc):
    """Global-frame Mandel stiffness and symmetric tensor from local ones."""
    Cg = np.empty((6, 6)); vg = np.empty(6)
    _load().oracle_rotate(_p(_f64(Q)), _p(_f64(C_loc)), _p(_f64(v_loc)), _p(Cg), _p(vg))
    return Cg, vg


def interp_orientation(A2):
    """(lam [n,2], Q [n,9]) from A2 [n,6] (Eq. of the eigen decomposition)."""
    A2 = _f64(A2)
    n = A2.shape[0]
    lam = np.empty((n, 2)); Q = np.empty((n, 9))
    _load().oracle_interp_orientation(n, _p(A2), _p(lam), _p(Q))
    return lam, Q


__all__ = ["build", "update", "normals", "barycentric", "gradient_operator", "newton_system", "phase_law",
           "rotate", "interp_orientation", "state_size", "phases_array", "eval_dual", "gradient_ift"]
if "--build" in sys.argv[1:]:  # pragma: no cover
    print(build(force=True))


def _with_params(tree, p=None, q=None, w=None):
    import copy
    t = copy.copy(tree)
    if p is not None:
        t.p = p
    if q is not None:
        t.q = q
    if w is not None:
        t.w = w
    return t


def eval_dual(tree, lam1, lam2, E_loc, a, z_n, dp=None, dq=None, dw=None, dE=None, da=None, tangent=False):
    """Exact directional derivatives at fixed z^n (local frame; forward-mode dual numbers of
    dmn_oracle.c): R = A^T W sigma, sigma_bar and, with tangent=True, the algorithmic tangent C,
    at (p, q, w, E_loc, a), each with its derivative along (dp, dq, dw, dE, da) (zeros where
    None).  w is the weight vector as given (before normalisation); z_n [2^K, 7] per leaf."""
    p = _f64(tree.p); q = _f64(tree.q); w = _f64(tree.w); m = phases_array(tree.phases)
    a = _f64(a)
    n_a = a.size
    z = lambda x, like: _f64(np.zeros_like(like) if x is None else x)
    dp, dq, dw = z(dp, p), z(dq, q), z(dw, w)
    dE, da = z(dE, np.zeros(6)), z(da, a)
    R = np.empty(max(n_a, 1)); dR = np.empty(max(n_a, 1)); sb = np.empty(6); dsb = np.empty(6)
    C = np.empty(36); dC = np.empty(36)
    rc = _load().oracle_eval_dual(tree.K, tree.M, _p(p), _p(q), _p(w), _p(m), _p(dp), _p(dq), _p(dw),
                                  float(lam1), float(lam2), _p(_f64(E_loc)), _p(dE), _p(a), _p(da),
                                  _p(_f64(z_n)), int(bool(tangent)), _p(R), _p(dR), _p(sb), _p(dsb), _p(C), _p(dC))
    if rc != 0:
        raise ValueError("oracle_eval_dual failed (rc=%d)" % rc)
    out = dict(R=R[:n_a], dR=dR[:n_a], sbar=sb, dsbar=dsb)
    if tangent:
        out.update(C=C.reshape(6, 6), dC=dC.reshape(6, 6))
    return out


def gradient_ift(tree, lam, Q, E_glob, a_star, z_leaf, g_glob, directions=None, G_glob=None):
    """Gradient of L = g . sigma_bar (+ G : C with a tangent seed G) at the converged jumps
    a_star of one point, by the implicit function theorem applied to R(a, theta) = A^T W sigma = 0
    (Sec. 3.2):
        J lam = (d sigma_bar/d a)^T g + (dC/da)^T : G,   J = A^T W D A,
        dL/dtheta = g . d sigma_bar/d theta|_a + G : dC/d theta|_a - lam . dR/d theta|_a.
    Every partial derivative is exact (dual numbers, oracle_gradient in dmn_oracle.c) and the
    solve uses the oracle's Cholesky factor of J.  theta = (p, q, w) with w the leaf weights
    before normalisation, and the macro strain E.  g_glob [6] and G_glob [6, 6] (or None) are
    in the global frame; returns dict(p, q, w, E) with E in the global frame.

    directions: a list of (dp, dq, dw) triples; returns the directional derivatives by the
    forward route instead (tangent-linear sensitivities: da = -J^-1 dR/dtheta, then the total
    derivative of sigma_bar and C along (dtheta, da) from one more dual evaluation)."""
    lam = np.asarray(lam, dtype=np.float64)
    Qm = np.asarray(Q, dtype=np.float64).reshape(3, 3)
    _, E_loc = rotate(Qm.T, np.zeros((6, 6)), E_glob)
    _, g_loc = rotate(Qm.T, np.zeros((6, 6)), g_glob)
    G_loc = None
    if G_glob is not None:
        G_loc, _ = rotate(Qm.T, np.asarray(G_glob, dtype=np.float64).reshape(6, 6), np.zeros(6))
    a_star = _f64(a_star)
    z_leaf = _f64(z_leaf)
    if directions is not None:
        J = newton_system(tree, lam[0], lam[1], E_loc, a_star, z_leaf)["J"]
        vals = []
        for dp, dq, dw in directions:
            r1 = eval_dual(tree, lam[0], lam[1], E_loc, a_star, z_leaf, dp, dq, dw)
            da = -np.linalg.solve(J, r1["dR"])
            r2 = eval_dual(tree, lam[0], lam[1], E_loc, a_star, z_leaf, dp, dq, dw, da=da,
                           tangent=G_loc is not None)
            v = g_loc @ r2["dsbar"]
            if G_loc is not None:
                v += (G_loc * r2["dC"]).sum()
            vals.append(v)
        return vals
    p = _f64(tree.p); q = _f64(tree.q); w = _f64(tree.w); m = phases_array(tree.phases)
    gp = np.empty_like(p); gq = np.empty_like(q); gw = np.empty_like(w); gE = np.empty(6)
    Gp = _p(_f64(G_loc)) if G_loc is not None else None
    rc = _load().oracle_gradient(tree.K, tree.M, _p(p), _p(q), _p(w), _p(m), float(lam[0]), float(lam[1]),
                                 _p(_f64(E_loc)), _p(a_star), _p(z_leaf), _p(_f64(g_loc)), Gp, _p(gp), _p(gq),
                                 _p(gw), _p(gE))
    if rc != 0:
        raise ValueError("oracle_gradient failed (rc=%d)" % rc)
    _, gE_glob = rotate(Qm, np.zeros((6, 6)), gE)
    return dict(p=gp, q=gq, w=gw, E=gE_glob)


def leaf_states(tree, state, i):
    """z^n of every leaf of point i, [2^K, 7] (alpha_bar, ep6), from a field-major state
    (leaves of weight zero carry no state: zeros)."""
    L = 1 << tree.K
    z = np.zeros((L, 7))
    slot = 0
    for l in range(L):
        if tree.phases[l % 2].kind != 0 and tree.w[l] > 0:
            b = state[6 * slot:6 * slot + 6, i]
            z[l] = [b[0], b[1], b[2], -(b[1] + b[2]), b[3], b[4], b[5]]
            slot += 1
    return z


def jumps(tree, state, i):
    """a of point i (paper ordering) from a field-major state."""
    L = 1 << tree.K
    nz = sum(1 for l in range(L) if tree.phases[l % 2].kind != 0 and tree.w[l] > 0)
    return np.array(state[6 * nz:, i])
