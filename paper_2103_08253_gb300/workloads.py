"""Seeded synthetic inputs for the DMN material-point update.

This module only draws inputs: tree parameters (angle coefficients p, q and leaf
weights w), fiber-orientation fields (A2 with its eigenvalues and frames) and
macro strain paths.  It contains none of the method's arithmetic (no normals,
no laminate algebra, no material law), so both the CUDA path and the CPU oracle
can be fed from it.

Conventions shared by every consumer:

* symmetric 3x3 tensors are 6-vectors ordered (11, 22, 33, 23, 13, 12);
  strains and stresses use the Mandel form (shear entries times sqrt(2)),
  the orientation tensor A2 uses plain components;
* frames Q are row-major 3x3 with the eigenvectors of A2 as columns,
  so that A2 = Q diag(lam1, lam2, lam3) Q^T;
* tree parameters follow the paper's ordering of laminates: the nodes of the
  deepest level K first, then level K-1, ..., the root last (Sec. 3.1);
  leaf weights are listed leaf 1 .. leaf 2^K;
* moduli are in MPa.

The paper's workloads (SAM microstructures, FFT training data, the drone-arm
orientation field) are not available; the generators below stand in for them
with the sizes and value distributions described in the module functions.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

SQRT2 = math.sqrt(2.0)

# Corners of the fiber-orientation triangle in (lam1, lam2): unidirectional,
# isotropic, planar isotropic (Sec. 2.2, Fig. of the orientation triangle).
TRIANGLE_CORNERS = np.array([[1.0, 0.0], [1.0 / 3.0, 1.0 / 3.0], [0.5, 0.5]])


@dataclass
class Phase:
    """One constituent: kind 0 = linear elastic, kind 1 = J2 plasticity with
    linear isotropic hardening sigma_Y = sigma0 + H * alpha_bar, kind 2 = J2
    plasticity with exponential-linear hardening
    sigma_Y = sigma0 + H alpha_bar + (sigma_inf - sigma0)(1 - exp(-(k0 - H)/(sigma_inf - sigma0) alpha_bar))
    (H = k_inf; Sec. 4.1)."""
    kind: int
    E: float
    nu: float
    sigma0: float = 0.0
    H: float = 0.0
    sigma_inf: float = 0.0
    k0: float = 0.0


# Materials of the synthetic workloads: glass fiber and a J2 matrix with linear
# hardening (the fiber data are those of the paper's Tab. of material parameters;
# the matrix law is the linear-hardening stand-in for its exp-linear law).
FIBER = Phase(kind=0, E=72000.0, nu=0.22)
MATRIX = Phase(kind=1, E=3000.0, nu=0.35, sigma0=40.0, H=300.0)
# The paper's polyamide matrix (its table of material parameters): exponential-linear hardening.
MATRIX_EXPLIN = Phase(kind=2, E=2100.0, nu=0.3, sigma0=29.0, H=139.0, sigma_inf=61.7, k0=10600.0)


@dataclass
class TreeParams:
    K: int
    M: int
    p: np.ndarray  # [2^K - 1, M] (rad), paper ordering
    q: np.ndarray  # [2^K - 1, M] (rad), paper ordering
    w: np.ndarray  # [2^K] leaf weights, >= 0
    phases: tuple = field(default_factory=lambda: (FIBER, MATRIX))


def n_nodes(K: int) -> int:
    return (1 << K) - 1


def n_leaves(K: int) -> int:
    return 1 << K


def d10_barycentric() -> np.ndarray:
    """The ten sampling points of the once-split orientation triangle (Sec. 4.3):
    the three corners, the three edge midpoints and the centres of the four
    sub-triangles, as weights on the (UD, ISO, PI) corners."""
    c = [(1, 0, 0), (0, 1, 0), (0, 0, 1),
         (0.5, 0.5, 0), (0.5, 0, 0.5), (0, 0.5, 0.5),
         (2 / 3, 1 / 6, 1 / 6), (1 / 6, 2 / 3, 1 / 6), (1 / 6, 1 / 6, 2 / 3),
         (1 / 3, 1 / 3, 1 / 3)]
    return np.array(c, dtype=np.float64)


def _uniform_sphere_angles(rng, size):
    alpha = np.arccos(rng.uniform(-1.0, 1.0, size=size))
    beta = rng.uniform(0.0, 2.0 * np.pi, size=size)
    return alpha, beta


def tree_constant_normals(K: int, seed: int, M: int = 3, phases=(FIBER, MATRIX)) -> TreeParams:
    """Uniformly random unit normals that do not vary over the orientation
    triangle, and Dirichlet(1, ..., 1) leaf weights.

    The shape functions of every interpolation order sum to one, so constant
    angles are represented by p_j = alpha_j * (1, ..., 1)."""
    rng = np.random.default_rng(seed)
    N = n_nodes(K)
    alpha, beta = _uniform_sphere_angles(rng, N)
    p = np.repeat(alpha[:, None], M, axis=1)
    q = np.repeat(beta[:, None], M, axis=1)
    w = rng.dirichlet(np.ones(n_leaves(K)))
    return TreeParams(K=K, M=M, p=p, q=q, w=w, phases=tuple(phases))


def tree_d10_fit(K: int, seed: int, spread: float = 0.35, phases=(FIBER, MATRIX)) -> TreeParams:
    """Linear (M = 3) angle coefficients fitted to seeded angles at the ten D10
    sampling points.

    Per laminate a base direction is drawn uniformly on the sphere; at each D10
    point its angles are perturbed by N(0, spread^2).  p, q are the least-squares
    coefficients of the linear interpolant through those ten samples: for linear
    interpolation the design matrix is the barycentric coordinates of the D10
    points themselves.  Leaf weights are Dirichlet(1, ..., 1)."""
    rng = np.random.default_rng(seed)
    N = n_nodes(K)
    alpha0, beta0 = _uniform_sphere_angles(rng, N)
    phi = d10_barycentric()                      # [10, 3]
    a_s = alpha0[:, None] + spread * rng.standard_normal((N, 10))
    b_s = beta0[:, None] + spread * rng.standard_normal((N, 10))
    pinv = np.linalg.pinv(phi)                   # [3, 10]
    p = a_s @ pinv.T
    q = b_s @ pinv.T
    w = rng.dirichlet(np.ones(n_leaves(K)))
    return TreeParams(K=K, M=3, p=p, q=q, w=w, phases=tuple(phases))


def tree_nodal_angles(K: int, M: int, seed: int, spread: float = 0.35, phases=(FIBER, MATRIX)) -> TreeParams:
    """Angle coefficients for the tri-linear (M = 4) or quadratic (M = 6) shape
    functions: per laminate a base direction uniform on the sphere, and at each
    of the M interpolation nodes its angles perturbed by N(0, spread^2).  The
    shape functions sum to one, so the coefficients are the nodal angles and the
    normals vary over the triangle about the base direction as in tree_d10_fit.
    Leaf weights are Dirichlet(1, ..., 1)."""
    rng = np.random.default_rng(seed)
    N = n_nodes(K)
    alpha0, beta0 = _uniform_sphere_angles(rng, N)
    p = alpha0[:, None] + spread * rng.standard_normal((N, M))
    q = beta0[:, None] + spread * rng.standard_normal((N, M))
    w = rng.dirichlet(np.ones(n_leaves(K)))
    return TreeParams(K=K, M=M, p=p, q=q, w=w, phases=tuple(phases))


def haar_rotations(rng, n: int) -> np.ndarray:
    """n Haar-distributed rotation matrices [n, 3, 3] (QR of Gaussian matrices
    with the sign of R's diagonal fixed, then det forced to +1)."""
    g = rng.standard_normal((n, 3, 3))
    Qm, R = np.linalg.qr(g)
    d = np.sign(np.diagonal(R, axis1=1, axis2=2))
    d[d == 0] = 1.0
    Qm = Qm * d[:, None, :]
    det = np.linalg.det(Qm)
    Qm[:, :, 2] *= np.sign(det)[:, None]
    return Qm


def orientation_field(n: int, seed: int):
    """Orientation tensors whose eigenvalue pairs are uniform over the fiber
    orientation triangle, with Haar-random principal frames.

    Returns (A2 [n,6] plain components, lam [n,2], Q [n,9] row-major with the
    eigenvectors as columns, sorted lam1 >= lam2 >= lam3)."""
    rng = np.random.default_rng(seed)
    wts = rng.dirichlet(np.ones(3), size=n)      # uniform over the triangle
    lam = wts @ TRIANGLE_CORNERS                 # [n, 2]
    lam3 = 1.0 - lam[:, 0] - lam[:, 1]
    Qm = haar_rotations(rng, n)
    L = np.stack([lam[:, 0], lam[:, 1], lam3], axis=1)
    A = np.einsum("nij,nj,nkj->nik", Qm, L, Qm)
    A2 = np.stack([A[:, 0, 0], A[:, 1, 1], A[:, 2, 2], A[:, 1, 2], A[:, 0, 2], A[:, 0, 1]], axis=1)
    return np.ascontiguousarray(A2), np.ascontiguousarray(lam), np.ascontiguousarray(Qm.reshape(n, 9))


def identity_orientation(n: int):
    """Identity frames and the isotropic corner, for trees whose normals do not
    depend on the orientation."""
    lam = np.tile(np.array([1.0 / 3.0, 1.0 / 3.0]), (n, 1))
    Q = np.tile(np.eye(3).reshape(1, 9), (n, 1))
    return lam, Q


def tensor_to_mandel(T: np.ndarray) -> np.ndarray:
    """[..., 3, 3] symmetric -> [..., 6] Mandel."""
    return np.stack([T[..., 0, 0], T[..., 1, 1], T[..., 2, 2],
                     SQRT2 * T[..., 1, 2], SQRT2 * T[..., 0, 2], SQRT2 * T[..., 0, 1]], axis=-1)


def uniaxial_path_final(n: int, eps_max: float, seed: int) -> np.ndarray:
    """Final macro strain of a uniaxial-strain ramp eps_max * R e1 (x) e1 R^T with
    a Haar-random R per point (Mandel, [n, 6])."""
    rng = np.random.default_rng(seed)
    R = haar_rotations(rng, n)
    d = R[:, :, 0]
    T = eps_max * np.einsum("ni,nj->nij", d, d)
    return tensor_to_mandel(T)


def random6_path_final(n: int, eps_eq_max: float, seed: int, min_dev_fraction: float = 0.5) -> np.ndarray:
    """Final macro strain of a proportional path along a random Gaussian Mandel
    direction, rejected while the deviatoric part carries less than
    `min_dev_fraction` of its norm, scaled so that the equivalent strain
    sqrt(2/3 E':E') reaches eps_eq_max ([n, 6])."""
    rng = np.random.default_rng(seed)
    out = np.empty((n, 6))
    todo = np.arange(n)
    while todo.size:
        d = rng.standard_normal((todo.size, 6))
        tr = d[:, 0] + d[:, 1] + d[:, 2]
        dev = d.copy()
        dev[:, :3] -= tr[:, None] / 3.0
        ndev = np.linalg.norm(dev, axis=1)
        ok = ndev >= min_dev_fraction * np.linalg.norm(d, axis=1)
        eq = np.sqrt(2.0 / 3.0) * ndev[ok]
        out[todo[ok]] = d[ok] * (eps_eq_max / eq)[:, None]
        todo = todo[~ok]
    return out


def proportional_increment(E_final: np.ndarray, step: int, n_steps: int):
    """(E_n, dE) of increment `step` (1-based) of a proportional ramp to E_final."""
    E_n = E_final * ((step - 1) / n_steps)
    dE = E_final * (step / n_steps) - E_n
    return np.ascontiguousarray(E_n), np.ascontiguousarray(dE)


def triangle_wave(step: int, n_steps: int, amp: float, periods: float = 1.0) -> float:
    """Amplitude of a triangle wave 0 -> +amp -> -amp -> 0 ... after `step` of
    `n_steps` increments (periods full cycles)."""
    t = periods * step / n_steps
    f = t - math.floor(t)
    if f < 0.25:
        return amp * 4.0 * f
    if f < 0.75:
        return amp * (2.0 - 4.0 * f)
    return amp * (4.0 * f - 4.0)


def state_size(K: int, phases=(FIBER, MATRIX)) -> int:
    """Doubles of state per point: 6 per inelastic leaf (alpha_bar and the five
    independent components of the deviatoric plastic strain), then 3 jumps per
    laminate."""
    L = n_leaves(K)
    n_inel = sum(1 for i in range(L) if phases[i % 2].kind != 0)
    return 6 * n_inel + 3 * n_nodes(K)


def cyclic_increment(E_amp: np.ndarray, step: int, n_steps: int, periods: float = 1.0):
    """(E_n, dE) of increment `step` (1-based) of a triangle-wave path
    0 -> +E_amp -> -E_amp -> 0 repeated `periods` times over n_steps."""
    a0 = triangle_wave(step - 1, n_steps, 1.0, periods)
    a1 = triangle_wave(step, n_steps, 1.0, periods)
    return np.ascontiguousarray(E_amp * a0), np.ascontiguousarray(E_amp * (a1 - a0))


def mixed_depth_batch(n: int, seed: int, depths=(5, 6, 7, 8)):
    """Tree ids of n points, equal shares of the given depths, shuffled, plus a
    per-point flag selecting the elastic-range half (True) or the cyclic half."""
    rng = np.random.default_rng(seed)
    tid = np.arange(n) % len(depths)
    rng.shuffle(tid)
    elastic = np.zeros(n, dtype=bool)
    elastic[rng.permutation(n)[: n // 2]] = True
    return tid.astype(np.int32), elastic


# ---------------------------------------------------------------------------------------------
# FE-coupled workload: a plate with a central hole in tension (stands in for the structural
# models of Sec. 5, whose geometry and orientation fields are not available).


@dataclass
class PlateMesh:
    xyz: np.ndarray        # [n_nodes, 3]
    conn: np.ndarray       # [n_elem, 8] int32, hexahedron node order (-,-,-), (+,-,-), (+,+,-), (-,+,-), top
    fixed: np.ndarray      # [3 n_nodes] bool: prescribed degrees of freedom
    pull: np.ndarray       # [3 n_nodes] float: 1 on the x dofs of the loaded face (u = delta * pull there)
    affine: np.ndarray     # [3 n_nodes] float: u_x = (x + H) / (2H), the uniform-strain field of unit delta
    centroid: np.ndarray   # [n_elem, 3] mean of each element's nodes
    H: float
    R: float
    T: float


def plate_with_hole_mesh(n_t: int, n_r: int, n_z: int, R: float = 5.0, H: float = 25.0, T: float = 4.0,
                         grade: float = 1.5) -> PlateMesh:
    """O-grid hexahedral mesh of the square plate [-H, H]^2 with a central hole of radius R,
    upper half of the thickness T (z in [0, T/2], the mid-plane z = 0 a symmetry plane).

    4 n_t node columns around the hole (n_t even), n_r elements from the hole to the outer
    square (spacing graded towards the hole by the exponent `grade`), n_z through the half
    thickness: 4 n_t n_r n_z elements.  A node at angle theta sits between the hole point
    R (cos, sin) and the square point H (cos, sin) / max(|cos|, |sin|).

    Boundary conditions (tension along x): u_z = 0 on z = 0; u_x = 0 on the face x = -H;
    u_x = delta on x = +H; u_y = 0 on the lines y = 0 of both loaded faces."""
    if n_t % 2:
        raise ValueError("n_t must be even")
    nk = 4 * n_t
    k = np.arange(nk)
    theta = 2.0 * np.pi * k / nk - np.pi / 4.0
    c, s = np.cos(theta), np.sin(theta)
    sq = np.maximum(np.abs(c), np.abs(s))
    inner = np.stack([R * c, R * s], axis=1)
    outer = np.stack([H * c / sq, H * s / sq], axis=1)
    rho = (np.arange(n_r + 1) / n_r) ** grade
    z = 0.5 * T * np.arange(n_z + 1) / n_z
    # node id = (j * (n_r + 1) + i) * nk + k
    xy = inner[None, :, :] + rho[:, None, None] * (outer - inner)[None, :, :]      # [n_r+1, nk, 2]
    xyz = np.zeros((n_z + 1, n_r + 1, nk, 3))
    xyz[..., :2] = xy[None]
    xyz[..., 2] = z[:, None, None]
    xyz = xyz.reshape(-1, 3)

    def nid(j, i, kk):
        return (j * (n_r + 1) + i) * nk + kk % nk

    J, I, Kk = np.meshgrid(np.arange(n_z), np.arange(n_r), np.arange(nk), indexing="ij")
    J, I, Kk = J.ravel(), I.ravel(), Kk.ravel()
    # local xi = radial (i), eta = angular (k), zeta = z: right-handed
    conn = np.stack([nid(J, I, Kk), nid(J, I + 1, Kk), nid(J, I + 1, Kk + 1), nid(J, I, Kk + 1),
                     nid(J + 1, I, Kk), nid(J + 1, I + 1, Kk), nid(J + 1, I + 1, Kk + 1), nid(J + 1, I, Kk + 1)],
                    axis=1).astype(np.int32)
    n_nodes = xyz.shape[0]
    fixed = np.zeros((n_nodes, 3), dtype=bool)
    pull = np.zeros((n_nodes, 3))
    eps = 1e-9 * H
    x, y = xyz[:, 0], xyz[:, 1]
    fixed[np.abs(xyz[:, 2]) < eps, 2] = True
    left = np.abs(x + H) < eps
    right = np.abs(x - H) < eps
    fixed[left, 0] = True
    fixed[right, 0] = True
    pull[right, 0] = 1.0
    fixed[(left | right) & (np.abs(y) < eps), 1] = True
    centroid = xyz[conn].mean(axis=1)
    affine = np.zeros((n_nodes, 3))
    affine[:, 0] = (x + H) / (2.0 * H)
    return PlateMesh(xyz=xyz, conn=conn, fixed=fixed.reshape(-1), pull=pull.reshape(-1), affine=affine.reshape(-1),
                     centroid=centroid, H=H, R=R, T=T)


def plate_orientation_field(centroid: np.ndarray, R: float, H: float, T: float, seed: int) -> np.ndarray:
    """Smooth fiber-orientation field A2 [n, 6] (plain components) at the given points.

    Flow direction d: the potential flow of a uniform stream along x past the hole, its angle
    perturbed by three seeded smooth modes (amplitude ~0.1 rad).  Through the thickness the
    field goes from a nearly planar-isotropic core (mid-plane) to a flow-aligned skin (faces):
    A2 = s A_flow + (1 - s) A_plane with s = 0.1 + 0.8 (2 z / T)^2,
    A_flow = 0.92 d(x)d + 0.05 t(x)t + 0.03 e3(x)e3, A_plane = 0.485 (d(x)d + t(x)t) + 0.03 e3(x)e3,
    t the in-plane normal of d (so lam3 = 0.03 >= 0.01 everywhere and lam1 > lam2)."""
    rng = np.random.default_rng(seed)
    x, y, z = centroid[:, 0], centroid[:, 1], centroid[:, 2]
    r2 = np.maximum(x * x + y * y, (1e-6 * R) ** 2)
    ux = 1.0 - R * R * (x * x - y * y) / (r2 * r2)
    uy = -2.0 * R * R * x * y / (r2 * r2)
    phi = np.arctan2(uy, ux)
    for _ in range(3):
        kx, ky = rng.uniform(0.5, 2.0, size=2) * np.pi / H
        phi = phi + 0.1 * rng.standard_normal() * np.sin(kx * x + ky * y + rng.uniform(0, 2 * np.pi))
    d = np.stack([np.cos(phi), np.sin(phi), np.zeros_like(phi)], axis=1)
    t = np.stack([-np.sin(phi), np.cos(phi), np.zeros_like(phi)], axis=1)
    e3 = np.array([0.0, 0.0, 1.0])
    s = 0.1 + 0.8 * (2.0 * z / T) ** 2
    l1 = s * 0.92 + (1 - s) * 0.485
    l2 = s * 0.05 + (1 - s) * 0.485
    A = (l1[:, None, None] * np.einsum("ni,nj->nij", d, d) + l2[:, None, None] * np.einsum("ni,nj->nij", t, t)
         + 0.03 * np.outer(e3, e3)[None])
    return np.ascontiguousarray(np.stack([A[:, 0, 0], A[:, 1, 1], A[:, 2, 2], A[:, 1, 2], A[:, 0, 2], A[:, 0, 1]],
                                         axis=1))


def tree_with_zero_weights(K: int, seed: int, zero_fraction: float = 0.3, phases=(FIBER, MATRIX)) -> TreeParams:
    """A D10-fitted tree whose leaf weights are partly zero, as after the offline training
    (Sec. 3.1: weights that reach zero stay there and the tree is compressed).  One whole
    subtree of the root's right child at depth 2 (a quarter of the leaves, when K >= 3) and a
    random further share of single leaves get weight zero, so the compressed tree has
    pass-through laminates, removed subtrees and leaves whose sibling is a laminate."""
    t = tree_d10_fit(K, seed=seed, phases=phases)
    rng = np.random.default_rng(seed + 7919)
    L = 1 << K
    w = t.w.copy()
    if K >= 3:
        w[L // 2: L // 2 + L // 4] = 0.0
    alive = np.nonzero(w > 0)[0]
    k = int(round(zero_fraction * L)) - (L - alive.size)
    if k > 0:
        w[rng.choice(alive, size=min(k, alive.size - 1), replace=False)] = 0.0
    return TreeParams(K=K, M=t.M, p=t.p, q=t.q, w=w, phases=t.phases)
