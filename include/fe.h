/*
 * fe.h - C ABI of the macroscopic finite-element operator that drives the DMN
 * update in an FE-DMN computation (Sec. 5: every Gauss point of the
 * structural model calls the DMN for its stress and algorithmic tangent).
 *
 * The paper couples the DMN to a commercial FE code through its material
 * subroutine interface.  This library supplies the small-strain FE side
 * itself, so that a structural run stays on the GPU: trilinear 8-node
 * hexahedra with 2 x 2 x 2 Gauss points, strains and stresses as Mandel
 * vectors (the conventions of dmn.h), internal forces, the tangent operator
 * applied matrix-free, its diagonal and a Jacobi-preconditioned conjugate
 * gradient solver.  The paper prescribes none of these choices; it names the
 * element types of its own meshes (quadratic tetrahedra) and leaves the
 * solver to the FE code.
 *
 * Conventions
 *   - Nodes [n_nodes][3] coordinates; degrees of freedom [n_nodes][3]
 *     (dof 3*a + i is displacement component i of node a).
 *   - Element e has nodes conn[8*e + 0..7] in the usual hexahedron order:
 *     (-,-,-), (+,-,-), (+,+,-), (-,+,-), then the same at +zeta.
 *   - Gauss point g of element e has index 8*e + g, g = gx + 2 gy + 4 gz over
 *     the points -1/sqrt(3), +1/sqrt(3) in each direction (weight 1).
 *   - Strain at a Gauss point: the Mandel vector of sym(grad u),
 *     (u1,1, u2,2, u3,3, (u2,3 + u3,2)/sqrt2, (u1,3 + u3,1)/sqrt2, (u1,2 + u2,1)/sqrt2).
 *   - Stress [n_gp][6] Mandel, tangent [n_gp][36] row-major Mandel (the
 *     outputs of dmn_update).
 *   - "dev" arrays are device pointers owned by the caller; the mesh handle
 *     owns its geometry and work space.  Calls are asynchronous on the given
 *     stream unless stated otherwise.
 *   - Return codes: 0 success, -1 invalid argument (nothing launched),
 *     -2 a CUDA call failed; fe_last_error gives the message.
 *   - A mesh belongs to the CUDA device that was current when fe_mesh_create
 *     ran; make that device current for every later call on it.  One call
 *     per mesh may be in flight at a time: its element vectors, partial sums
 *     and CG vectors are work space shared by all calls.
 */
#ifndef FE_H
#define FE_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct fe_mesh fe_mesh;

/* Upload a hexahedral mesh (host arrays xyz [n_nodes][3], conn [n_elem][8])
 * and precompute, per Gauss point, the shape-function gradients in physical
 * coordinates and the integration weight det(J).  Synchronous.  Errors: -1 for
 * n_nodes < 8, n_elem < 1, NULL arrays, a node index out of range, or an
 * element with det(J) <= 0 at a Gauss point (inverted or degenerate; the
 * message names the first one); -2 on a CUDA failure.  On error *out is NULL. */
int fe_mesh_create(int64_t n_nodes, int64_t n_elem, const double* xyz, const int32_t* conn, fe_mesh** out);

/* Free the mesh (synchronises the device).  NULL is a no-op. */
void fe_mesh_destroy(fe_mesh* m);

/* Number of Gauss points (8 n_elem) and of degrees of freedom (3 n_nodes). */
int64_t fe_num_gauss_points(const fe_mesh* m);
int64_t fe_num_dofs(const fe_mesh* m);

/* Sum of the integration weights (the mesh volume), computed on the host at
 * creation. */
double fe_volume(const fe_mesh* m);

/* E dev [n_gp][6] = strain of the displacement field u dev [n_dofs]. */
int fe_strain(fe_mesh* m, const double* u, double* E, void* stream);

/* f dev [n_dofs] = sum over Gauss points of B^T sigma det(J): the internal
 * force of the stress field sigma dev [n_gp][6] (overwrites f). */
int fe_internal_force(fe_mesh* m, const double* sigma, double* f, void* stream);

/* Kv dev [n_dofs] = K v with K = sum over Gauss points of B^T C B det(J)
 * (matrix-free; overwrites Kv).  C dev [n_gp][36]. */
int fe_apply_tangent(fe_mesh* m, const double* C, const double* v, double* Kv, void* stream);

/* diag dev [n_dofs] = the diagonal of K (overwrites). */
int fe_tangent_diagonal(fe_mesh* m, const double* C, double* diag, void* stream);

/* Solve K_ff x_f = b_f by conjugate gradients with the Jacobi
 * preconditioner diag_f, where f are the degrees of freedom with
 * free[dof] = 1 (free dev [n_dofs], 1 free, 0 prescribed).  x dev [n_dofs]
 * is overwritten: the solution on the free dofs, 0 on the others.  Stops
 * when ||r_f|| <= rtol ||b_f|| (checked every few iterations) or after
 * max_iter iterations.  Blocks until done and returns the iterations in
 * *iters and ||r_f|| / ||b_f|| in *rel_res (host pointers; either may be
 * NULL).  b_f = 0 gives x = 0 at once.  Errors: -1 for NULL arrays,
 * rtol <= 0 or max_iter < 1; -2 on a CUDA failure. */
int fe_pcg(fe_mesh* m, const double* C, const double* free, const double* diag, const double* b, double* x,
           double rtol, int32_t max_iter, int32_t* iters, double* rel_res, void* stream);

/* fe_pcg with the products K p formed in FP32: C is rounded to FP32 on each
 * call (a field-major copy), the shape-function gradients on the first call;
 * element sums are FP32, node sums and the CG vectors and scalars FP64.  The
 * operator's rounding (about 1e-7 relative) bounds the attainable residual, so
 * rtol should be 1e-6 or larger; an inexact Newton method on the macroscopic
 * equilibrium needs no more.  GB300's FP32 rate is 64 times its FP64 rate, which
 * is why this form exists.  Allocates about n_gp x 244 bytes on first use.
 * Same arguments, results and errors as fe_pcg. */
int fe_pcg_f32(fe_mesh* m, const double* C, const double* free, const double* diag, const double* b, double* x,
               double rtol, int32_t max_iter, int32_t* iters, double* rel_res, void* stream);

/* Blocking reductions for the Newton loop (host results):
 * *out = sum over dofs of free[dof] * a[dof] * b[dof] (free may be NULL: all dofs). */
int fe_dot(fe_mesh* m, const double* a, const double* b, const double* free, double* out, void* stream);

/* y[dof] += alpha * free[dof] * x[dof] (free may be NULL: all dofs). */
int fe_axpy(fe_mesh* m, double alpha, const double* x, const double* free, double* y, void* stream);

/* Message of the last error on m (or of the last failed fe_mesh_create when m is NULL). */
const char* fe_last_error(const fe_mesh* m);

#ifdef __cplusplus
}
#endif

#endif /* FE_H */
