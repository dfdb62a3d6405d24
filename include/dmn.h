/*
 * dmn.h - C ABI of the batched DMN material-point update on GB300 (sm_103a).
 *
 * A direct deep material network (DMN) is a perfect binary tree of depth K of
 * rank-one laminates (Gajek, Schneider, Boehlke, "An FE-DMN method for the
 * multiscale analysis of fiber reinforced plastic components", Sec. 2.1).
 * Leaves alternate between phase 1 (odd leaves, e.g. elastic glass fiber) and
 * phase 2 (even leaves, e.g. a J2-elastoplastic matrix).  Lamination normals
 * are interpolated over the fiber-orientation triangle (Sec. 2.3).  For every
 * Gauss point the update solves the DMN's Euler-Lagrange equation
 * A^T W sigma(E + A a, z^n) = 0 for the displacement jumps a by Newton's
 * method and returns the effective stress, the algorithmic tangent and the
 * new state (Sec. 3.2; criterion and tolerance of Sec. 4.6).
 *
 * Conventions used by every entry point
 *   - Symmetric tensors are 6-vectors ordered (11, 22, 33, 23, 13, 12).
 *     Strains and stresses are Mandel vectors (shear entries times sqrt(2)),
 *     so the Euclidean norm is the Frobenius norm.  The orientation tensor A2
 *     uses plain components.  Tangents are Mandel 6x6, row-major.
 *   - Frames Q are row-major 3x3 with the eigenvectors of A2 as columns
 *     (A2 = Q diag(lam1, lam2, lam3) Q^T, det Q = +1).  Strains are rotated
 *     into that frame before the DMN is evaluated, stress and tangent back.
 *   - Per-point arrays are point-major ([n][6] means element c of point i at
 *     index 6*i + c).  The state is field-major: field f of point i lives at
 *     state[f * n + i].  Per inelastic leaf, in leaf order, six fields
 *     (alpha_bar, ep11, ep22, sqrt2*ep23, sqrt2*ep13, sqrt2*ep12) of the
 *     equivalent plastic strain and the deviatoric plastic strain
 *     (ep33 = -ep11 - ep22); then three jump components per laminate in the
 *     paper's ordering (level K first, root last; Sec. 3.2, Eq. of the normal
 *     ordering).  A compressed tree (leaf weights of zero, Sec. 3.1) keeps
 *     only its remaining inelastic leaves and laminates, in the same orders.  With the extrapolated start (dmn_options.predictor = 1) more
 *     fields follow: the jump change a^{n+1} - a^n of the last update (same
 *     ordering, three per laminate), then that update's strain increment dE
 *     (six, Mandel, global frame).  A zero state is the virgin state.
 *   - Pointers named "dev" are CUDA device pointers; "host" are host
 *     pointers.  The caller owns every array passed in; the handle owns its
 *     parameters and work space.  Device calls are asynchronous on the given
 *     stream (a cudaStream_t passed as void*, NULL = legacy default stream).
 *   - Return codes: 0 = success; DMN_ERR_ARG (-1) invalid argument, nothing
 *     launched; DMN_ERR_CUDA (-2) a CUDA call failed (dmn_last_error has the
 *     message).  Kernels never trap: per-point failures are reported in the
 *     status array.
 *   - One handle may have one call in flight at a time (dmn_update,
 *     dmn_update_host, dmn_grad or dmn_set_params): calls on the same handle
 *     share its work space, and a call that grows a buffer waits only for its
 *     own stream before freeing the old one.  Calls on different streams must
 *     be ordered by the caller (events); different handles are independent.
 *   - A handle belongs to the CUDA device that was current when dmn_create
 *     ran: its parameters and work space live there.  Make that device
 *     current for every later call, and pass arrays in its memory (or, for
 *     dmn_update_host, in host memory).
 */
#ifndef DMN_H
#define DMN_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct dmn_handle dmn_handle;

enum { DMN_OK = 0, DMN_ERR_ARG = -1, DMN_ERR_CUDA = -2 };

/* phase laws: linear elastic (sigma = 3K P1 eps + 2G P2 eps) and J2
 * plasticity with isotropic hardening, integrated by implicit Euler (radial
 * return; Sec. 4.1 takes the J2 law from Simo-Hughes ch. 3):
 *   DMN_PHASE_J2_LINEAR  sigma_Y = sigma0 + H alpha_bar;
 *   DMN_PHASE_J2_EXPLIN  sigma_Y = sigma0 + H alpha_bar
 *                          + (sigma_inf - sigma0) (1 - exp(-(k0 - H) / (sigma_inf - sigma0) alpha_bar)),
 *                        the exponential-linear law of Sec. 4.1 (H = k_inf); the
 *                        plastic multiplier is found by a scalar Newton iteration.
 * alpha_bar is the equivalent plastic strain. */
enum { DMN_PHASE_ELASTIC = 0, DMN_PHASE_J2_LINEAR = 1, DMN_PHASE_J2_EXPLIN = 2 };

/* DMN_PREC_F64: every step in FP64.
 * DMN_PREC_MIXED: leaf tangents, laminate condensation and jump corrections
 * in FP32; leaf stresses, strains, jumps, the Newton residual and the final
 * sweep that yields stress and tangent in FP64.
 * DMN_PREC_MIXED_F32_TANGENT: the Newton iteration of DMN_PREC_MIXED (same
 * jumps, state and FP64 stress), without the FP64 final sweep: the tangent is
 * the FP32 condensation of the last Newton pass, which ran at the converged
 * jumps (relative error a few 1e-7 at depth 8).  For callers whose solver rounds the
 * tangent to FP32 anyway, or that only need a Newton matrix (Sec. 3.2's
 * algorithmic tangent drives the macroscopic Newton method, Sec. 4.6). */
enum { DMN_PREC_F64 = 0, DMN_PREC_MIXED = 1, DMN_PREC_MIXED_F32_TANGENT = 2 };

/* per-point status */
enum {
  DMN_STATUS_OK = 0,
  DMN_STATUS_MAXITER = 1,     /* max_iter corrections without meeting the criterion */
  DMN_STATUS_NONFINITE = 2,   /* NaN or Inf in the inputs or the iterates */
  DMN_STATUS_LINESEARCH = 3,  /* line search: 8 halvings did not lower the residual norm */
  DMN_STATUS_BAD_TREE = 4     /* tree id outside 0 .. n_trees-1 */
};

/* trees per handle */
enum { DMN_MAX_TREES = 8 };

typedef struct {
  int32_t kind;      /* DMN_PHASE_* */
  double E, nu;      /* Young's modulus (MPa), Poisson's ratio */
  double sigma0;     /* J2: initial yield stress (MPa), > 0 */
  double H;          /* J2: linear hardening modulus (MPa), >= 0 (k_inf of the exponential-linear law) */
  double sigma_inf;  /* DMN_PHASE_J2_EXPLIN: saturation stress (MPa), >= sigma0 */
  double k0;         /* DMN_PHASE_J2_EXPLIN: initial hardening modulus (MPa), >= H */
} dmn_phase;

typedef struct {
  int32_t K;         /* depth, 1..8: 2^K - 1 laminates, 2^K leaves (Sec. 2.1) */
  int32_t M;         /* shape functions: 3 linear, 4 tri-linear, 6 quadratic (Tab. of shape functions) */
  const double* p;   /* host [(2^K-1) * M]: alpha_j = p_j . phi(lam1, lam2) (rad), paper ordering (Sec. 3.1) */
  const double* q;   /* host [(2^K-1) * M]: beta_j  = q_j . phi(lam1, lam2) (rad) */
  const double* w;   /* host [2^K]: leaf weights >= 0, not all zero; normalised to sum 1 (Sec. 2.1).
                      * Leaves of weight zero are removed and the tree compressed (Sec. 3.1): a laminate
                      * with one weightless side is replaced by the other side. */
  dmn_phase phase[2];/* phase 1 = odd leaves, phase 2 = even leaves (Sec. 2.1) */
} dmn_tree_desc;

typedef struct {
  double tol;          /* ||A^T W sigma|| / ((2^K - 1) ||sigma_bar||) <= tol (Sec. 4.6); <= 0 selects 1e-12 */
  int32_t max_iter;    /* Newton corrections before status MAXITER; <= 0 selects 50 */
  int32_t precision;   /* DMN_PREC_F64, DMN_PREC_MIXED or DMN_PREC_MIXED_F32_TANGENT */
  int32_t block;       /* threads per CTA of the Newton kernel (multiple of 32); 0 selects 128 */
  int32_t ctas_per_sm; /* resident CTAs per SM of the persistent Newton kernel; 0 selects 384 threads
                        * per SM for DMN_PREC_F64 and 512 for the mixed forms;
                        * block * ctas_per_sm <= 512 (registers are capped to fit) */
  int32_t line_search; /* 0: full Newton steps; 1: backtracking (Sec. 3.2 allows a step in (0, 1]):
                        * a trial step is accepted when it lowers ||A^T W sigma||, else halved, at
                        * most 8 times (then status LINESEARCH and the last accepted iterate).
                        * Needs 2x the per-lane scratch and at most 256 threads per SM. */
  int32_t predictor;   /* 0: each update's Newton iteration starts from the stored jumps a^n, as in
                        * Sec. 4.7.  1: it starts from a^n + rho (a^n - a^{n-1}), with
                        * rho = (dE . dE_prev) / (dE_prev . dE_prev) clamped to [0, 1] (0 when
                        * dE_prev = 0 or the ratio is not finite): the jumps of the last update
                        * extrapolated along the new strain increment while the load keeps its
                        * sense.  A point with rho > 0 that has not met the criterion after 6
                        * corrections (or whose iterates are not finite, or whose line search
                        * fails) restarts from a^n with max_iter corrections; iters counts both
                        * attempts.  The paper has no such start; it reaches the same solution
                        * (up to the stopping criterion) in fewer Newton steps on smooth load
                        * paths.  The state then carries 3 fields per laminate and 6 more (see
                        * the state layout above). */
  int32_t first_stage; /* 1 starts each point's Newton iteration with an all-FP32 stage -- jumps,
                        * strains, the leaf return mapping, the residual and the condensation in FP32 --
                        * until its FP32 residual meets ||A^T W sigma|| <= 1e-8 (2^K - 1) ||sigma_bar||
                        * or min(12, max_iter - 1) corrections; the iteration of the chosen precision
                        * then continues from its jumps to tol, so the results are those of that form
                        * (its residual, criterion, Newton matrix and tangent; the FP64 form takes at
                        * least one FP64 Newton step after the stage).  iters counts the
                        * corrections of both, and both together stay within max_iter.  An FP32 pass
                        * costs about half an FP64-residual pass, and the update needs fewer of the
                        * latter.  0 (default): on in the mixed forms, off in the FP64 form.  -1: off.
                        * Not run with line_search or predictor. */
  int32_t stage_ctas_per_sm; /* resident CTAs of 128 threads per SM of the first stage's persistent kernel:
                              * 2, 3, 4, 6 or 8 (registers capped to fit); 0 selects the default */
  int32_t warp_per_point; /* small batches: 0 (default) updates a call of at most 1024 points per SM
                           * of the device in the FP64 form, 256 in the mixed forms (155648 / 38912 on
                           * 152 SMs) in the warp organisation: a point per group of 32, 16 or 8 lanes
                           * of a warp, the group's lanes sharing each level of the tree (the same
                           * arithmetic per laminate and the same iterates to rounding), where one point
                           * per thread would leave SMs idle; 1 does so for every call; -1 never.  The choice is made per call (for
                           * dmn_update_host on the whole batch, not per chunk); first_stage = 1 turns
                           * the default off.  The extrapolated start always runs one point per thread; the
                           * first stage is not run in this organisation.  Compressed trees (weightless
                           * leaves) run it level by level of the full tree's heap positions. */
  int32_t warp_lanes;     /* lanes per point in that organisation: 32 (one point per warp), 16 or 8 (two
                           * or four points per warp, side by side); 0 (default) chooses by the call's
                           * size: 32 up to 16 points per SM, then 8 in the FP64 form, 16 in the mixed
                           * forms */
} dmn_options;

/* Create a handle for n_trees DMNs (1 <= n_trees <= DMN_MAX_TREES; trees may
 * differ in depth, shape functions, weights and phases, e.g. a batch mixing
 * depths 5 to 8).  Copies the parameters to the device, propagates the leaf
 * weights to the laminate volume fractions (Sec. 2.1) and allocates the work
 * space of the persistent Newton kernel on the current CUDA device.  opt may
 * be NULL (defaults).  Errors: DMN_ERR_ARG for n_trees out of range, K outside
 * 1..8, M not in {3,4,6}, a weight < 0 or non-finite, all weights zero, NULL
 * or non-finite p, q, an unknown phase kind,
 * non-positive moduli or hardening parameters outside the ranges above; DMN_ERR_CUDA if an allocation fails.  On error *out
 * is NULL. */
int dmn_create(const dmn_tree_desc* trees, int32_t n_trees, const dmn_options* opt, dmn_handle** out);

/* Free the handle and its device memory (synchronises the device).  NULL is a no-op. */
void dmn_destroy(dmn_handle* h);

/* Doubles of state per point for tree tree_id: 6 per inelastic leaf plus
 * 3 per laminate (1533 for K = 8 with one inelastic phase; the paper counts
 * the same 128 x (1 + 5) + 255 x 3 scalars, Sec. 4.7), plus 3 per laminate
 * and 6 with the extrapolated start (2304 for K = 8).  tree_id = -1 gives
 * the maximum over the handle's trees: the number of fields S of the state
 * arrays passed to dmn_update (a point of tree t uses the first
 * dmn_state_size(h, t) of them).  -1 on a bad argument. */
int64_t dmn_state_size(const dmn_handle* h, int32_t tree_id);

/* The organisation dmn_update (and dmn_update_host) gives a call of n points on this handle, as
 * lanes per point: 1 one point per thread of the persistent kernel, 32 / 16 / 8 the warp
 * organisation with one / two / four points per warp (dmn_options.warp_per_point, warp_lanes);
 * -1 on a NULL handle or n < 0.  A query only: no device work. */
int dmn_update_lanes_per_point(const dmn_handle* h, int64_t n);

/* Orientation set-up (Sec. 2.2, Eq. of the eigen decomposition of A2):
 * A2 dev [n][6] (plain components, symmetric positive semi-definite, unit
 * trace) -> lam dev [n][2] = (lam1, lam2), the two largest eigenvalues,
 * lam1 >= lam2 >= lam3, and Q dev [n][9], the eigenvectors as columns of a
 * rotation; each of the first two columns is signed so that its entry of
 * largest magnitude is positive, the third is their cross product.
 * n = 0 is a no-op.  Errors: DMN_ERR_ARG for n < 0 or NULL arrays with n > 0. */
int dmn_interp_orientation(dmn_handle* h, int64_t n, const double* A2, double* lam, double* Q, void* stream);

/* One implicit material-point update of n points (Sec. 3.2):
 *   lam      dev [n][2]   orientation eigenvalues (from dmn_interp_orientation)
 *   Q        dev [n][9]   principal frames
 *   E_n, dE  dev [n][6]   macro strain at the start of the increment and its
 *                          increment (Mandel, global frame); E = E_n + dE
 *   state_in dev [S][n]   z^n and the last converged jumps a^n (read only)
 *   state_out dev [S][n]  z^{n+1}, a^{n+1}; must not overlap state_in
 *   stress   dev [n][6]   effective stress sigma_bar = sum_i w_i sigma_i (Mandel, global)
 *   tangent  dev [n][36]  algorithmic tangent d sigma_bar / d E (Eq. lin_system_da_dE)
 *   iters    dev [n]      Newton corrections applied
 *   status   dev [n]      DMN_STATUS_*; NONFINITE writes NaN to stress,
 *                          tangent and the point's state_out
 *   tree_id  dev [n]      tree of each point (0 .. n_trees-1), or NULL for
 *                          tree 0 everywhere; a point with another value gets
 *                          status BAD_TREE, NaN stress and tangent, and its
 *                          state_out is left untouched
 * With several trees the points are first sorted by tree on the device so
 * that the lanes of a warp walk the same tree.  The Newton iteration starts
 * from a^n (Sec. 4.7), or from the extrapolated jumps of dmn_options.predictor,
 * and stops when the criterion of Sec. 4.6 holds.  The
 * first call with a larger n than any earlier call allocates per-point work
 * space (cudaMalloc, synchronous); calls with at most that n allocate nothing
 * and may be captured in a CUDA graph.  Errors: DMN_ERR_ARG for n < 0, NULL
 * arrays with n > 0, state_in == state_out. */
int dmn_update(dmn_handle* h, int64_t n, const int32_t* tree_id, const double* lam, const double* Q,
               const double* E_n, const double* dE, const double* state_in, double* state_out, double* stress,
               double* tangent, int32_t* iters, int32_t* status, void* stream);

/* The update of dmn_update for arrays in HOST memory, the form a finite-element
 * code calls per Gauss-point batch (the UMAT call of Sec. 5).  Same arguments,
 * layouts and results as dmn_update, all arrays host arrays:
 *   tree_id [n] or NULL, lam [n][2], Q [n][9], E_n, dE [n][6] in;
 *   state_in, state_out [S][n] with S = dmn_state_size(h, -1), row pitch n;
 *   stress [n][6], tangent [n][36], iters, status [n] out.
 * Unlike dmn_update, state_out may be state_in itself (each point's state is
 * read before it is written), and a point of an unknown tree (status
 * BAD_TREE) gets its state_in as state_out.  The points are processed in chunks of `chunk`
 * points (<= 0: twice the resident lanes of the Newton kernel) through two
 * stages of device buffers owned by the handle, on streams of the handle: the
 * copy-in of chunk j+1 and the copy-out of chunk j-1 overlap the update of
 * chunk j, and the updates of consecutive chunks may overlap (the two stages
 * use separate work space).  Work queued earlier on `stream` is waited for;
 * the call returns when every copy has ended, so the host arrays may be
 * reused at once.  Pinned host memory (cudaHostAlloc / cudaHostRegister)
 * gives overlapped copies; pageable memory works, slower.  The first call,
 * and a call with a larger chunk than any before, allocate the stage buffers
 * (about 2 x chunk x (2 S + 67) x 8 bytes) and a second Newton work space.
 * Not for stream capture.  Errors: DMN_ERR_ARG for n < 0 or NULL arrays with
 * n > 0; DMN_ERR_CUDA if a CUDA call fails (the call still waits for the
 * copies it queued). */
int dmn_update_host(dmn_handle* h, int64_t n, const int32_t* tree_id, const double* lam, const double* Q,
                    const double* E_n, const double* dE, const double* state_in, double* state_out, double* stress,
                    double* tangent, int32_t* iters, int32_t* status, int64_t chunk, void* stream);

/* Replace the parameters of tree tree_id (host arrays laid out as in
 * dmn_tree_desc: p, q [(2^K-1) * M] in the paper's ordering, w [2^K] >= 0),
 * e.g. after an optimiser step of the offline training (Sec. 3.1).  Depth,
 * shape functions and phases stay, and so does the set of leaves of weight
 * zero: a handle without zero weights takes only positive ones, a handle of
 * compressed trees only weights that are zero exactly where they were (a new
 * compression needs a new handle).  Synchronises the device.  Errors:
 * DMN_ERR_ARG for a bad tree_id, parameters that dmn_create rejects, or a
 * changed set of zero weights. */
int dmn_set_params(dmn_handle* h, int32_t tree_id, const double* p, const double* q, const double* w);

/* Adjoint of the converged update (FP64): for a loss
 * L(sigma_bar, C) with g_stress = dL/d sigma_bar (dev [n][6], global frame)
 * and g_tangent = dL/dC (dev [n][36], row-major, global frame: the
 * derivative with respect to each of the 36 entries of the tangent of
 * dmn_update; only its symmetric part matters), adds to
 *   g_p, g_q  dev [(2^K-1) * M]  dL/dp, dL/dq (paper ordering, Sec. 3.1),
 *   g_w       dev [2^K]          dL/dw for the leaf weights as given to
 *                                dmn_create / dmn_set_params (before their
 *                                normalisation to sum 1),
 * summed over the n points, and writes g_E dev [n][6] = dL/dE = C^T g_stress
 * (may be NULL).  The stress part is the implicit-function derivative of the
 * converged Newton solution of the Euler-Lagrange equation (Sec. 3.2):
 * dL/dtheta = g.d sigma_bar/d theta + mu.dR/d theta with mu = (da/dE) g, the
 * response of the condensed tree to a macro perturbation g (no extra solve);
 * the condensation at the converged jumps is recomputed, nothing from the
 * Newton iterations is stored.  The tangent part is offered for trees whose
 * two phases are elastic, the linear DMN that the offline training of
 * Sec. 3.1 fits to effective stiffnesses: there the tangent is the laminate
 * recursion of the leaf stiffnesses (Eq. of the stiffness propagation),
 * independent of the strain and the jumps, and its adjoint is one reverse
 * pass through that recursion per point (one forward pass recomputes every
 * laminate's stiffness).  For a compressed tree the gradient covers the
 * remaining laminates and leaves; laminates passed through and leaves of
 * weight zero get none (the weights' Macaulay bracket of Sec. 3.1 passes none
 * below zero either).  Inputs are those of the dmn_update call that produced
 * state_out (its output, read only) from state_in; points whose update did not
 * converge should get zero seeds.  Either seed may be NULL, not both; with
 * g_stress NULL, E_n, dE, state_in and state_out may be NULL and g_E (if
 * given) is set to zero.  One tree per handle (tree_id must be NULL).  The
 * first call with a larger n than any earlier call (up to 65536 points per
 * chunk, about 71 KB each at K = 8) allocates work space.  Errors: DMN_ERR_ARG
 * for NULL arrays, both seeds NULL, a tangent seed on a tree with an inelastic
 * phase, n < 0, a non-NULL tree_id or a handle with several trees. */
int dmn_grad(dmn_handle* h, int64_t n, const int32_t* tree_id, const double* lam, const double* Q, const double* E_n,
             const double* dE, const double* state_in, const double* state_out, const double* g_stress,
             const double* g_tangent, double* g_p, double* g_q, double* g_w, double* g_E, void* stream);

/* Per-kernel timing of dmn_update, for measurement: while enabled, CUDA
 * events are recorded on the update's stream before and after each of its
 * kernels.  enable != 0 clears the totals and starts recording; 0 stops.
 * Errors: DMN_ERR_ARG for a NULL handle. */
int dmn_profile_enable(dmn_handle* h, int32_t enable);

/* Totals since dmn_profile_enable(h, 1): ms[0] orientation normals kernel,
 * ms[1] Newton kernel (with the first stage), ms[2] final-sweep kernel (milliseconds, summed over
 * the timed updates), *updates = number of timed updates.  Waits for the
 * recorded events.  Errors: DMN_ERR_ARG for NULL arguments, DMN_ERR_CUDA if
 * an event query fails. */
int dmn_profile_read(dmn_handle* h, double ms[3], int64_t* updates);

/* The same totals with the mixed forms' first stage apart: ms[0] normals, ms[1] first stage (0 when it
 * did not run), ms[2] Newton kernel, ms[3] final sweep; passes (may be NULL): passes[0] tree passes of
 * the first stage, passes[1] of the Newton kernel, summed over points and timed updates (waits for the
 * device).  Errors as dmn_profile_read. */
int dmn_profile_read_stages(dmn_handle* h, double ms[4], int64_t passes[2], int64_t* updates);

/* The same FP64 update as dmn_update, for callers that cannot allocate device
 * memory -- for example code whose device memory is all handed out by an
 * application's own pool or arena, or that runs under a policy forbidding
 * cudaMalloc once it has started.  The paper has no counterpart: this is an
 * interface choice of this library.
 *
 * It needs no handle and allocates nothing (no cudaMalloc, cudaFree or other
 * allocating call).  Its work space -- tree parameters, a work counter and the
 * per-lane scratch of the Newton kernel -- is one static device array of
 * 64 MiB inside this library, which every GPU that loads the library holds
 * until the process exits.  Each call looks up that array's device address on
 * the current device (cudaGetSymbolAddress); the first call on a device also
 * loads the library's device code there, so make that first call before any
 * stream capture.  Every call shares the array: calls that overlap on the GPU
 * (other streams, other host threads) race and must be serialised by the
 * caller.  Each call re-uploads the tree and clears the counter; the tree's
 * parameters travel by value as a kernel argument, so nothing the call queues
 * refers to the caller's host memory after it returns.
 *
 * Arguments are those of dmn_create (tree, opt) and dmn_update (n and the
 * arrays, same layouts and ownership), for one uncompressed tree: all leaf
 * weights must be > 0.  Only the FP64 form with full Newton steps is offered
 * (opt may be NULL; otherwise opt->precision must be DMN_PREC_F64, and
 * opt->predictor and opt->line_search 0); opt->block and opt->ctas_per_sm are
 * ignored.  The static work space limits parallelism: 1152 lanes at K = 8
 * (more for shallower trees), so it is slower than dmn_update.  Errors:
 * DMN_ERR_ARG for the argument errors of dmn_create and dmn_update, for the
 * options above and for a tree whose parameters or one CTA of scratch do not
 * fit the 64 MiB; DMN_ERR_CUDA if a CUDA call fails.  Messages are returned by
 * dmn_last_error(NULL). */
int dmn_update_noalloc(const dmn_tree_desc* tree, const dmn_options* opt, int64_t n, const double* lam,
                       const double* Q, const double* E_n, const double* dE, const double* state_in,
                       double* state_out, double* stress, double* tangent, int32_t* iters, int32_t* status,
                       void* stream);

/* Message of the last failed call on this handle (or of the last failed
 * dmn_create when h is NULL); "" if none.  Valid until the next call. */
const char* dmn_last_error(const dmn_handle* h);

#ifdef __cplusplus
}
#endif

#endif /* DMN_H */
