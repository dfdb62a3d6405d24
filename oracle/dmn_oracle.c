/*
 * Plain FP64 CPU oracle of the DMN material-point update.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the bench's
 * CPU-baseline leg may load this code.  It shares nothing with the CUDA path:
 * its own tree indexing, its own Mandel helpers, its own material law and a
 * different linear solver (the paper's assembled system with a Cholesky
 * factorisation instead of the GPU's tree condensation).
 *
 * What it follows (Gajek, Schneider, Boehlke, "An FE-DMN method for the
 * multiscale analysis of fiber reinforced plastic components"):
 *   - tree, alternating phases, weight propagation, volume fractions: Sec. 2.1;
 *   - orientation triangle and eigen-decomposition of A2: Sec. 2.2, Eq. (eigen
 *     decomposition of A);
 *   - barycentric coordinates (3x3 linear system), shape functions (Tab. of
 *     shape functions), interpolated angles, spherical normals: Sec. 2.3;
 *   - ordering of laminates (level K first, root last): Sec. 3.1, Eq. (normal
 *     ordering);
 *   - gradient operator A with blocks -c2 N / +c1 N (Eq. of the gradient
 *     operator, depth-3 example), symmetrisation N a = sym(a (x) n), mass
 *     matrix W, Euler-Lagrange residual A^T W sigma, Newton system
 *     A^T W D A (Eq. newton_complex), effective stress, algorithmic tangent via
 *     the six-right-hand-side system (Eq. lin_system_da_dE): Sec. 3.2;
 *   - convergence criterion ||A^T W sigma|| / ((2^K - 1) ||sigma_bar||) <= tol
 *     and a Cholesky solve: Sec. 4.6;
 *   - matrix law: J2 plasticity with isotropic hardening (Sec. 4.1, radial
 *     return of Simo-Hughes ch. 3), with linear or exponential-linear
 *     hardening.
 *
 * Conventions: Mandel 6-vectors (11, 22, 33, sqrt2*23, sqrt2*13, sqrt2*12);
 * the state of a point is stored field-major ("SoA"): field f of point i is
 * state[f * n + i].  Per inelastic leaf (leaf order) the fields are
 * (alpha_bar, ep11, ep22, sqrt2*ep23, sqrt2*ep13, sqrt2*ep12) with
 * ep33 = -ep11 - ep22; then 3 jump components per laminate in the paper's
 * ordering.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define OR_KMAX 8
#define OR_NMAX ((1 << OR_KMAX) - 1)
#define OR_LMAX (1 << OR_KMAX)

static const double R2 = 1.41421356237309504880;

/* ------------------------------------------------------------------ */
/* Tree indexing in the paper's notation: laminate (k, i), k = 1..K is the
 * level (root k = 1), i = 1..2^(k-1); its children are (k+1, 2i-1) and
 * (k+1, 2i); level K+1 holds the leaves 1..2^K.  The flat index of a laminate
 * follows the paper's ordering: level K first, then K-1, ..., root last.    */
static int node_index(int K, int k, int i) { return (1 << K) - (1 << k) + (i - 1); }
static void node_level_pos(int K, int j, int* k, int* i) {
  int kk = K, off = 0;
  while (j >= off + (1 << (kk - 1))) { off += 1 << (kk - 1); kk--; }
  *k = kk; *i = j - off + 1;
}
/* is leaf l (1..2^K) below laminate (k, i)?  side: -1 left subtree, +1 right */
static int leaf_side(int K, int k, int i, int l) {
  int span = 1 << (K - k + 1);              /* leaves below (k, i) */
  if ((l - 1) / span + 1 != i) return 0;
  int child = (l - 1) / (span / 2) + 1;     /* child index at level k+1 */
  return (child == 2 * i - 1) ? -1 : +1;
}

/* ------------------------------------------------------------------ */
typedef struct { int kind; double E, nu, s0, H, sinf, k0; } or_phase;
#define OR_MAT 7   /* doubles per phase: kind, E, nu, sigma0, H (k_inf), sigma_inf, k0 */

typedef struct {
  int K, M, N, L;
  const double *p, *q;
  double w[OR_LMAX];          /* normalised leaf weights */
  double c1[OR_NMAX], c2[OR_NMAX];
  or_phase ph[2];
  double tol; int max_iter; int line_search;
  /* Tree compression (Sec. 3.1, removing laminates with a weightless
   * subtree): a laminate is active when both of its subtrees carry weight;
   * a laminate with one weightless subtree passes the other through (its
   * jump does not reach a weighted leaf), one with two is dead.  Only the
   * active laminates carry unknown jumps; they are numbered in the paper's
   * order (cidx), and a leaf of zero weight has no strain, no state.  With
   * all weights positive every laminate is active. */
  int nact;
  int act[OR_NMAX];           /* paper index of the c-th active laminate */
  int cidx[OR_NMAX];          /* compressed index of laminate j, or -1 */
  /* active ancestors of every leaf (0-based; none for a weightless leaf): the
   * laminate's paper index and the coefficient (-c2 or +c1) of its A block */
  int nanc[OR_LMAX];
  int anc_node[OR_LMAX][OR_KMAX];
  double anc_coef[OR_LMAX][OR_KMAX];
  /* active descendants / ancestors of every active laminate, as compressed
   * indices (the Cholesky pattern) */
  int n_desc[OR_NMAX]; int* desc[OR_NMAX];
  int n_anc[OR_NMAX]; int anc[OR_NMAX][OR_KMAX];
  int nz;  /* number of inelastic leaves */
  int z_slot[OR_LMAX];  /* inelastic slot of each leaf or -1 */
} or_tree;

static void tree_free(or_tree* t) {
  for (int c = 0; c < t->nact; ++c) free(t->desc[c]);
}

/* weights: Sec. 2.1, w^i_k = w^{2i-1}_{k+1} + w^{2i}_{k+1}; c1 = w_left / (w_left + w_right). */
static int tree_init(or_tree* t, int K, int M, const double* p, const double* q, const double* w,
                     const double* mat, double tol, int max_iter, int line_search) {
  if (K < 1 || K > OR_KMAX || (M != 3 && M != 4 && M != 6)) return -1;
  memset(t, 0, sizeof(*t));
  t->K = K; t->M = M; t->N = (1 << K) - 1; t->L = 1 << K; t->p = p; t->q = q;
  t->tol = tol; t->max_iter = max_iter; t->line_search = line_search;
  for (int f = 0; f < 2; ++f) {
    const double* m = mat + OR_MAT * f;
    t->ph[f].kind = (int)m[0]; t->ph[f].E = m[1]; t->ph[f].nu = m[2];
    t->ph[f].s0 = m[3]; t->ph[f].H = m[4]; t->ph[f].sinf = m[5]; t->ph[f].k0 = m[6];
    if (t->ph[f].kind < 0 || t->ph[f].kind > 2) return -1;
  }
  double sw = 0.0;
  for (int l = 0; l < t->L; ++l) { if (!(w[l] >= 0.0) || !isfinite(w[l])) return -2; sw += w[l]; }
  if (!(sw > 0.0)) return -2;
  for (int l = 0; l < t->L; ++l) t->w[l] = w[l] / sw;
  /* subtree weights level by level, leaves -> root */
  double Wlev[OR_KMAX + 2][OR_LMAX];
  for (int l = 0; l < t->L; ++l) Wlev[K + 1][l] = t->w[l];
  for (int k = K; k >= 1; --k)
    for (int i = 1; i <= (1 << (k - 1)); ++i) {
      double wl = Wlev[k + 1][2 * i - 2], wr = Wlev[k + 1][2 * i - 1];
      Wlev[k][i - 1] = wl + wr;
      int j = node_index(K, k, i);
      t->c1[j] = (wl + wr > 0.0) ? wl / (wl + wr) : 0.5;   /* dead laminate: any split, never used */
      t->c2[j] = 1.0 - t->c1[j];
      t->cidx[j] = (wl > 0.0 && wr > 0.0) ? 0 : -1;
    }
  t->nact = 0;
  for (int j = 0; j < t->N; ++j)
    if (t->cidx[j] >= 0) { t->cidx[j] = t->nact; t->act[t->nact++] = j; }
  for (int l = 1; l <= t->L; ++l) {
    t->nanc[l - 1] = 0;
    if (!(t->w[l - 1] > 0.0)) continue;
    for (int k = 1; k <= K; ++k) {
      int i = (l - 1) / (1 << (K - k + 1)) + 1;
      int j = node_index(K, k, i);
      if (t->cidx[j] < 0) continue;
      int s = leaf_side(K, k, i, l);
      t->anc_node[l - 1][t->nanc[l - 1]] = j;
      t->anc_coef[l - 1][t->nanc[l - 1]++] = (s < 0) ? -t->c2[j] : t->c1[j];
    }
  }
  for (int c = 0; c < t->nact; ++c) {
    int j = t->act[c], k, i;
    node_level_pos(K, j, &k, &i);
    t->n_anc[c] = 0;
    for (int kk = k - 1; kk >= 1; --kk) {
      int ii = (i - 1) / (1 << (k - kk)) + 1;
      int a = t->cidx[node_index(K, kk, ii)];
      if (a >= 0) t->anc[c][t->n_anc[c]++] = a;
    }
    int cnt = 0;
    for (int kk = k + 1; kk <= K; ++kk) cnt += 1 << (kk - k);
    t->desc[c] = (int*)malloc(sizeof(int) * (cnt > 0 ? cnt : 1));
    int d = 0;
    for (int kk = K; kk > k; --kk) {                /* in index order (deepest first) */
      int span = 1 << (kk - k);
      for (int ii = (i - 1) * span + 1; ii <= i * span; ++ii) {
        int a = t->cidx[node_index(K, kk, ii)];
        if (a >= 0) t->desc[c][d++] = a;
      }
    }
    t->n_desc[c] = d;
  }
  t->nz = 0;
  for (int l = 0; l < t->L; ++l) {
    int f = l % 2;   /* leaf l+1 odd -> phase 1, even -> phase 2 */
    t->z_slot[l] = (t->ph[f].kind != 0 && t->w[l] > 0.0) ? t->nz++ : -1;
  }
  return 0;
}

/* ------------------------------------------------------------------ */
/* Sec. 2.3: barycentric coordinates from the 3x3 system, solved by Gaussian
 * elimination with partial pivoting exactly as printed:
 *   [1 1/3 1/2; 0 1/3 1/2; 1 1 1] [phi1 phi2 phi3]^T = [lam1 lam2 1]^T      */
static void barycentric(double lam1, double lam2, double phi[3]) {
  double A[3][4] = {{1.0, 1.0 / 3.0, 0.5, lam1}, {0.0, 1.0 / 3.0, 0.5, lam2}, {1.0, 1.0, 1.0, 1.0}};
  for (int c = 0; c < 3; ++c) {
    int piv = c;
    for (int r = c + 1; r < 3; ++r) if (fabs(A[r][c]) > fabs(A[piv][c])) piv = r;
    if (piv != c) for (int k = 0; k < 4; ++k) { double tmp = A[c][k]; A[c][k] = A[piv][k]; A[piv][k] = tmp; }
    for (int r = c + 1; r < 3; ++r) {
      double f = A[r][c] / A[c][c];
      for (int k = c; k < 4; ++k) A[r][k] -= f * A[c][k];
    }
  }
  for (int r = 2; r >= 0; --r) {
    double s = A[r][3];
    for (int k = r + 1; k < 3; ++k) s -= A[r][k] * phi[k];
    phi[r] = s / A[r][r];
  }
}

/* Tab. of shape functions: linear (M=3), tri-linear (M=4), quadratic (M=6). */
static void shape_functions(int M, const double v[3], double* ph) {
  if (M == 3) { ph[0] = v[0]; ph[1] = v[1]; ph[2] = v[2]; }
  else if (M == 4) {
    double b = v[0] * v[1] * v[2];
    ph[0] = v[0] - 9.0 * b; ph[1] = v[1] - 9.0 * b; ph[2] = v[2] - 9.0 * b; ph[3] = 27.0 * b;
  } else {
    ph[0] = v[0] * (2.0 * v[0] - 1.0); ph[1] = v[1] * (2.0 * v[1] - 1.0); ph[2] = v[2] * (2.0 * v[2] - 1.0);
    ph[3] = 4.0 * v[0] * v[1]; ph[4] = 4.0 * v[0] * v[2]; ph[5] = 4.0 * v[1] * v[2];
  }
}

/* Eq. (interpolating the angles) and the spherical normal of Sec. 2.3. */
static void normals(const or_tree* t, double lam1, double lam2, double nrm[][3]) {
  double v[3], ph[6];
  barycentric(lam1, lam2, v);
  shape_functions(t->M, v, ph);
  for (int j = 0; j < t->N; ++j) {
    double al = 0.0, be = 0.0;
    for (int m = 0; m < t->M; ++m) { al += t->p[j * t->M + m] * ph[m]; be += t->q[j * t->M + m] * ph[m]; }
    nrm[j][0] = sin(al) * cos(be);
    nrm[j][1] = sin(al) * sin(be);
    nrm[j][2] = cos(al);
  }
}

/* ------------------------------------------------------------------ */
/* Mandel helpers written on plain 3x3 tensors. */
static void mandel_to_tensor(const double v[6], double T[3][3]) {
  T[0][0] = v[0]; T[1][1] = v[1]; T[2][2] = v[2];
  T[1][2] = T[2][1] = v[3] / R2; T[0][2] = T[2][0] = v[4] / R2; T[0][1] = T[1][0] = v[5] / R2;
}
static void tensor_to_mandel(double T[3][3], double v[6]) {
  v[0] = T[0][0]; v[1] = T[1][1]; v[2] = T[2][2];
  v[3] = R2 * 0.5 * (T[1][2] + T[2][1]); v[4] = R2 * 0.5 * (T[0][2] + T[2][0]); v[5] = R2 * 0.5 * (T[0][1] + T[1][0]);
}
/* index pair of Mandel component I and its weight (1 or sqrt2) */
static const int MI[6][2] = {{0, 0}, {1, 1}, {2, 2}, {1, 2}, {0, 2}, {0, 1}};
static double mweight(int I) { return I < 3 ? 1.0 : R2; }

/* N(n) as a 6x3 matrix: column m is the Mandel vector of sym(e_m (x) n). */
static void sym_operator(const double n[3], double Nm[6][3]) {
  for (int m = 0; m < 3; ++m) {
    double T[3][3];
    for (int r = 0; r < 3; ++r)
      for (int c = 0; c < 3; ++c)
        T[r][c] = 0.5 * (((r == m) ? n[c] : 0.0) + ((c == m) ? n[r] : 0.0));
    double v[6]; tensor_to_mandel(T, v);
    for (int I = 0; I < 6; ++I) Nm[I][m] = v[I];
  }
}

/* ------------------------------------------------------------------ */
/* Phase laws.  Elastic: sigma = 3K P1 eps + 2G P2 eps.  J2 plasticity with
 * isotropic hardening sigma_Y(ab), ab the equivalent plastic strain,
 * integrated by implicit Euler = radial return (Simo-Hughes ch. 3):
 *   s_tr = 2G (dev eps - ep_n), f = |s_tr| - sqrt(2/3) sigma_Y(ab_n);
 *   f > 0: dg solves |s_tr| - 2G dg - sqrt(2/3) sigma_Y(ab_n + sqrt(2/3) dg) = 0,
 *          nhat = s_tr/|s_tr|, s = s_tr - 2G dg nhat,
 *          ep = ep_n + dg nhat, ab = ab_n + sqrt(2/3) dg,
 *          D = K 1(x)1 + 2G th Idev - 2G thb nhat(x)nhat,
 *          th = 1 - 2G dg/|s_tr|, thb = 1/(1 + H'/(3G)) - (1 - th),
 *          H' = d sigma_Y / d ab at the new ab.
 * kind 1, linear hardening: sigma_Y = s0 + H ab, so dg = f / (2G + 2H/3).
 * kind 2, exponential-linear hardening (Sec. 4.1, the matrix law of the
 *   paper's material table): sigma_Y = s0 + H ab + (sinf - s0)(1 - exp(-(k0 - H)/(sinf - s0) ab))
 *   with H = k_inf; dg by Newton's method on the scalar equation above,
 *   started at 0 (the equation is convex and decreasing in dg, so the
 *   iterates increase monotonically to the root).
 * z = (ab, ep in Mandel, 6 comps with ep33 = -ep11-ep22).  gap = |f| / sigma_Y. */
static double yield_stress(const or_phase* ph, double ab, double* slope) {
  if (ph->kind == 2 && ph->sinf > ph->s0) {
    double ds = ph->sinf - ph->s0, r = (ph->k0 - ph->H) / ds;
    double e = exp(-r * ab);
    if (slope) *slope = ph->H + (ph->k0 - ph->H) * e;
    return ph->s0 + ph->H * ab + ds * (1.0 - e);
  }
  if (slope) *slope = ph->H;
  return ph->s0 + ph->H * ab;
}

static void phase_law(const or_phase* ph, const double eps[6], const double z_n[7],
                      double sig[6], double D[6][6], double z_new[7], double* gap) {
  double K = ph->E / (3.0 * (1.0 - 2.0 * ph->nu));
  double G = ph->E / (2.0 * (1.0 + ph->nu));
  double tr = eps[0] + eps[1] + eps[2];
  double dev[6];
  for (int I = 0; I < 6; ++I) dev[I] = eps[I] - (I < 3 ? tr / 3.0 : 0.0);
  double Idev[6][6];
  for (int I = 0; I < 6; ++I)
    for (int J = 0; J < 6; ++J) Idev[I][J] = (I == J ? 1.0 : 0.0) - ((I < 3 && J < 3) ? 1.0 / 3.0 : 0.0);
  if (ph->kind == 0) {
    for (int I = 0; I < 6; ++I) sig[I] = (I < 3 ? K * tr : 0.0) + 2.0 * G * dev[I];
    for (int I = 0; I < 6; ++I)
      for (int J = 0; J < 6; ++J) D[I][J] = ((I < 3 && J < 3) ? K : 0.0) + 2.0 * G * Idev[I][J];
    if (gap) *gap = INFINITY;
    return;
  }
  double ab_n = z_n[0];
  const double* ep_n = z_n + 1;
  double str[6], nrm2 = 0.0;
  for (int I = 0; I < 6; ++I) { str[I] = 2.0 * G * (dev[I] - ep_n[I]); nrm2 += str[I] * str[I]; }
  double ns = sqrt(nrm2);
  double sy = yield_stress(ph, ab_n, NULL);
  double f = ns - sqrt(2.0 / 3.0) * sy;
  if (gap) *gap = fabs(f) / sy;
  if (f <= 0.0) {
    for (int I = 0; I < 6; ++I) sig[I] = (I < 3 ? K * tr : 0.0) + str[I];
    for (int I = 0; I < 6; ++I)
      for (int J = 0; J < 6; ++J) D[I][J] = ((I < 3 && J < 3) ? K : 0.0) + 2.0 * G * Idev[I][J];
    if (z_new) for (int c = 0; c < 7; ++c) z_new[c] = z_n[c];
    return;
  }
  double dg, Hp;
  if (ph->kind == 1) {
    dg = f / (2.0 * G + 2.0 * ph->H / 3.0);
    Hp = ph->H;
  } else {
    dg = 0.0;
    for (int it = 0; it < 100; ++it) {
      double slope, r = ns - 2.0 * G * dg - sqrt(2.0 / 3.0) * yield_stress(ph, ab_n + sqrt(2.0 / 3.0) * dg, &slope);
      double step = r / (2.0 * G + (2.0 / 3.0) * slope);
      dg += step;
      if (fabs(step) <= 1e-15 * dg) break;
    }
    yield_stress(ph, ab_n + sqrt(2.0 / 3.0) * dg, &Hp);
  }
  double nh[6];
  for (int I = 0; I < 6; ++I) nh[I] = str[I] / ns;
  double th = 1.0 - 2.0 * G * dg / ns;
  double thb = 1.0 / (1.0 + Hp / (3.0 * G)) - (1.0 - th);
  for (int I = 0; I < 6; ++I) sig[I] = (I < 3 ? K * tr : 0.0) + str[I] - 2.0 * G * dg * nh[I];
  for (int I = 0; I < 6; ++I)
    for (int J = 0; J < 6; ++J)
      D[I][J] = ((I < 3 && J < 3) ? K : 0.0) + 2.0 * G * th * Idev[I][J] - 2.0 * G * thb * nh[I] * nh[J];
  if (z_new) {
    z_new[0] = ab_n + sqrt(2.0 / 3.0) * dg;
    for (int I = 0; I < 6; ++I) z_new[1 + I] = ep_n[I] + dg * nh[I];
  }
}

/* ------------------------------------------------------------------ */
/* Per-point work space. */
typedef struct {
  double nrm[OR_NMAX][3];
  double Nm[OR_NMAX][6][3];
  double eps[OR_LMAX][6], sig[OR_LMAX][6], D[OR_LMAX][6][6];
  double z_n[OR_LMAX][7], z_new[OR_LMAX][7];
  double gap;
  double* J;   /* dense [3N][3N], lower triangle overwritten by the Cholesky factor */
  double R[3 * OR_NMAX], da[3 * OR_NMAX], a[3 * OR_NMAX], a_try[3 * OR_NMAX];
  double sbar[6];
} or_work;

/* eps_l = E + sum over the laminates above leaf l of coef * N_j a_j  (eps = E + A a) */
static void leaf_strains(const or_tree* t, or_work* ws, const double E[6], const double* a) {
  for (int l = 0; l < t->L; ++l) {
    for (int I = 0; I < 6; ++I) ws->eps[l][I] = E[I];
    for (int k = 0; k < t->nanc[l]; ++k) {
      int j = t->anc_node[l][k], cj = t->cidx[j];
      double c = t->anc_coef[l][k];
      for (int I = 0; I < 6; ++I)
        for (int m = 0; m < 3; ++m) ws->eps[l][I] += c * ws->Nm[j][I][m] * a[3 * cj + m];
    }
  }
}

/* phase stresses/tangents, R = A^T W sigma, sigma_bar = sum w sigma; returns ||R||. */
static double evaluate(const or_tree* t, or_work* ws, const double E[6], const double* a) {
  leaf_strains(t, ws, E, a);
  ws->gap = INFINITY;
  for (int l = 0; l < t->L; ++l) {
    double g;
    phase_law(&t->ph[l % 2], ws->eps[l], ws->z_n[l], ws->sig[l], ws->D[l], ws->z_new[l], &g);
    if (g < ws->gap && t->w[l] > 0.0) ws->gap = g;
  }
  for (int I = 0; I < 6; ++I) ws->sbar[I] = 0.0;
  for (int l = 0; l < t->L; ++l)
    for (int I = 0; I < 6; ++I) ws->sbar[I] += t->w[l] * ws->sig[l][I];
  for (int r = 0; r < 3 * t->nact; ++r) ws->R[r] = 0.0;
  for (int l = 0; l < t->L; ++l)
    for (int k = 0; k < t->nanc[l]; ++k) {
      int j = t->anc_node[l][k], cj = t->cidx[j];
      double c = t->anc_coef[l][k] * t->w[l];
      for (int m = 0; m < 3; ++m)
        for (int I = 0; I < 6; ++I) ws->R[3 * cj + m] += c * ws->Nm[j][I][m] * ws->sig[l][I];
    }
  double s = 0.0;
  for (int r = 0; r < 3 * t->nact; ++r) s += ws->R[r] * ws->R[r];
  return sqrt(s);
}

/* J = A^T W D A, assembled leaf by leaf over pairs of the leaf's ancestors. */
static void assemble_J(const or_tree* t, or_work* ws) {
  int n = 3 * t->nact;
  memset(ws->J, 0, sizeof(double) * (size_t)n * n);
  for (int l = 0; l < t->L; ++l) {
    double DN[OR_KMAX][6][3];
    for (int k = 0; k < t->nanc[l]; ++k) {
      int j = t->anc_node[l][k];
      for (int I = 0; I < 6; ++I)
        for (int m = 0; m < 3; ++m) {
          double s = 0.0;
          for (int J2 = 0; J2 < 6; ++J2) s += ws->D[l][I][J2] * ws->Nm[j][J2][m];
          DN[k][I][m] = s;
        }
    }
    for (int k1 = 0; k1 < t->nanc[l]; ++k1)
      for (int k2 = 0; k2 < t->nanc[l]; ++k2) {
        int j1 = t->anc_node[l][k1], j2 = t->anc_node[l][k2];
        int c1 = t->cidx[j1], c2 = t->cidx[j2];
        double c = t->w[l] * t->anc_coef[l][k1] * t->anc_coef[l][k2];
        for (int m1 = 0; m1 < 3; ++m1)
          for (int m2 = 0; m2 < 3; ++m2) {
            double s = 0.0;
            for (int I = 0; I < 6; ++I) s += ws->Nm[j1][I][m1] * DN[k2][I][m2];
            ws->J[(size_t)(3 * c1 + m1) * n + 3 * c2 + m2] += c * s;
          }
      }
  }
}

/* Cholesky J = L L^T in the paper's laminate order (leaves-to-root).  In this
 * order the factor has no fill: L(r, c) can be non-zero only when the laminate
 * of row r is the laminate of column c or one of its ancestors; the sums run
 * over the descendants of the column's laminate. */
static int cholesky(const or_tree* t, or_work* ws) {
  int n = 3 * t->nact;
  double* L = ws->J;
#define LL(r, c) L[(size_t)(r) * n + (c)]
  for (int cn = 0; cn < t->nact; ++cn)
    for (int a = 0; a < 3; ++a) {
      int c = 3 * cn + a;
      double s = LL(c, c);
      for (int u = 0; u < t->n_desc[cn]; ++u)
        for (int b = 0; b < 3; ++b) { double v = LL(c, 3 * t->desc[cn][u] + b); s -= v * v; }
      for (int b = 0; b < a; ++b) { double v = LL(c, 3 * cn + b); s -= v * v; }
      if (!(s > 0.0)) return -1;
      double d = sqrt(s);
      LL(c, c) = d;
      /* rows below c in the pattern: same laminate, then its ancestors */
      int rows[3 + 3 * OR_KMAX], nr = 0;
      for (int b = a + 1; b < 3; ++b) rows[nr++] = 3 * cn + b;
      for (int u = 0; u < t->n_anc[cn]; ++u)
        for (int b = 0; b < 3; ++b) rows[nr++] = 3 * t->anc[cn][u] + b;
      for (int x = 0; x < nr; ++x) {
        int r = rows[x];
        double v = LL(r, c);
        for (int u = 0; u < t->n_desc[cn]; ++u)
          for (int b = 0; b < 3; ++b) { int k = 3 * t->desc[cn][u] + b; v -= LL(r, k) * LL(c, k); }
        for (int b = 0; b < a; ++b) { int k = 3 * cn + b; v -= LL(r, k) * LL(c, k); }
        LL(r, c) = v / d;
      }
    }
  return 0;
}

/* solve L L^T x = b in place */
static void chol_solve(const or_tree* t, or_work* ws, double* x) {
  int n = 3 * t->nact;
  double* L = ws->J;
  for (int rn = 0; rn < t->nact; ++rn)
    for (int a = 0; a < 3; ++a) {
      int r = 3 * rn + a;
      double s = x[r];
      for (int u = 0; u < t->n_desc[rn]; ++u)
        for (int b = 0; b < 3; ++b) { int k = 3 * t->desc[rn][u] + b; s -= LL(r, k) * x[k]; }
      for (int b = 0; b < a; ++b) s -= LL(r, 3 * rn + b) * x[3 * rn + b];
      x[r] = s / LL(r, r);
    }
  for (int cn = t->nact - 1; cn >= 0; --cn)
    for (int a = 2; a >= 0; --a) {
      int c = 3 * cn + a;
      double s = x[c];
      for (int b = a + 1; b < 3; ++b) s -= LL(3 * cn + b, c) * x[3 * cn + b];
      for (int u = 0; u < t->n_anc[cn]; ++u)
        for (int b = 0; b < 3; ++b) { int r = 3 * t->anc[cn][u] + b; s -= LL(r, c) * x[r]; }
      x[c] = s / LL(c, c);
    }
#undef LL
}

static double mandel_norm(const double v[6]) {
  double s = 0.0;
  for (int I = 0; I < 6; ++I) s += v[I] * v[I];
  return sqrt(s);
}

/* C_algo = [I..I]^T W [D + D A dadE], with dadE from the six-RHS system. */
static void algorithmic_tangent(const or_tree* t, or_work* ws, double C[6][6]) {
  int n = 3 * t->nact;
  double* X = (double*)malloc(sizeof(double) * (size_t)n * 6);
  for (int col = 0; col < 6; ++col) {
    double* x = X + (size_t)col * n;
    for (int r = 0; r < n; ++r) x[r] = 0.0;
    /* rhs = -A^T W D e_col */
    for (int l = 0; l < t->L; ++l)
      for (int k = 0; k < t->nanc[l]; ++k) {
        int j = t->anc_node[l][k];
        double c = t->anc_coef[l][k] * t->w[l];
        for (int m = 0; m < 3; ++m) {
          double s = 0.0;
          for (int I = 0; I < 6; ++I) s += ws->Nm[j][I][m] * ws->D[l][I][col];
          x[3 * t->cidx[j] + m] -= c * s;
        }
      }
    chol_solve(t, ws, x);
  }
  for (int I = 0; I < 6; ++I) for (int J = 0; J < 6; ++J) C[I][J] = 0.0;
  for (int l = 0; l < t->L; ++l) {
    double G[6][6];  /* I + (A dadE)_l */
    for (int I = 0; I < 6; ++I) for (int J = 0; J < 6; ++J) G[I][J] = (I == J) ? 1.0 : 0.0;
    for (int k = 0; k < t->nanc[l]; ++k) {
      int j = t->anc_node[l][k];
      double c = t->anc_coef[l][k];
      for (int I = 0; I < 6; ++I)
        for (int col = 0; col < 6; ++col)
          for (int m = 0; m < 3; ++m) G[I][col] += c * ws->Nm[j][I][m] * X[(size_t)col * n + 3 * t->cidx[j] + m];
    }
    for (int I = 0; I < 6; ++I)
      for (int J = 0; J < 6; ++J) {
        double s = 0.0;
        for (int P = 0; P < 6; ++P) s += ws->D[l][I][P] * G[P][J];
        C[I][J] += t->w[l] * s;
      }
  }
  free(X);
}

/* strain/stress rotation with the frame Q (columns = principal directions):
 * local = Q^T global Q ; global = Q local Q^T */
static void rotate_sym(const double Q[9], const double v[6], double out[6], int to_local) {
  double T[3][3], S[3][3];
  mandel_to_tensor(v, T);
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      double s = 0.0;
      for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b)
          s += to_local ? Q[a * 3 + i] * T[a][b] * Q[b * 3 + j] : Q[i * 3 + a] * T[a][b] * Q[j * 3 + b];
      S[i][j] = s;
    }
  tensor_to_mandel(S, out);
}
/* fourth-order rotation of a Mandel 6x6 stiffness to the global frame:
 * C_ijkl = Q_ia Q_jb Q_kc Q_ld C_abcd */
static void rotate_stiffness(const double Q[9], double Cl[6][6], double Cg[6][6]) {
  double (*c4)[3][3][3] = (double (*)[3][3][3])malloc(sizeof(double) * 81);
  double (*g4)[3][3][3] = (double (*)[3][3][3])malloc(sizeof(double) * 81);
  for (int I = 0; I < 6; ++I)
    for (int J = 0; J < 6; ++J) {
      double v = Cl[I][J] / (mweight(I) * mweight(J));
      int a = MI[I][0], b = MI[I][1], c = MI[J][0], d = MI[J][1];
      c4[a][b][c][d] = c4[b][a][c][d] = c4[a][b][d][c] = c4[b][a][d][c] = v;
    }
  for (int i = 0; i < 3; ++i) for (int j = 0; j < 3; ++j) for (int k = 0; k < 3; ++k) for (int l = 0; l < 3; ++l) {
    double s = 0.0;
    for (int a = 0; a < 3; ++a) for (int b = 0; b < 3; ++b) for (int c = 0; c < 3; ++c) for (int d = 0; d < 3; ++d)
      s += Q[i * 3 + a] * Q[j * 3 + b] * Q[k * 3 + c] * Q[l * 3 + d] * c4[a][b][c][d];
    g4[i][j][k][l] = s;
  }
  for (int I = 0; I < 6; ++I)
    for (int J = 0; J < 6; ++J)
      Cg[I][J] = g4[MI[I][0]][MI[I][1]][MI[J][0]][MI[J][1]] * mweight(I) * mweight(J);
  free(c4); free(g4);
}

static int all_finite(const double* v, int n) {
  for (int i = 0; i < n; ++i) if (!isfinite(v[i])) return 0;
  return 1;
}

/* One material-point update (Sec. 3.2, Sec. 4.6). */
static void update_point(const or_tree* t, or_work* ws, long n, long pt, const double* lam, const double* Q,
                         const double* E_n, const double* dE, const double* state_in, double* state_out,
                         double* stress, double* tangent, int* iters, int* status, double* yield_gap) {
  int N = t->nact, nzf = 6 * t->nz;
  const double* Qp = Q + 9 * pt;
  double Eg[6], E[6];
  for (int I = 0; I < 6; ++I) Eg[I] = E_n[6 * pt + I] + dE[6 * pt + I];
  rotate_sym(Qp, Eg, E, 1);
  normals(t, lam[2 * pt], lam[2 * pt + 1], ws->nrm);
  for (int j = 0; j < t->N; ++j) sym_operator(ws->nrm[j], ws->Nm[j]);
  /* z^n of every leaf (elastic leaves: zeros, unused) */
  for (int l = 0; l < t->L; ++l) {
    for (int c = 0; c < 7; ++c) ws->z_n[l][c] = 0.0;
    int s = t->z_slot[l];
    if (s >= 0) {
      const double* b = state_in + (size_t)(6 * s) * n + pt;
      ws->z_n[l][0] = b[0];
      ws->z_n[l][1] = b[(size_t)1 * n]; ws->z_n[l][2] = b[(size_t)2 * n];
      ws->z_n[l][3] = -(b[(size_t)1 * n] + b[(size_t)2 * n]);
      ws->z_n[l][4] = b[(size_t)3 * n]; ws->z_n[l][5] = b[(size_t)4 * n]; ws->z_n[l][6] = b[(size_t)5 * n];
    }
  }
  for (int r = 0; r < 3 * N; ++r) ws->a[r] = state_in[(size_t)(nzf + r) * n + pt];
  int st = 0, it = 0;
  int finite_in = all_finite(E, 6) && all_finite(ws->a, 3 * N);
  for (int l = 0; l < t->L; ++l) finite_in = finite_in && all_finite(ws->z_n[l], 7);
  double rn = finite_in ? evaluate(t, ws, E, ws->a) : NAN;
  for (;;) {
    if (!isfinite(rn) || !all_finite(ws->sbar, 6)) { st = 2; break; }
    if (rn <= t->tol * (double)N * mandel_norm(ws->sbar)) break;
    if (it >= t->max_iter) { st = 1; break; }
    assemble_J(t, ws);
    if (cholesky(t, ws) != 0) { st = 2; break; }
    for (int r = 0; r < 3 * N; ++r) ws->da[r] = -ws->R[r];
    chol_solve(t, ws, ws->da);
    double s = 1.0;
    if (!t->line_search) {
      for (int r = 0; r < 3 * N; ++r) ws->a[r] += ws->da[r];
      rn = evaluate(t, ws, E, ws->a);
    } else {
      /* backtracking: halve the step while the residual norm does not decrease, at most 8 times */
      int ok = 0;
      for (int h = 0; h <= 8; ++h) {
        for (int r = 0; r < 3 * N; ++r) ws->a_try[r] = ws->a[r] + s * ws->da[r];
        double rt = evaluate(t, ws, E, ws->a_try);
        if (rt < rn) { ok = 1; rn = rt; break; }
        s *= 0.5;
      }
      if (!ok) { rn = evaluate(t, ws, E, ws->a); st = 3; it++; break; }
      for (int r = 0; r < 3 * N; ++r) ws->a[r] = ws->a_try[r];
    }
    it++;
  }
  double Cl[6][6], Cg[6][6], sg[6];
  if (st != 2) {
    assemble_J(t, ws);
    if (cholesky(t, ws) != 0) st = 2;
  }
  if (st != 2) {
    algorithmic_tangent(t, ws, Cl);
    rotate_stiffness(Qp, Cl, Cg);
    rotate_sym(Qp, ws->sbar, sg, 0);
  } else {
    for (int I = 0; I < 6; ++I) { sg[I] = NAN; for (int J = 0; J < 6; ++J) Cg[I][J] = NAN; }
  }
  for (int I = 0; I < 6; ++I) stress[6 * pt + I] = sg[I];
  for (int I = 0; I < 6; ++I) for (int J = 0; J < 6; ++J) tangent[36 * pt + 6 * I + J] = Cg[I][J];
  iters[pt] = it; status[pt] = st;
  if (yield_gap) yield_gap[pt] = ws->gap;
  /* z^{n+1} from the return mapping at the final iterate, and the jumps a^{n+1};
   * a non-finite failure (status 2) writes NaN throughout */
  for (int l = 0; l < t->L; ++l) {
    int s = t->z_slot[l];
    if (s < 0) continue;
    double* b = state_out + (size_t)(6 * s) * n + pt;
    const double* z = ws->z_new[l];
    double nan = NAN;
    b[0] = st == 2 ? nan : z[0];
    b[(size_t)1 * n] = st == 2 ? nan : z[1]; b[(size_t)2 * n] = st == 2 ? nan : z[2];
    b[(size_t)3 * n] = st == 2 ? nan : z[4]; b[(size_t)4 * n] = st == 2 ? nan : z[5];
    b[(size_t)5 * n] = st == 2 ? nan : z[6];
  }
  for (int r = 0; r < 3 * N; ++r) state_out[(size_t)(nzf + r) * n + pt] = st == 2 ? NAN : ws->a[r];
}

static or_work* work_alloc(const or_tree* t) {
  or_work* ws = (or_work*)calloc(1, sizeof(or_work));
  size_t n = 3 * (size_t)(t->nact > 0 ? t->nact : 1);
  ws->J = (double*)calloc(n * n, sizeof(double));
  return ws;
}
static void work_free(or_work* ws) { free(ws->J); free(ws); }

/* ================================================================== */
/* Exported entry points (ctypes).  mat = (kind, E, nu, sigma0, H, sigma_inf, k0)
 * for phase 1 then phase 2 (H is k_inf for kind 2).  Return 0 on success, < 0 on invalid arguments.           */

int oracle_state_size(int K, const double* mat) {
  or_tree t;
  double w[OR_LMAX];
  if (K < 1 || K > OR_KMAX) return -1;
  for (int l = 0; l < (1 << K); ++l) w[l] = 1.0;
  double pq[OR_NMAX * 3] = {0};
  if (tree_init(&t, K, 3, pq, pq, w, mat, 1e-12, 1, 0) != 0) return -1;
  int s = 6 * t.nz + 3 * t.nact;
  tree_free(&t);
  return s;
}

/* doubles of state per point for the given weights (compressed tree) */
int oracle_state_size_w(int K, const double* mat, const double* w) {
  or_tree t;
  if (K < 1 || K > OR_KMAX) return -1;
  double pq[OR_NMAX * 6] = {0};
  if (tree_init(&t, K, 3, pq, pq, w, mat, 1e-12, 1, 0) != 0) return -1;
  int s = 6 * t.nz + 3 * t.nact;
  tree_free(&t);
  return s;
}

int oracle_update(int K, int M, const double* p, const double* q, const double* w, const double* mat,
                  double tol, int max_iter, int line_search, long n, const double* lam, const double* Q,
                  const double* E_n, const double* dE, const double* state_in, double* state_out,
                  double* stress, double* tangent, int* iters, int* status, double* yield_gap, int nthreads) {
  or_tree t;
  if (tree_init(&t, K, M, p, q, w, mat, tol, max_iter, line_search) != 0) return -1;
  if (nthreads <= 0) nthreads = 1;
#pragma omp parallel num_threads(nthreads)
  {
    or_work* ws = work_alloc(&t);
#pragma omp for schedule(dynamic, 1)
    for (long pt = 0; pt < n; ++pt)
      update_point(&t, ws, n, pt, lam, Q, E_n, dE, state_in, state_out, stress, tangent, iters, status, yield_gap);
    work_free(ws);
  }
  tree_free(&t);
  return 0;
}

/* normals [N][3] of one orientation (lam1, lam2), paper ordering */
int oracle_normals(int K, int M, const double* p, const double* q, double lam1, double lam2, double* out) {
  or_tree t;
  double w[OR_LMAX];
  double mat[2 * OR_MAT] = {0, 1, 0.2, 0, 0, 0, 0, 0, 1, 0.2, 0, 0, 0, 0};
  if (K < 1 || K > OR_KMAX) return -1;
  for (int l = 0; l < (1 << K); ++l) w[l] = 1.0;
  if (tree_init(&t, K, M, p, q, w, mat, 1e-12, 1, 0) != 0) return -1;
  double (*nrm)[3] = (double (*)[3])malloc(sizeof(double) * 3 * t.N);
  normals(&t, lam1, lam2, nrm);
  for (int j = 0; j < t.N; ++j) for (int c = 0; c < 3; ++c) out[3 * j + c] = nrm[j][c];
  free(nrm);
  tree_free(&t);
  return 0;
}

int oracle_barycentric(double lam1, double lam2, double* phi) { barycentric(lam1, lam2, phi); return 0; }

/* dense gradient operator A [6 * 2^K][3 * N] for one orientation */
int oracle_gradient_operator(int K, int M, const double* p, const double* q, const double* w,
                             double lam1, double lam2, double* A) {
  or_tree t;
  double mat[2 * OR_MAT] = {0, 1, 0.2, 0, 0, 0, 0, 0, 1, 0.2, 0, 0, 0, 0};
  if (tree_init(&t, K, M, p, q, w, mat, 1e-12, 1, 0) != 0) return -1;
  or_work* ws = work_alloc(&t);
  normals(&t, lam1, lam2, ws->nrm);
  for (int j = 0; j < t.N; ++j) sym_operator(ws->nrm[j], ws->Nm[j]);
  int nc = 3 * t.N;
  memset(A, 0, sizeof(double) * 6 * t.L * nc);
  for (int l = 0; l < t.L; ++l)
    for (int k = 0; k < t.nanc[l]; ++k) {
      int j = t.anc_node[l][k];
      for (int I = 0; I < 6; ++I)
        for (int m = 0; m < 3; ++m) A[(size_t)(6 * l + I) * nc + 3 * j + m] = t.anc_coef[l][k] * ws->Nm[j][I][m];
    }
  work_free(ws);
  tree_free(&t);
  return 0;
}

/* Newton system at one iterate (local frame): J (dense, full, before
 * factorisation), R = A^T W sigma, the Cholesky step da = -J^{-1} R, the leaf
 * strains/stresses and sigma_bar.  z_n: [2^K][7] per leaf (alpha_bar, ep6). */
int oracle_newton_system(int K, int M, const double* p, const double* q, const double* w, const double* mat,
                         double lam1, double lam2, const double* E, const double* a, const double* z_n,
                         double* J, double* R, double* da, double* eps, double* sig, double* sbar) {
  or_tree t;
  if (tree_init(&t, K, M, p, q, w, mat, 1e-12, 1, 0) != 0) return -1;
  or_work* ws = work_alloc(&t);
  normals(&t, lam1, lam2, ws->nrm);
  for (int j = 0; j < t.N; ++j) sym_operator(ws->nrm[j], ws->Nm[j]);
  for (int l = 0; l < t.L; ++l) for (int c = 0; c < 7; ++c) ws->z_n[l][c] = z_n[7 * l + c];
  evaluate(&t, ws, E, a);
  int n = 3 * t.nact;
  assemble_J(&t, ws);
  memcpy(J, ws->J, sizeof(double) * (size_t)n * n);
  int rc = cholesky(&t, ws);
  for (int r = 0; r < n; ++r) { R[r] = ws->R[r]; da[r] = -ws->R[r]; }
  if (rc == 0) chol_solve(&t, ws, da);
  for (int l = 0; l < t.L; ++l) for (int I = 0; I < 6; ++I) { eps[6 * l + I] = ws->eps[l][I]; sig[6 * l + I] = ws->sig[l][I]; }
  for (int I = 0; I < 6; ++I) sbar[I] = ws->sbar[I];
  work_free(ws);
  tree_free(&t);
  return rc;
}

/* one leaf law evaluation: phase = (kind, E, nu, sigma0, H, sigma_inf, k0); z = (alpha_bar, ep6) */
int oracle_phase_law(const double* phase, const double* eps, const double* z_n, double* sig, double* D,
                     double* z_new) {
  or_phase ph = {(int)phase[0], phase[1], phase[2], phase[3], phase[4], phase[5], phase[6]};
  double Dm[6][6], zz[7];
  phase_law(&ph, eps, z_n, sig, Dm, zz, NULL);
  for (int I = 0; I < 6; ++I) for (int J = 0; J < 6; ++J) D[6 * I + J] = Dm[I][J];
  if (ph.kind == 0) for (int c = 0; c < 7; ++c) zz[c] = z_n[c];
  for (int c = 0; c < 7; ++c) z_new[c] = zz[c];
  return 0;
}

/* fourth-order rotation of a Mandel stiffness and Mandel rotation of a
 * symmetric tensor (exposed for the convention tests) */
int oracle_rotate(const double* Q, const double* Cl, const double* vl, double* Cg, double* vg) {
  double a[6][6], b[6][6];
  for (int I = 0; I < 6; ++I) for (int J = 0; J < 6; ++J) a[I][J] = Cl[6 * I + J];
  rotate_stiffness(Q, a, b);
  for (int I = 0; I < 6; ++I) for (int J = 0; J < 6; ++J) Cg[6 * I + J] = b[I][J];
  rotate_sym(Q, vl, vg, 0);
  return 0;
}

/* ================================================================== */
/* Exact derivatives by forward-mode dual numbers.
 *
 * A dual number x = v + d e (e^2 = 0) carries a value v and the derivative d
 * of that value along one chosen direction of the inputs.  Every operation
 * below applies the matching rule of differentiation, so each function written
 * on duals returns the exact directional derivative of what its double
 * counterpart above computes (no step size, no truncation error):
 *   - the normals of Sec. 2.3 through the angle coefficients p, q;
 *   - the normalised leaf weights and the volume fractions of Sec. 2.1
 *     through the leaf weights w as given (before their normalisation);
 *   - the leaf strains E + A a (Sec. 3.2) through E, a, the normals and the
 *     fractions;
 *   - the phase laws (Sec. 4.1; the exponential-linear law's scalar Newton
 *     iteration carries its derivative along and ends at the implicit
 *     derivative of the consistency condition);
 *   - the residual R = A^T W sigma (Eq. euler_lagrange), the effective stress
 *     sum w_i sigma_i and the algorithmic tangent of Eq. (lin_system_da_dE),
 *     whose six right-hand sides are differentiated through the Cholesky
 *     solve: d(J^-1 b) = J^-1 (db - dJ J^-1 b).
 * oracle_gradient assembles from these partial derivatives the
 * implicit-function gradient of the converged solve (Sec. 3.2). */
typedef struct { double v, d; } dual;
static dual dn(double v, double d) { dual r; r.v = v; r.d = d; return r; }
static dual dc(double v) { return dn(v, 0.0); }
static dual d_add(dual a, dual b) { return dn(a.v + b.v, a.d + b.d); }
static dual d_sub(dual a, dual b) { return dn(a.v - b.v, a.d - b.d); }
static dual d_mul(dual a, dual b) { return dn(a.v * b.v, a.d * b.v + a.v * b.d); }
static dual d_div(dual a, dual b) { return dn(a.v / b.v, (a.d * b.v - a.v * b.d) / (b.v * b.v)); }
static dual d_scale(double s, dual a) { return dn(s * a.v, s * a.d); }
static dual d_sqrt(dual a) { double r = sqrt(a.v); return dn(r, a.d / (2.0 * r)); }
static dual d_sin(dual a) { return dn(sin(a.v), cos(a.v) * a.d); }
static dual d_cos(dual a) { return dn(cos(a.v), -sin(a.v) * a.d); }
static dual d_exp(dual a) { double e = exp(a.v); return dn(e, e * a.d); }
/* a + b c */
static dual d_fma(dual a, dual b, dual c) { return d_add(a, d_mul(b, c)); }

/* sigma_Y and its slope at a dual alpha_bar (yield_stress on duals) */
static dual yield_stress_dual(const or_phase* ph, dual ab, dual* slope) {
  if (ph->kind == 2 && ph->sinf > ph->s0) {
    double ds = ph->sinf - ph->s0, r = (ph->k0 - ph->H) / ds;
    dual e = d_exp(d_scale(-r, ab));
    if (slope) *slope = d_add(dc(ph->H), d_scale(ph->k0 - ph->H, e));
    return d_add(d_add(dc(ph->s0), d_scale(ph->H, ab)), d_scale(ds, d_sub(dc(1.0), e)));
  }
  if (slope) *slope = dc(ph->H);
  return d_add(dc(ph->s0), d_scale(ph->H, ab));
}

/* phase_law on a dual strain; z_n is fixed (the state of the last increment).
 * The elastic/plastic branch is the one the value takes. */
static void phase_law_dual(const or_phase* ph, const dual eps[6], const double z_n[7], dual sig[6], dual D[6][6]) {
  double K = ph->E / (3.0 * (1.0 - 2.0 * ph->nu));
  double G = ph->E / (2.0 * (1.0 + ph->nu));
  dual tr = d_add(d_add(eps[0], eps[1]), eps[2]);
  dual dev[6];
  for (int I = 0; I < 6; ++I) dev[I] = I < 3 ? d_sub(eps[I], d_scale(1.0 / 3.0, tr)) : eps[I];
  double Idev[6][6];
  for (int I = 0; I < 6; ++I)
    for (int J = 0; J < 6; ++J) Idev[I][J] = (I == J ? 1.0 : 0.0) - ((I < 3 && J < 3) ? 1.0 / 3.0 : 0.0);
  int elastic = ph->kind == 0;
  dual str[6], ns = dc(0.0), f = dc(-1.0);
  if (!elastic) {
    dual nrm2 = dc(0.0);
    for (int I = 0; I < 6; ++I) { str[I] = d_scale(2.0 * G, d_sub(dev[I], dc(z_n[1 + I]))); nrm2 = d_fma(nrm2, str[I], str[I]); }
    ns = d_sqrt(nrm2);
    f = d_sub(ns, dc(sqrt(2.0 / 3.0) * yield_stress(ph, z_n[0], NULL)));
  }
  if (elastic || f.v <= 0.0) {
    for (int I = 0; I < 6; ++I)
      sig[I] = d_add(I < 3 ? d_scale(K, tr) : dc(0.0), elastic ? d_scale(2.0 * G, dev[I]) : str[I]);
    if (D)
      for (int I = 0; I < 6; ++I)
        for (int J = 0; J < 6; ++J) D[I][J] = dc(((I < 3 && J < 3) ? K : 0.0) + 2.0 * G * Idev[I][J]);
    return;
  }
  dual dg, Hp;
  if (ph->kind == 1) {
    dg = d_scale(1.0 / (2.0 * G + 2.0 * ph->H / 3.0), f);
    Hp = dc(ph->H);
  } else {
    dg = dc(0.0);
    for (int it = 0; it < 100; ++it) {
      dual slope;
      dual sy = yield_stress_dual(ph, d_add(dc(z_n[0]), d_scale(sqrt(2.0 / 3.0), dg)), &slope);
      dual r = d_sub(d_sub(ns, d_scale(2.0 * G, dg)), d_scale(sqrt(2.0 / 3.0), sy));
      dual step = d_div(r, d_add(dc(2.0 * G), d_scale(2.0 / 3.0, slope)));
      dg = d_add(dg, step);
      if (fabs(step.v) <= 1e-15 * dg.v) break;
    }
    yield_stress_dual(ph, d_add(dc(z_n[0]), d_scale(sqrt(2.0 / 3.0), dg)), &Hp);
  }
  dual nh[6];
  for (int I = 0; I < 6; ++I) nh[I] = d_div(str[I], ns);
  dual th = d_sub(dc(1.0), d_div(d_scale(2.0 * G, dg), ns));
  dual thb = d_sub(d_div(dc(1.0), d_add(dc(1.0), d_scale(1.0 / (3.0 * G), Hp))), d_sub(dc(1.0), th));
  for (int I = 0; I < 6; ++I)
    sig[I] = d_sub(d_add(I < 3 ? d_scale(K, tr) : dc(0.0), str[I]), d_scale(2.0 * G, d_mul(dg, nh[I])));
  if (D)
    for (int I = 0; I < 6; ++I)
      for (int J = 0; J < 6; ++J)
        D[I][J] = d_sub(d_add(dc((I < 3 && J < 3) ? K : 0.0), d_scale(2.0 * G * Idev[I][J], th)),
                        d_scale(2.0 * G, d_mul(thb, d_mul(nh[I], nh[J]))));
}

/* Per-point dual work space. */
typedef struct {
  dual nrm[OR_NMAX][3];
  double Nv[OR_NMAX][6][3], Nd[OR_NMAX][6][3];   /* N(n) and its derivative (N is linear in n) */
  dual wn[OR_LMAX], c1[OR_NMAX], c2[OR_NMAX];
  dual eps[OR_LMAX][6], sig[OR_LMAX][6], D[OR_LMAX][6][6];
  dual R[3 * OR_NMAX], sbar[6], C[6][6];
} or_dual;

/* entry (I, m) of N_j on duals */
static dual Nm_dual(const or_dual* u, int j, int I, int m) { return dn(u->Nv[j][I][m], u->Nd[j][I][m]); }
/* coefficient of laminate j's block in leaf l's row of A: -c2 (left subtree) or +c1 (right) */
static dual coef_dual(const or_tree* t, const or_dual* u, int l, int k) {
  int j = t->anc_node[l][k];
  return t->anc_coef[l][k] < 0.0 ? d_scale(-1.0, u->c2[j]) : u->c1[j];
}

/* One evaluation at (p + e dp, q + e dq, w + e dw, E + e dE, a + e da) with z^n
 * fixed: R, sigma_bar and (when fac holds the Cholesky factor of J at the
 * values) the algorithmic tangent, each with its derivative.  w_raw are the
 * weights as given; t was initialised with them. */
static void eval_dual(const or_tree* t, or_dual* u, const double* w_raw, const double* dp, const double* dq,
                      const double* dw, double lam1, double lam2, const double* E, const double* dE,
                      const double* a, const double* da, const double z_n[][7], or_work* fac) {
  /* normals: alpha_j = p_j . phi, beta_j = q_j . phi (phi fixed by the orientation) */
  double v[3], ph[6];
  barycentric(lam1, lam2, v);
  shape_functions(t->M, v, ph);
  for (int j = 0; j < t->N; ++j) {
    dual al = dc(0.0), be = dc(0.0);
    for (int m = 0; m < t->M; ++m) {
      al = d_add(al, dn(t->p[j * t->M + m] * ph[m], dp[j * t->M + m] * ph[m]));
      be = d_add(be, dn(t->q[j * t->M + m] * ph[m], dq[j * t->M + m] * ph[m]));
    }
    u->nrm[j][0] = d_mul(d_sin(al), d_cos(be));
    u->nrm[j][1] = d_mul(d_sin(al), d_sin(be));
    u->nrm[j][2] = d_cos(al);
    double nv[3] = {u->nrm[j][0].v, u->nrm[j][1].v, u->nrm[j][2].v};
    double nd[3] = {u->nrm[j][0].d, u->nrm[j][1].d, u->nrm[j][2].d};
    sym_operator(nv, u->Nv[j]);
    sym_operator(nd, u->Nd[j]);
  }
  /* weights normalised to sum 1, subtree weights and fractions, leaves -> root */
  dual sw = dc(0.0);
  for (int l = 0; l < t->L; ++l) sw = d_add(sw, dn(w_raw[l], dw[l]));
  dual Wlev[OR_LMAX];
  for (int l = 0; l < t->L; ++l) { u->wn[l] = d_div(dn(w_raw[l], dw[l]), sw); Wlev[l] = u->wn[l]; }
  for (int k = t->K; k >= 1; --k)
    for (int i = 1; i <= (1 << (k - 1)); ++i) {
      dual wl = Wlev[2 * i - 2], wr = Wlev[2 * i - 1], W = d_add(wl, wr);
      int j = node_index(t->K, k, i);
      u->c1[j] = W.v > 0.0 ? d_div(wl, W) : dc(0.5);
      u->c2[j] = d_sub(dc(1.0), u->c1[j]);
      Wlev[i - 1] = W;
    }
  /* leaf strains, laws, effective stress and residual */
  for (int l = 0; l < t->L; ++l) {
    for (int I = 0; I < 6; ++I) u->eps[l][I] = dn(E[I], dE[I]);
    for (int k = 0; k < t->nanc[l]; ++k) {
      int j = t->anc_node[l][k], cj = t->cidx[j];
      dual c = coef_dual(t, u, l, k);
      for (int I = 0; I < 6; ++I)
        for (int m = 0; m < 3; ++m)
          u->eps[l][I] = d_fma(u->eps[l][I], c, d_mul(Nm_dual(u, j, I, m), dn(a[3 * cj + m], da[3 * cj + m])));
    }
    phase_law_dual(&t->ph[l % 2], u->eps[l], z_n[l], u->sig[l], fac ? u->D[l] : NULL);
  }
  for (int I = 0; I < 6; ++I) u->sbar[I] = dc(0.0);
  for (int l = 0; l < t->L; ++l)
    for (int I = 0; I < 6; ++I) u->sbar[I] = d_fma(u->sbar[I], u->wn[l], u->sig[l][I]);
  for (int r = 0; r < 3 * t->nact; ++r) u->R[r] = dc(0.0);
  for (int l = 0; l < t->L; ++l)
    for (int k = 0; k < t->nanc[l]; ++k) {
      int j = t->anc_node[l][k], cj = t->cidx[j];
      dual c = d_mul(coef_dual(t, u, l, k), u->wn[l]);
      for (int m = 0; m < 3; ++m)
        for (int I = 0; I < 6; ++I)
          u->R[3 * cj + m] = d_fma(u->R[3 * cj + m], c, d_mul(Nm_dual(u, j, I, m), u->sig[l][I]));
    }
  if (!fac) return;
  /* algorithmic tangent C = sum_l w_l D_l (I + A_l X), J X = -A^T W D [I..I]:
   * X from the factor of J at the values; dX = J^-1 (dB - dJ X), with dJ the
   * derivative of J = A^T W D A assembled on duals and dB that of the RHS. */
  int n = 3 * t->nact;
  double* dJ = (double*)calloc((size_t)n * n, sizeof(double));
  double* X = (double*)malloc(sizeof(double) * (size_t)n * 6);
  double* dX = (double*)malloc(sizeof(double) * (size_t)n * 6);
  for (int i = 0; i < n * 6; ++i) { X[i] = 0.0; dX[i] = 0.0; }
  for (int l = 0; l < t->L; ++l) {
    dual DN[OR_KMAX][6][3];
    for (int k = 0; k < t->nanc[l]; ++k) {
      int j = t->anc_node[l][k];
      for (int I = 0; I < 6; ++I)
        for (int m = 0; m < 3; ++m) {
          dual s = dc(0.0);
          for (int P = 0; P < 6; ++P) s = d_fma(s, u->D[l][I][P], Nm_dual(u, j, P, m));
          DN[k][I][m] = s;
        }
    }
    for (int k1 = 0; k1 < t->nanc[l]; ++k1) {
      int j1 = t->anc_node[l][k1], r1 = 3 * t->cidx[j1];
      dual cw1 = d_mul(u->wn[l], coef_dual(t, u, l, k1));
      for (int k2 = 0; k2 < t->nanc[l]; ++k2) {
        int r2 = 3 * t->cidx[t->anc_node[l][k2]];
        dual c = d_mul(cw1, coef_dual(t, u, l, k2));
        for (int m1 = 0; m1 < 3; ++m1)
          for (int m2 = 0; m2 < 3; ++m2) {
            dual s = dc(0.0);
            for (int I = 0; I < 6; ++I) s = d_fma(s, Nm_dual(u, j1, I, m1), DN[k2][I][m2]);
            dJ[(size_t)(r1 + m1) * n + r2 + m2] += d_mul(c, s).d;
          }
      }
      /* right-hand sides -A^T W D e_col and their derivatives */
      for (int col = 0; col < 6; ++col)
        for (int m = 0; m < 3; ++m) {
          dual s = dc(0.0);
          for (int I = 0; I < 6; ++I) s = d_fma(s, Nm_dual(u, j1, I, m), u->D[l][I][col]);
          dual b = d_mul(cw1, s);
          X[(size_t)col * n + r1 + m] -= b.v;
          dX[(size_t)col * n + r1 + m] -= b.d;
        }
    }
  }
  for (int col = 0; col < 6; ++col) {
    double* x = X + (size_t)col * n;
    double* dx = dX + (size_t)col * n;
    chol_solve(t, fac, x);
    for (int r = 0; r < n; ++r) {
      double s = 0.0;
      for (int c = 0; c < n; ++c) s += dJ[(size_t)r * n + c] * x[c];
      dx[r] -= s;
    }
    chol_solve(t, fac, dx);
  }
  for (int I = 0; I < 6; ++I) for (int J = 0; J < 6; ++J) u->C[I][J] = dc(0.0);
  for (int l = 0; l < t->L; ++l) {
    dual Gm[6][6];   /* I + (A X)_l */
    for (int I = 0; I < 6; ++I) for (int J = 0; J < 6; ++J) Gm[I][J] = dc(I == J ? 1.0 : 0.0);
    for (int k = 0; k < t->nanc[l]; ++k) {
      int j = t->anc_node[l][k], r0 = 3 * t->cidx[j];
      dual c = coef_dual(t, u, l, k);
      for (int I = 0; I < 6; ++I)
        for (int col = 0; col < 6; ++col)
          for (int m = 0; m < 3; ++m)
            Gm[I][col] = d_fma(Gm[I][col], c, d_mul(Nm_dual(u, j, I, m),
                                                    dn(X[(size_t)col * n + r0 + m], dX[(size_t)col * n + r0 + m])));
    }
    for (int I = 0; I < 6; ++I)
      for (int J = 0; J < 6; ++J) {
        dual s = dc(0.0);
        for (int P = 0; P < 6; ++P) s = d_fma(s, u->D[l][I][P], Gm[P][J]);
        u->C[I][J] = d_fma(u->C[I][J], u->wn[l], s);
      }
  }
  free(dJ); free(X); free(dX);
}

/* value pass at the given point: the Cholesky factor of J = A^T W D A in ws->J */
static int factor_at(const or_tree* t, or_work* ws, double lam1, double lam2, const double* E, const double* a,
                     const double z_n[][7]) {
  normals(t, lam1, lam2, ws->nrm);
  for (int j = 0; j < t->N; ++j) sym_operator(ws->nrm[j], ws->Nm[j]);
  for (int l = 0; l < t->L; ++l) for (int c = 0; c < 7; ++c) ws->z_n[l][c] = z_n[l][c];
  evaluate(t, ws, E, a);
  assemble_J(t, ws);
  return cholesky(t, ws);
}

/* derivative of g . sigma_bar + G : C along the direction of the last eval_dual */
static double seed_value(const or_dual* u, const double* g, const double* Gt) {
  double s = 0.0;
  for (int I = 0; I < 6; ++I) s += g[I] * u->sbar[I].d;
  if (Gt)
    for (int I = 0; I < 6; ++I)
      for (int J = 0; J < 6; ++J) s += Gt[6 * I + J] * u->C[I][J].d;
  return s;
}

/* One directional derivative (local frame): R, sigma_bar and, if want_tangent,
 * the algorithmic tangent C [6][6] at (p, q, w, E, a) with z^n fixed, and their
 * derivatives along (dp, dq, dw, dE, da).  R, dR: [3 * active laminates];
 * z_n: [2^K][7] per leaf.  Returns 0, -1 for invalid arguments, -2 if J is not
 * positive definite. */
int oracle_eval_dual(int K, int M, const double* p, const double* q, const double* w, const double* mat,
                     const double* dp, const double* dq, const double* dw, double lam1, double lam2,
                     const double* E, const double* dE, const double* a, const double* da, const double* z_n,
                     int want_tangent, double* R, double* dR, double* sbar, double* dsbar, double* C, double* dC) {
  or_tree t;
  if (tree_init(&t, K, M, p, q, w, mat, 1e-12, 1, 0) != 0) return -1;
  or_work* ws = work_alloc(&t);
  or_dual* u = (or_dual*)calloc(1, sizeof(or_dual));
  int rc = 0;
  const double (*zl)[7] = (const double (*)[7])z_n;
  if (want_tangent && factor_at(&t, ws, lam1, lam2, E, a, zl) != 0) rc = -2;
  if (rc == 0) {
    eval_dual(&t, u, w, dp, dq, dw, lam1, lam2, E, dE, a, da, zl, want_tangent ? ws : NULL);
    for (int r = 0; r < 3 * t.nact; ++r) { R[r] = u->R[r].v; dR[r] = u->R[r].d; }
    for (int I = 0; I < 6; ++I) { sbar[I] = u->sbar[I].v; dsbar[I] = u->sbar[I].d; }
    if (want_tangent)
      for (int I = 0; I < 6; ++I)
        for (int J = 0; J < 6; ++J) { C[6 * I + J] = u->C[I][J].v; dC[6 * I + J] = u->C[I][J].d; }
  }
  free(u);
  work_free(ws);
  tree_free(&t);
  return rc;
}

/* Gradient of L = g . sigma_bar + G : C (local frame; G may be NULL) at the
 * converged jumps a of one point, by the implicit function theorem applied to
 * R(a, theta) = 0 (Sec. 3.2): with J = dR/da = A^T W D A,
 *   J lam = (d sigma_bar/da)^T g + (dC/da)^T : G,
 *   dL/dtheta = g . d sigma_bar/dtheta + G : dC/dtheta - lam . dR/dtheta,
 * every partial derivative at fixed a from eval_dual (exact), the solve with
 * the Cholesky factor of J in the paper's leaf-to-root order.  theta runs
 * over p, q [N][M] (paper ordering), the leaf weights w [L] as given (leaves of
 * weight zero get 0: the Macaulay bracket of Sec. 3.1 passes no change below
 * zero) and the local macro strain E [6].  Returns 0, -1 for invalid
 * arguments, -2 if J is not positive definite. */
int oracle_gradient(int K, int M, const double* p, const double* q, const double* w, const double* mat,
                    double lam1, double lam2, const double* E, const double* a, const double* z_n, const double* g,
                    const double* Gt, double* gp, double* gq, double* gw, double* gE) {
  or_tree t;
  if (tree_init(&t, K, M, p, q, w, mat, 1e-12, 1, 0) != 0) return -1;
  int L = t.L, NM = t.N * t.M, n = 3 * t.nact;
  or_work* ws = work_alloc(&t);
  or_dual* u = (or_dual*)calloc(1, sizeof(or_dual));
  double* zp = (double*)calloc((size_t)NM, sizeof(double));
  double* zq = (double*)calloc((size_t)NM, sizeof(double));
  double* zw = (double*)calloc((size_t)L, sizeof(double));
  double* za = (double*)calloc((size_t)n > 0 ? n : 1, sizeof(double));
  double* lam = (double*)calloc((size_t)n > 0 ? n : 1, sizeof(double));
  double zE[6] = {0, 0, 0, 0, 0, 0};
  const double (*zl)[7] = (const double (*)[7])z_n;
  int rc = factor_at(&t, ws, lam1, lam2, E, a, zl) != 0 ? -2 : 0;
  or_work* fac = Gt ? ws : NULL;
  if (rc == 0) {
    for (int k = 0; k < n; ++k) {   /* right-hand side of the adjoint system, one jump at a time */
      za[k] = 1.0;
      eval_dual(&t, u, w, zp, zq, zw, lam1, lam2, E, zE, a, za, zl, fac);
      lam[k] = seed_value(u, g, Gt);
      za[k] = 0.0;
    }
    chol_solve(&t, ws, lam);
    for (int x = 0; x < 2 * NM + L + 6; ++x) {
      double* dp = zp; double* dq = zq; double* dw = zw; double dE[6] = {0, 0, 0, 0, 0, 0};
      if (x < NM) dp[x] = 1.0;
      else if (x < 2 * NM) dq[x - NM] = 1.0;
      else if (x < 2 * NM + L) { if (!(w[x - 2 * NM] > 0.0)) { gw[x - 2 * NM] = 0.0; continue; } dw[x - 2 * NM] = 1.0; }
      else dE[x - 2 * NM - L] = 1.0;
      eval_dual(&t, u, w, dp, dq, dw, lam1, lam2, E, dE, a, za, zl, fac);
      double v = seed_value(u, g, Gt);
      for (int r = 0; r < n; ++r) v -= lam[r] * u->R[r].d;
      if (x < NM) { gp[x] = v; dp[x] = 0.0; }
      else if (x < 2 * NM) { gq[x - NM] = v; dq[x - NM] = 0.0; }
      else if (x < 2 * NM + L) { gw[x - 2 * NM] = v; dw[x - 2 * NM] = 0.0; }
      else gE[x - 2 * NM - L] = v;
    }
  }
  free(zp); free(zq); free(zw); free(za); free(lam);
  free(u);
  work_free(ws);
  tree_free(&t);
  return rc;
}

/* ------------------------------------------------------------------ */
/* Eq. (eigen decomposition of A): cyclic Jacobi rotations on the symmetric
 * 3x3 matrix, eigenvalues sorted descending; each of the first two
 * eigenvectors is signed so that its entry of largest magnitude is positive,
 * the third is their cross product (det Q = +1).  Q row-major, eigenvectors
 * as columns.  A2 given as (11, 22, 33, 23, 13, 12).                      */
static void jacobi_eig(const double a6[6], double lam[3], double V[3][3]) {
  double A[3][3] = {{a6[0], a6[5], a6[4]}, {a6[5], a6[1], a6[3]}, {a6[4], a6[3], a6[2]}};
  for (int i = 0; i < 3; ++i) for (int j = 0; j < 3; ++j) V[i][j] = (i == j) ? 1.0 : 0.0;
  for (int sweep = 0; sweep < 60; ++sweep) {
    double off = fabs(A[0][1]) + fabs(A[0][2]) + fabs(A[1][2]);
    if (off == 0.0) break;
    for (int p = 0; p < 2; ++p)
      for (int q = p + 1; q < 3; ++q) {
        if (A[p][q] == 0.0) continue;
        double theta = (A[q][q] - A[p][p]) / (2.0 * A[p][q]);
        double tt = (theta >= 0.0 ? 1.0 : -1.0) / (fabs(theta) + sqrt(theta * theta + 1.0));
        double c = 1.0 / sqrt(tt * tt + 1.0), s = tt * c;
        for (int k = 0; k < 3; ++k) {        /* A <- A J */
          double akp = A[k][p], akq = A[k][q];
          A[k][p] = c * akp - s * akq; A[k][q] = s * akp + c * akq;
        }
        for (int k = 0; k < 3; ++k) {        /* A <- J^T A */
          double apk = A[p][k], aqk = A[q][k];
          A[p][k] = c * apk - s * aqk; A[q][k] = s * apk + c * aqk;
        }
        for (int k = 0; k < 3; ++k) {        /* V <- V J */
          double vkp = V[k][p], vkq = V[k][q];
          V[k][p] = c * vkp - s * vkq; V[k][q] = s * vkp + c * vkq;
        }
      }
  }
  for (int i = 0; i < 3; ++i) lam[i] = A[i][i];
  /* sort descending (selection) */
  for (int i = 0; i < 2; ++i) {
    int m = i;
    for (int j = i + 1; j < 3; ++j) if (lam[j] > lam[m]) m = j;
    if (m != i) {
      double tl = lam[i]; lam[i] = lam[m]; lam[m] = tl;
      for (int k = 0; k < 3; ++k) { double tv = V[k][i]; V[k][i] = V[k][m]; V[k][m] = tv; }
    }
  }
  for (int c = 0; c < 2; ++c) {
    int m = 0;
    for (int k = 1; k < 3; ++k) if (fabs(V[k][c]) > fabs(V[m][c])) m = k;
    if (V[m][c] < 0.0) for (int k = 0; k < 3; ++k) V[k][c] = -V[k][c];
  }
  V[0][2] = V[1][0] * V[2][1] - V[2][0] * V[1][1];
  V[1][2] = V[2][0] * V[0][1] - V[0][0] * V[2][1];
  V[2][2] = V[0][0] * V[1][1] - V[1][0] * V[0][1];
}

int oracle_interp_orientation(long n, const double* A2, double* lam, double* Q) {
  for (long i = 0; i < n; ++i) {
    double l3[3], V[3][3];
    jacobi_eig(A2 + 6 * i, l3, V);
    lam[2 * i] = l3[0]; lam[2 * i + 1] = l3[1];
    for (int r = 0; r < 3; ++r) for (int c = 0; c < 3; ++c) Q[9 * i + 3 * r + c] = V[r][c];
  }
  return 0;
}
