// Kernels and C ABI of the batched DMN material-point update (include/dmn.h).
//
// Per update three kernels run on the caller's stream:
//   k_prepare  one thread per point: lamination normals of every laminate from
//              the orientation (barycentric coordinates, shape functions,
//              interpolated angles, spherical normal; Sec. 2.3) and the macro
//              strain in the principal frame;
//   k_newton   persistent, one thread per point slot: the Newton loop of
//              Sec. 3.2.  A lane that converges writes its results and takes
//              the next point from a global counter at once, so lanes stay busy
//              although points need different numbers of Newton steps;
//   k_final    one thread per point: the return mapping at the converged jumps
//              writes z^{n+1}, and stress and tangent are rotated back to the
//              global frame; in the mixed form this kernel first runs the FP64
//              sweep that yields them (the form with an FP32 tangent skips it
//              and rotates what the last Newton pass condensed).
#include <cuda_runtime.h>

#include <algorithm>
#include <array>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/dmn.h"
#include "dmn_device.cuh"
#include "dmn_launch.cuh"

using namespace dmn;

namespace {

thread_local std::string g_create_error;

}  // namespace

// the message dmn_last_error(NULL) returns, also set by the peak measurement (peak.cu)
void dmn_set_create_error(const std::string& msg) { g_create_error = msg; }

namespace {

struct Tree {
  int K, M, N, L, nz, z_both, S;
  double* d_p = nullptr;
  double* d_q = nullptr;
  double* d_c = nullptr;   // c1 [N], c2 [N], sc [N], normalised leaf weights [L], 1 / (c1 c2) [N]
  float* d_cf = nullptr;   // c1f [N], c2f [N], c12f [N], scf [N], 1 / (c1 c2) [N]
  double wsum = 1.0;       // sum of the leaf weights as given
  PhaseDev ph[2];
  // compressed trees (some leaf weight zero): N laminates left, Lc leaves left,
  // traversal tables lf [Lc] (int4), pre [N], post [N], paper index [N] in one allocation
  int cmp = 0, Lc = 0;
  int* d_tab = nullptr;
  std::vector<char> alive;  // compressed trees: which leaf weights are positive
};

}  // namespace

// Work space of one update in flight: the per-lane scratch of the persistent
// Newton kernel, its counters and the per-point buffers.  Updates that may run at
// the same time (the two stages of dmn_update_host) use separate work sets.
struct WorkSet {
  double* scr_d = nullptr;      // per slot: normals [3N] + jumps [3N] (FP64)
  void* scr_t = nullptr;        // per slot: g, H [21N] (FP64 or FP32) + FP32 normals [3N]
  unsigned long long* counter = nullptr;  // [0] work counter, [1..9] points per tree, [10..18] cursors
  float* scr_s = nullptr;       // the mixed forms' first stage, per slot of its kernel: g, H [21N], normals [3N],
                                // jumps [3N] (FP32)
  int64_t nslots_s = 0;         // slots of the first stage's kernel
  double* scr_w = nullptr;      // small calls, the warp organisation: a block of scratch per group of lanes
  int64_t nwarps_w = 0;
  double* nbuf = nullptr;       // per point: normals [3N] + local macro strain [6], field-major
  int64_t* perm = nullptr;      // points sorted by tree (several trees)
  int64_t nbuf_cap = 0;
};

// Device buffers, streams and events of dmn_update_host: two stages, each with
// room for one chunk of points.
struct HostPipe {
  int64_t cap = 0;              // points per stage
  char* buf[2] = {nullptr, nullptr};
  cudaStream_t up = nullptr, down = nullptr, comp[2] = {nullptr, nullptr};
  cudaEvent_t start = nullptr, h2d[2] = {nullptr, nullptr}, done[2] = {nullptr, nullptr},
              d2h[2] = {nullptr, nullptr};
};

struct dmn_handle {
  std::vector<Tree> trees;
  int N_max = 0;                // laminates of the deepest tree
  int64_t S_max = 0;            // state fields of the largest tree
  dmn_options opt;
  int device = 0, n_sm = 0;
  int64_t nslots = 0;
  bool cmp = false;             // trees walked by tables (some tree has weightless leaves)
  WorkSet ws[2];                // [0]: dmn_update; [1]: second stage of dmn_update_host
  HostPipe hp;
  double* gwork = nullptr;      // dmn_grad per-point work, one chunk
  int64_t gwork_cap = 0;
  bool profiling = false;
  std::vector<std::array<cudaEvent_t, 5>> events;  // per timed update: before/after each kernel
  unsigned long long* d_passes = nullptr;          // profiling: tree passes of the first stage and of k_newton
  size_t events_used = 0;
  std::string err;
};

namespace {

int fail(dmn_handle* h, int code, const std::string& msg) {
  if (h) h->err = msg; else g_create_error = msg;
  return code;
}

int cuda_fail(dmn_handle* h, cudaError_t e, const char* what) {
  return fail(h, DMN_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

TreeDev tree_dev(const Tree& t) {
  TreeDev d{};
  d.K = t.K; d.M = t.M; d.N = t.N; d.L = t.L; d.nz = t.nz; d.z_both = t.z_both;
  d.p = t.d_p; d.q = t.d_q;
  d.c1 = t.d_c; d.c2 = t.d_c + t.N; d.sc = t.d_c + 2 * t.N;
  d.c1f = t.d_cf; d.c2f = t.d_cf + t.N; d.c12f = t.d_cf + 2 * t.N; d.scf = t.d_cf + 3 * t.N;
  d.wl = t.d_c + 3 * t.N; d.wsum = t.wsum;
  d.ic12 = t.d_c + 3 * t.N + t.L; d.ic12f = t.d_cf + 4 * t.N;
  d.ph[0] = t.ph[0]; d.ph[1] = t.ph[1];
  d.Lc = t.Lc;
  d.lf = reinterpret_cast<const int4*>(t.d_tab);
  d.pre = t.d_tab ? t.d_tab + 4 * t.Lc : nullptr;
  d.post = t.d_tab ? t.d_tab + 4 * t.Lc + t.N : nullptr;
  d.pidx = t.d_tab ? t.d_tab + 4 * t.Lc + 2 * t.N : nullptr;
  d.kid = t.d_tab ? t.d_tab + 4 * t.Lc + 3 * t.N : nullptr;
  d.hcid = t.d_tab ? t.d_tab + 4 * t.Lc + 5 * t.N : nullptr;
  d.kslot = t.d_tab ? t.d_tab + 4 * t.Lc + 5 * t.N + ((1 << t.K) - 1) : nullptr;
  return d;
}

// The FP32 copies of a phase's constants (the mixed forms' all-FP32 first stage).
void phase_f32(PhaseDev& o) {
  o.f.K = (float)o.K; o.f.G = (float)o.G; o.f.s0 = (float)o.s0; o.f.H = (float)o.H; o.f.lam = (float)o.lam;
  o.f.inv_den = (float)o.inv_den; o.f.thb0 = (float)o.thb0;
  o.f.ds = (float)o.ds; o.f.dk = (float)o.dk; o.f.rate = (float)o.rate;
}

// Checks one phase of a tree description and derives its device constants.
const char* make_phase(const dmn_phase& p, PhaseDev& out) {
  if (p.kind != DMN_PHASE_ELASTIC && p.kind != DMN_PHASE_J2_LINEAR && p.kind != DMN_PHASE_J2_EXPLIN)
    return "unknown phase kind";
  if (!(p.E > 0.0) || !(p.nu > -1.0) || !(p.nu < 0.5)) return "need E > 0 and -1 < nu < 0.5";
  if (p.kind != DMN_PHASE_ELASTIC && (!(p.sigma0 > 0.0) || !(p.H >= 0.0) || !std::isfinite(p.H)))
    return "J2 phase needs sigma0 > 0 and H >= 0";
  if (p.kind == DMN_PHASE_J2_EXPLIN && (!(p.sigma_inf >= p.sigma0) || !(p.k0 >= p.H) || !std::isfinite(p.k0) ||
                                        !std::isfinite(p.sigma_inf)))
    return "exponential-linear hardening needs sigma_inf >= sigma0 and k0 >= H";
  out.kind = p.kind;
  out.ds = out.dk = out.rate = 0.0;
  if (p.kind == DMN_PHASE_J2_EXPLIN) {
    if (p.sigma_inf > p.sigma0 && p.k0 > p.H) {
      out.ds = p.sigma_inf - p.sigma0;
      out.dk = p.k0 - p.H;
      out.rate = out.dk / out.ds;
    } else {
      out.kind = DMN_PHASE_J2_LINEAR;   // no exponential term: the linear law
    }
  }
  out.K = p.E / (3.0 * (1.0 - 2.0 * p.nu));
  out.G = p.E / (2.0 * (1.0 + p.nu));
  out.s0 = p.sigma0;
  out.H = p.H;
  out.lam = out.K - 2.0 * out.G / 3.0;
  out.lamf = (float)out.lam;
  out.Gf = (float)out.G;
  out.inv_den = 1.0 / (2.0 * out.G + 2.0 * p.H / 3.0);
  out.thb0 = 1.0 / (1.0 + p.H / (3.0 * out.G));
  phase_f32(out);
  return nullptr;
}

// ---------------------------------------------------------------------------
// Weights (Sec. 2.1): w normalised to sum 1; w^i_k = w^{2i-1}_{k+1} + w^{2i}_{k+1};
// c1 = w_left / (w_left + w_right), c2 = 1 - c1; sc = W c1 c2 scales the
// laminate's residual.  Heap order.  One thread.
__global__ void k_setup_tree(int K, const double* w_raw, double* c, float* cf) {
  if (blockIdx.x != 0 || threadIdx.x != 0) return;
  const int L = 1 << K, N = L - 1;
  double W[NMAX];
  double s = 0.0;
  for (int l = 0; l < L; ++l) s += w_raw[l];
  for (int h = N; h >= 1; --h) {
    double wl, wr;
    if (h >= (1 << (K - 1))) {
      const int m = h - (1 << (K - 1));
      wl = w_raw[2 * m] / s;
      wr = w_raw[2 * m + 1] / s;
    } else {
      wl = W[2 * h - 1];
      wr = W[2 * h];
    }
    W[h - 1] = wl + wr;
    const double c1 = wl / (wl + wr), c2 = 1.0 - c1;
    c[h - 1] = c1;
    c[N + h - 1] = c2;
    c[2 * N + h - 1] = W[h - 1] * c1 * c2;
    cf[h - 1] = (float)c1;
    cf[N + h - 1] = (float)c2;
    cf[2 * N + h - 1] = (float)(c1 * c2);
    cf[3 * N + h - 1] = (float)(W[h - 1] * c1 * c2);
    c[3 * N + L + h - 1] = 1.0 / (c1 * c2);
    cf[4 * N + h - 1] = (float)(1.0 / (c1 * c2));
  }
  for (int l = 0; l < L; ++l) c[3 * N + l] = w_raw[l] / s;
}

// ---------------------------------------------------------------------------
// Orientation set-up: cyclic Jacobi rotations on the symmetric 3x3 A2,
// eigenvalues sorted descending, eigenvector signs normalised (see dmn.h).
__global__ void k_interp(int64_t n, const double* __restrict__ A2, double* __restrict__ lam, double* __restrict__ Q) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double* a = A2 + 6 * i;
  double S[3][3] = {{a[0], a[5], a[4]}, {a[5], a[1], a[3]}, {a[4], a[3], a[2]}};
  double V[3][3] = {{1, 0, 0}, {0, 1, 0}, {0, 0, 1}};
  for (int sweep = 0; sweep < 32; ++sweep) {
    const double off = fabs(S[0][1]) + fabs(S[0][2]) + fabs(S[1][2]);
    const double dia = fabs(S[0][0]) + fabs(S[1][1]) + fabs(S[2][2]);
    if (off <= 1e-30 * dia) break;
#pragma unroll
    for (int pr = 0; pr < 3; ++pr) {
      const int p = pr == 2 ? 1 : 0, q = pr == 0 ? 1 : 2;
      const double apq = S[p][q];
      if (apq == 0.0) continue;
      // rotation angle that annihilates S[p][q]: t = tan(phi), |phi| <= pi/4
      const double tau = (S[q][q] - S[p][p]) / (2.0 * apq);
      const double t = copysign(1.0, tau) / (fabs(tau) + sqrt(1.0 + tau * tau));
      const double c = rsqrt(1.0 + t * t), s = t * c;
      for (int k = 0; k < 3; ++k) {
        const double skp = S[k][p], skq = S[k][q];
        S[k][p] = c * skp - s * skq;
        S[k][q] = s * skp + c * skq;
      }
      for (int k = 0; k < 3; ++k) {
        const double spk = S[p][k], sqk = S[q][k];
        S[p][k] = c * spk - s * sqk;
        S[q][k] = s * spk + c * sqk;
      }
      for (int k = 0; k < 3; ++k) {
        const double vkp = V[k][p], vkq = V[k][q];
        V[k][p] = c * vkp - s * vkq;
        V[k][q] = s * vkp + c * vkq;
      }
    }
  }
  double l[3] = {S[0][0], S[1][1], S[2][2]};
  int o[3] = {0, 1, 2};
  // order indices by descending eigenvalue
  if (l[o[1]] > l[o[0]]) { int x = o[0]; o[0] = o[1]; o[1] = x; }
  if (l[o[2]] > l[o[1]]) { int x = o[1]; o[1] = o[2]; o[2] = x; }
  if (l[o[1]] > l[o[0]]) { int x = o[0]; o[0] = o[1]; o[1] = x; }
  double v[2][3];
  for (int c = 0; c < 2; ++c) {
    int m = 0;
    for (int k = 1; k < 3; ++k)
      if (fabs(V[k][o[c]]) > fabs(V[m][o[c]])) m = k;
    const double sg = V[m][o[c]] < 0.0 ? -1.0 : 1.0;
    for (int k = 0; k < 3; ++k) v[c][k] = sg * V[k][o[c]];
  }
  const double w3[3] = {v[0][1] * v[1][2] - v[0][2] * v[1][1], v[0][2] * v[1][0] - v[0][0] * v[1][2],
                        v[0][0] * v[1][1] - v[0][1] * v[1][0]};
  lam[2 * i] = l[o[0]];
  lam[2 * i + 1] = l[o[1]];
  double* Qi = Q + 9 * i;
  for (int k = 0; k < 3; ++k) { Qi[3 * k + 0] = v[0][k]; Qi[3 * k + 1] = v[1][k]; Qi[3 * k + 2] = w3[k]; }
}

// ---------------------------------------------------------------------------
// Normals of every laminate of one point (Sec. 2.3): phi = barycentric
// coordinates of (lam1, lam2) in the triangle UD (1,0), ISO (1/3,1/3),
// PI (1/2,1/2), i.e. phi = (lam1 - lam2, 3 lam3, 2 lam1 + 4 lam2 - 2); shape
// functions of order M; alpha = p.phi, beta = q.phi;
// n = (sin a cos b, sin a sin b, cos a).  Written to strided storage.
// normals of the laminates first, first + step, ... (all of them by default)
__device__ void point_normals(const TreeDev& t, double l1, double l2, double* out, size_t stride, int first = 0,
                              int step = 1) {
  const double v[3] = {l1 - l2, 3.0 * (1.0 - l1 - l2), 2.0 * l1 + 4.0 * l2 - 2.0};
  double ph[6];
  if (t.M == 3) {
    ph[0] = v[0]; ph[1] = v[1]; ph[2] = v[2];
  } else if (t.M == 4) {
    const double b = v[0] * v[1] * v[2];
    ph[0] = v[0] - 9.0 * b; ph[1] = v[1] - 9.0 * b; ph[2] = v[2] - 9.0 * b; ph[3] = 27.0 * b;
  } else {
    ph[0] = v[0] * (2.0 * v[0] - 1.0); ph[1] = v[1] * (2.0 * v[1] - 1.0); ph[2] = v[2] * (2.0 * v[2] - 1.0);
    ph[3] = 4.0 * v[0] * v[1]; ph[4] = 4.0 * v[0] * v[2]; ph[5] = 4.0 * v[1] * v[2];
  }
  for (int j = first; j < t.N; j += step) {
    double al = 0.0, be = 0.0;
    for (int m = 0; m < t.M; ++m) {
      al += __ldg(t.p + j * t.M + m) * ph[m];
      be += __ldg(t.q + j * t.M + m) * ph[m];
    }
    double sa, ca, sb, cb;
    sincos(al, &sa, &ca);
    sincos(be, &sb, &cb);
    out[(size_t)(3 * j + 0) * stride] = sa * cb;
    out[(size_t)(3 * j + 1) * stride] = sa * sb;
    out[(size_t)(3 * j + 2) * stride] = ca;
  }
}

__device__ __forceinline__ void local_strain(const double* Q, const double* En, const double* dE, double Eloc[6]) {
  double R[6][6], Eg[6];
  mandel_rotation(Q, R);
#pragma unroll
  for (int I = 0; I < 6; ++I) Eg[I] = En[I] + dE[I];
#pragma unroll
  for (int J = 0; J < 6; ++J) {
    double s = 0.0;
#pragma unroll
    for (int I = 0; I < 6; ++I) s += R[I][J] * Eg[I];
    Eloc[J] = s;
  }
}

// Sorting points by tree (several trees): count per tree, exclusive offsets,
// scatter.  Lanes of a warp with the same tree share one atomic.  The order
// inside a tree is not deterministic; results do not depend on it.
__global__ void k_tree_count(int64_t n, const int32_t* __restrict__ tid, int n_trees, unsigned long long* cnt) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  int b = -1;
  if (i < n) {
    const int t = tid[i];
    b = (t >= 0 && t < n_trees) ? t : n_trees;
  }
  const unsigned peers = __match_any_sync(0xffffffffu, b);
  if (b >= 0 && (threadIdx.x & 31) == __ffs(peers) - 1) atomicAdd(cnt + b, (unsigned long long)__popc(peers));
}

__global__ void k_tree_offsets(int n_trees, const unsigned long long* cnt, unsigned long long* cursor) {
  if (blockIdx.x != 0 || threadIdx.x != 0) return;
  unsigned long long s = 0;
  for (int b = 0; b <= n_trees; ++b) { cursor[b] = s; s += cnt[b]; }
}

__global__ void k_tree_scatter(int64_t n, const int32_t* __restrict__ tid, int n_trees, unsigned long long* cursor,
                               int64_t* __restrict__ perm) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int lane = threadIdx.x & 31;
  int b = -1;
  if (i < n) {
    const int t = tid[i];
    b = (t >= 0 && t < n_trees) ? t : n_trees;
  }
  const unsigned peers = __match_any_sync(0xffffffffu, b);
  const int leader = __ffs(peers) - 1;
  unsigned long long base = 0;
  if (b >= 0 && lane == leader) base = atomicAdd(cursor + b, (unsigned long long)__popc(peers));
  base = __shfl_sync(peers, base, leader);
  if (b >= 0) perm[base + __popc(peers & ((1u << lane) - 1u))] = i;
}

// per point: normals and the macro strain in the principal frame
__global__ void k_prepare(Forest F, int64_t n, const int32_t* __restrict__ tid, const int64_t* __restrict__ perm,
                          const double* __restrict__ lam, const double* __restrict__ Q, const double* __restrict__ En,
                          const double* __restrict__ dE, double* __restrict__ nbuf, int N_max) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  int64_t p;
  int tr;
  point_of(perm, tid, F.n, i, p, tr);
  if (tr >= F.n) return;
  point_normals(F.t[tr], lam[2 * p], lam[2 * p + 1], nbuf + p, (size_t)n);
  double E[6];
  local_strain(Q + 9 * p, En + 6 * p, dE + 6 * p, E);
#pragma unroll
  for (int I = 0; I < 6; ++I) nbuf[(size_t)(3 * N_max + I) * n + p] = E[I];
}

template <typename T>
__device__ __forceinline__ void write_stress_tangent(const double* Q, const double sb[6], const T C[21], double* stress,
                                                     double* tangent) {
  double R[6][6];
  mandel_rotation(Q, R);
  double Cl[21];
#pragma unroll
  for (int k = 0; k < 21; ++k) Cl[k] = (double)C[k];
#pragma unroll
  for (int I = 0; I < 6; ++I) {
    double s = 0.0;
#pragma unroll
    for (int J = 0; J < 6; ++J) s += R[I][J] * sb[J];
    stress[I] = s;
  }
  double RC[6][6];
#pragma unroll
  for (int I = 0; I < 6; ++I)
#pragma unroll
    for (int J = 0; J < 6; ++J) {
      double s = 0.0;
#pragma unroll
      for (int P = 0; P < 6; ++P) s += R[I][P] * Cl[sidx(P, J)];
      RC[I][J] = s;
    }
#pragma unroll
  for (int I = 0; I < 6; ++I)
#pragma unroll
    for (int J = 0; J < 6; ++J) {
      double s = 0.0;
#pragma unroll
      for (int P = 0; P < 6; ++P) s += RC[I][P] * R[J][P];
      tangent[6 * I + J] = s;
    }
}

// MINB: resident CTAs per SM the register allocation is sized for (255, 170 or
// 128 registers per thread at 2, 3 or 4 CTAs of 128 threads).
// LS: backtracking line search (Sec. 3.2 allows a step s in (0, 1]): a trial
// step is accepted when it lowers the residual norm, else it is halved, at
// most 8 times.  Jumps and g, H are then kept in two buffers per lane: a pass
// reads the accepted ones and writes the trial's, so a rejected trial leaves
// the accepted iterate intact.
// CMP: trees walked by their compressed-traversal tables (tree_pass_c), jumps
// numbered as in the state; otherwise heap arithmetic (tree_pass).
// Extrapolated start: corrections allowed before a point restarts from a^n.
constexpr int PRED_TRIES = 6;

// PRED: extrapolated start (a separate instantiation, so that the paper's start pays nothing for it).
template <typename T, int MINB, bool LS, bool CMP, bool PRED>
__global__ void __launch_bounds__(128, MINB) k_newton(NewtonParams<T> P) {
  const int64_t slot = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int lane = threadIdx.x & 31;
  const int NM = P.N_max;
  const size_t ns = (size_t)P.nslots;
  double* my_nrm = P.scr_d + slot;
  float* my_nrmf = (float*)(P.scr_t + (size_t)((LS ? 42 : 21) * NM) * ns) + slot;
  double* abuf[2] = {P.scr_d + (size_t)(3 * NM) * ns + slot, P.scr_d + (size_t)((LS ? 6 : 3) * NM) * ns + slot};
  T* gbuf[2] = {P.scr_t + slot, P.scr_t + (size_t)((LS ? 21 : 0) * NM) * ns + slot};
  PointArrays A{};
  A.nrm = my_nrm; A.ns = ns;
  A.nrmf = my_nrmf;
  A.as = ns;
  A.paper = false;
  A.z = nullptr; A.zs = (size_t)P.n;
  const double qnan = __longlong_as_double(0x7ff8000000000000LL);
  int64_t pt = -1;   // point of this lane; -1: needs work; >= n: no work left
  int tr = 0;        // its tree
  int it = 0;
  int it0 = 0;       // corrections of the first stage (they count against max_iter)
  int cur = 0;       // buffer holding the accepted jumps and g, H
  bool first = true; // the next pass evaluates the starting jumps
  T step = (T)1;     // line search: scale of the trial step
  int halvings = 0;
  bool retry = false; // extrapolated start: restart from a^n if it has not converged by lim
  int lim = 0;        // corrections after which the current attempt ends with MAXITER
  double rn_acc = 0.0;
  Sub<T> root_acc;   // line search: results at the accepted iterate
  double Eloc[6];
  unsigned long long npass = 0;
  // the extrapolated start failed: continue from the stored jumps a^n, as a new point would
  auto restart = [&](const TreeDev& t) {
    const int nzf = 6 * t.nz;
    for (int f = 0; f < 3 * t.N; ++f) {
      const int node = f / 3, c = f - 3 * node;
      const int lvl = 32 - __clz(node + 1);
      const int j = CMP ? node : (1 << t.K) - 3 * (1 << (lvl - 1)) + node + 1;
      abuf[cur][(size_t)f * ns] = P.state_in[(size_t)(nzf + 3 * j + c) * P.n + pt];
    }
    retry = false;
    lim = it + P.max_iter;
    first = true;
    step = (T)1;
    halvings = 0;
  };
  for (;;) {
    const bool need = pt < 0;
    const unsigned mask = __ballot_sync(0xffffffffu, need);
    if (mask) {
      const int leader = __ffs(mask) - 1;
      unsigned long long base = 0;
      if (lane == leader) base = atomicAdd(P.counter, (unsigned long long)__popc(mask));
      base = __shfl_sync(0xffffffffu, base, leader);
      if (need) {
        const int64_t i = (int64_t)(base + __popc(mask & ((1u << lane) - 1u)));
        if (i >= P.n) {
          pt = P.n;
        } else {
          point_of(P.perm, P.tid, P.F.n, i, pt, tr);
          if (tr >= P.F.n) {      // unknown tree: report and take the next point
            P.iters[pt] = 0;
            P.status[pt] = DMN_STATUS_BAD_TREE;
            for (int I = 0; I < 6; ++I) P.stress[6 * pt + I] = qnan;
            for (int I = 0; I < 36; ++I) P.tangent[36 * pt + I] = qnan;
            pt = -1;
          } else {
            const TreeDev& t = P.F.t[tr];
            const int nzf = 6 * t.nz;
            cur = 0;
#pragma unroll
            for (int I = 0; I < 6; ++I) Eloc[I] = P.nbuf[(size_t)(3 * NM + I) * P.n + pt];
            // extrapolated start: rho = (dE . dE_prev) / (dE_prev . dE_prev), clamped to [-2, 2]
            const int pf0 = nzf + 3 * t.N;   // first field of the last jump change
            double rho = 0.0;
            if (PRED) {
              double num = 0.0, den = 0.0;
#pragma unroll
              for (int c = 0; c < 6; ++c) {
                const double q = P.state_in[(size_t)(pf0 + 3 * t.N + c) * P.n + pt];
                num += P.dE[6 * pt + c] * q;
                den += q * q;
              }
              const double r = num / den;
              rho = (den > 0.0 && isfinite(r)) ? fmin(fmax(r, 0.0), 1.0) : 0.0;
            }
            if (PRED) {
              retry = rho > 0.0;
              lim = retry ? PRED_TRIES : P.max_iter;
            }
            for (int f = 0; f < 3 * t.N; ++f) {
              const int node = f / 3, c = f - 3 * node;
              // heap node -> paper index of its jumps
              const int lvl = 32 - __clz(node + 1);
              const int j = CMP ? node : (1 << t.K) - 3 * (1 << (lvl - 1)) + node + 1;
              double a0 = (P.a_start ? P.a_start : P.state_in)[(size_t)(nzf + 3 * j + c) * P.n + pt];
              if (PRED) a0 += rho * P.state_in[(size_t)(pf0 + 3 * j + c) * P.n + pt];
              abuf[0][(size_t)f * ns] = a0;
              const double nv = P.nbuf[(size_t)f * P.n + pt];
              my_nrm[(size_t)f * ns] = nv;
              if (sizeof(T) == 4) my_nrmf[(size_t)f * ns] = narrow_rn(nv);
            }
            A.z = P.state_in + pt;
            it = 0;
            it0 = P.a_start ? P.iters[pt] : 0;
            first = true;
            step = (T)1;
            halvings = 0;
          }
        }
      }
    }
    const bool active = pt >= 0 && pt < P.n;
    if (!__any_sync(0xffffffffu, active)) {
      if (!__any_sync(0xffffffffu, pt < 0)) break;
      continue;
    }
    if (!active) continue;
    const TreeDev& t = P.F.t[tr];
    ++npass;
    A.a = abuf[cur];
    A.a_out = abuf[LS ? 1 - cur : cur];
    GH<T> gh{gbuf[cur], ns, gbuf[LS ? 1 - cur : cur]};
    Sub<T> root;
    double r2;
    if (CMP) tree_pass_c<T, true>(t, Eloc, A, gh, !first, step, root, r2, nullptr);
    else tree_pass<T, true>(t, Eloc, A, gh, !first, step, root, r2, nullptr);
    const double rn = sqrt(r2);
    double sn2 = 0.0;
#pragma unroll
    for (int I = 0; I < 6; ++I) sn2 += root.sb[I] * root.sb[I];
    const double sn = sqrt(sn2);
    int st = -1;
    if (!LS) {
      first = false;
      if (!isfinite(rn) || !isfinite(sn)) st = DMN_STATUS_NONFINITE;
      else if (rn <= P.tol * (double)t.N * sn && it >= P.min_corr) st = DMN_STATUS_OK;
      else if (it >= (PRED ? lim : P.max_iter - it0)) st = DMN_STATUS_MAXITER;
      if (st < 0) { ++it; continue; }
    } else {
      bool accepted = first || rn < rn_acc;
      if (accepted) {
        first = false;
        cur = 1 - cur;
        rn_acc = rn;
        root_acc = root;
        step = (T)1;
        halvings = 0;
        if (!isfinite(rn) || !isfinite(sn)) st = DMN_STATUS_NONFINITE;
        else if (rn <= P.tol * (double)t.N * sn) st = DMN_STATUS_OK;
        else if (it >= (PRED ? lim : P.max_iter)) st = DMN_STATUS_MAXITER;
        if (st < 0) { ++it; continue; }
      } else if (++halvings > 8) {
        st = DMN_STATUS_LINESEARCH;   // no halving lowered the residual: keep the accepted iterate
        ++it;
        root = root_acc;
      } else {
        step *= (T)0.5;
        continue;
      }
    }
    if (PRED && st > 0 && retry) {   // the extrapolated start failed: the stored jumps a^n, as a new point
      restart(t);
      continue;
    }
    // finished point: jumps (paper ordering), counters, and without a final sweep
    // the local-frame stress and packed tangent for k_final to rotate
    const double* afin = abuf[cur];
    const int nzf = 6 * t.nz;
    for (int f = 0; f < 3 * t.N; ++f) {
      const int node = f / 3, c = f - 3 * node;
      const int lvl = 32 - __clz(node + 1);
      const int j = CMP ? node : (1 << t.K) - 3 * (1 << (lvl - 1)) + node + 1;
      const double af = st == DMN_STATUS_NONFINITE ? qnan : afin[(size_t)f * ns];
      P.state_out[(size_t)(nzf + 3 * j + c) * P.n + pt] = af;
      if (PRED)   // this update's jump change, for the next update's start
        P.state_out[(size_t)(nzf + 3 * t.N + 3 * j + c) * P.n + pt] = af - P.state_in[(size_t)(nzf + 3 * j + c) * P.n + pt];
    }
    if (PRED) {
#pragma unroll
      for (int c = 0; c < 6; ++c) P.state_out[(size_t)(nzf + 6 * t.N + c) * P.n + pt] = P.dE[6 * pt + c];
    }
    P.iters[pt] = it + it0;
    P.status[pt] = st;
    if (P.write_outputs) {
#pragma unroll
      for (int I = 0; I < 6; ++I) P.stress[6 * pt + I] = root.sb[I];
#pragma unroll
      for (int k = 0; k < 21; ++k) P.tangent[36 * pt + k] = widen(root.C[k]);
    }
    pt = -1;
  }
  if (P.passes && npass) atomicAdd(P.passes, npass);
}

// The mixed forms' first stage (Sec. 3.2's Newton iteration with every quantity in FP32: jumps,
// strains, leaf return mapping, residual and condensation).  Persistent like k_newton, with its own
// work counter and launch shape; per slot the FP32 scratch g, H [21 N], normals [3 N], jumps
// [3 N].  A point iterates until its FP32 residual meets ||A^T W sigma|| <= tol (2^K - 1)
// ||sigma_bar|| or max_iter corrections, then writes its jumps (widened) to the jump fields of
// state_out and the corrections to iters; k_newton continues from there with the FP64 residual.
// A point whose FP32 iterates are not finite hands on a^n and zero corrections.  Points of
// unknown trees are left to k_newton.
constexpr int STAGE_CTAS_DEFAULT = 4;   // resident CTAs of 128 threads per SM

struct StageParams {
  Forest F;
  int64_t n, nslots;
  int N_max;
  const int32_t* tid;
  const int64_t* perm;
  const double* state_in;
  double* state_out;
  int32_t* iters;
  const double* nbuf;
  float* scr;
  unsigned long long* counter;
  float tol;
  int max_iter;
  unsigned long long* passes;  // profiling: tree passes of all points added here, or NULL
};

template <int MINB, bool CMP>
__global__ void __launch_bounds__(128, MINB) k_stage32(StageParams P) {
  const int64_t slot = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int lane = threadIdx.x & 31;
  const int NM = P.N_max;
  const size_t ns = (size_t)P.nslots;
  float* gh = P.scr + slot;
  float* nrmf = P.scr + (size_t)(21 * NM) * ns + slot;
  float* af = P.scr + (size_t)(24 * NM) * ns + slot;
  PointArrays A{};
  A.ns = ns; A.nrmf = nrmf;
  A.as = ns; A.paper = false;
  A.af = af; A.af_out = af;
  A.zs = (size_t)P.n;
  int64_t pt = -1;
  int tr = 0, it = 0;
  bool first = true;
  float E32[6];
  unsigned long long npass = 0;
  for (;;) {
    const bool need = pt < 0;
    const unsigned mask = __ballot_sync(0xffffffffu, need);
    if (mask) {
      const int leader = __ffs(mask) - 1;
      unsigned long long base = 0;
      if (lane == leader) base = atomicAdd(P.counter, (unsigned long long)__popc(mask));
      base = __shfl_sync(0xffffffffu, base, leader);
      if (need) {
        const int64_t i = (int64_t)(base + __popc(mask & ((1u << lane) - 1u)));
        if (i >= P.n) {
          pt = P.n;
        } else {
          point_of(P.perm, P.tid, P.F.n, i, pt, tr);
          if (tr >= P.F.n) {
            pt = -1;
          } else {
            const TreeDev& t = P.F.t[tr];
            const int nzf = 6 * t.nz;
#pragma unroll
            for (int I = 0; I < 6; ++I) E32[I] = narrow_rn(P.nbuf[(size_t)(3 * NM + I) * P.n + pt]);
            for (int f = 0; f < 3 * t.N; ++f) {
              const int node = f / 3, c = f - 3 * node;
              const int lvl = 32 - __clz(node + 1);
              const int j = CMP ? node : (1 << t.K) - 3 * (1 << (lvl - 1)) + node + 1;
              af[(size_t)f * ns] = narrow_rn(P.state_in[(size_t)(nzf + 3 * j + c) * P.n + pt]);
              nrmf[(size_t)f * ns] = narrow_rn(P.nbuf[(size_t)f * P.n + pt]);
            }
            A.z = P.state_in + pt;
            it = 0;
            first = true;
          }
        }
      }
    }
    const bool active = pt >= 0 && pt < P.n;
    if (!__any_sync(0xffffffffu, active)) {
      if (!__any_sync(0xffffffffu, pt < 0)) break;
      continue;
    }
    if (!active) continue;
    const TreeDev& t = P.F.t[tr];
    ++npass;
    GH<float> g{gh, ns, gh};
    Sub<float, float> root;
    float r2;
    if (CMP) tree_pass_c<float, true, float>(t, E32, A, g, !first, 1.0f, root, r2, nullptr);
    else tree_pass<float, true, float>(t, E32, A, g, !first, 1.0f, root, r2, nullptr);
    first = false;
    float sn2 = 0.0f;
#pragma unroll
    for (int I = 0; I < 6; ++I) sn2 += root.sb[I] * root.sb[I];
    const float rn = sqrtf(r2), sn = sqrtf(sn2);
    const bool bad = !isfinite(rn) || !isfinite(sn);
    if (!bad && rn > P.tol * (float)t.N * sn && it < P.max_iter) {
      ++it;
      continue;
    }
    const int nzf = 6 * t.nz;
    for (int f = 0; f < 3 * t.N; ++f) {
      const int node = f / 3, c = f - 3 * node;
      const int lvl = 32 - __clz(node + 1);
      const int j = CMP ? node : (1 << t.K) - 3 * (1 << (lvl - 1)) + node + 1;
      const size_t at = (size_t)(nzf + 3 * j + c) * P.n + pt;
      P.state_out[at] = bad ? P.state_in[at] : widen(af[(size_t)f * ns]);
    }
    P.iters[pt] = bad ? 0 : it;
    pt = -1;
  }
  if (P.passes && npass) atomicAdd(P.passes, npass);
}

struct FinalParams {
  Forest F;
  int64_t n;
  int N_max;
  const int32_t* tid;
  const int64_t* perm;
  const double *Q, *state_in;
  double *state_out, *stress, *tangent;
  const int32_t* status;
  const double* nbuf;
};

template <bool SWEEP, bool CMP>
__global__ void __launch_bounds__(128) k_final(FinalParams P) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= P.n) return;
  int64_t pt;
  int tr;
  point_of(P.perm, P.tid, P.F.n, i, pt, tr);
  if (tr >= P.F.n) return;  // unknown tree: reported by the Newton kernel
  const TreeDev& t = P.F.t[tr];
  const int st = P.status[pt];
  double Eloc[6];
#pragma unroll
  for (int I = 0; I < 6; ++I) Eloc[I] = P.nbuf[(size_t)(3 * P.N_max + I) * P.n + pt];
  PointArrays A{};
  A.nrm = P.nbuf + pt; A.ns = (size_t)P.n;
  A.nrmf = nullptr;
  A.a = P.state_out + (size_t)(6 * t.nz) * P.n + pt; A.as = (size_t)P.n;
  A.a_out = A.a;
  A.paper = true;
  A.z = P.state_in + pt; A.zs = (size_t)P.n;
  if (st == DMN_STATUS_NONFINITE) {
    const double qnan = __longlong_as_double(0x7ff8000000000000LL);
    for (int I = 0; I < 6; ++I) P.stress[6 * pt + I] = qnan;
    for (int I = 0; I < 36; ++I) P.tangent[36 * pt + I] = qnan;
  } else if (SWEEP) {   // stress and tangent from one FP64 pass at the converged jumps
    Sub<double> root;
    double r2;
    GH<double> gh{nullptr, 0, nullptr};
    if (CMP) tree_pass_c<double, false>(t, Eloc, A, gh, false, 1.0, root, r2, nullptr);
    else tree_pass<double, false>(t, Eloc, A, gh, false, 1.0, root, r2, nullptr);
    write_stress_tangent<double>(P.Q + 9 * pt, root.sb, root.C, P.stress + 6 * pt, P.tangent + 36 * pt);
  } else {
    double sb[6], C[21];
#pragma unroll
    for (int I = 0; I < 6; ++I) sb[I] = P.stress[6 * pt + I];
#pragma unroll
    for (int k = 0; k < 21; ++k) C[k] = P.tangent[36 * pt + k];
    write_stress_tangent<double>(P.Q + 9 * pt, sb, C, P.stress + 6 * pt, P.tangent + 36 * pt);
  }
  if (CMP) write_leaf_states_c(t, Eloc, A, P.state_out + pt, (size_t)P.n, st == DMN_STATUS_NONFINITE);
  else write_leaf_states(t, Eloc, A, P.state_out + pt, (size_t)P.n, st == DMN_STATUS_NONFINITE);
}

// ---------------------------------------------------------------------------
// Adjoint kernels (dmn_grad).  One thread per point of a chunk; per-point work
// arrays are field-major over the chunk.
struct GradParams {
  TreeDev t;
  int64_t n, n0, nc;   // points in the batch, first point of the chunk, chunk size
  const double *lam, *Q, *En, *dE, *state_in, *state_out, *g_stress;
  double* g_E;
  double* work;
};

// work fields per point
__host__ __device__ inline size_t grad_fields(int N, int L) { return (size_t)33 * N + 2 * L + 6; }
// with tangent seeds: one more field block, every laminate's stiffness adjoint [21 N]
__host__ __device__ inline size_t grad_fields_tangent(int N, int L) { return grad_fields(N, L) + (size_t)21 * N; }

// CMP: the tree is walked by its compressed-traversal tables.
template <bool CMP>
__global__ void __launch_bounds__(128) k_grad(GradParams P) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= P.nc) return;
  const int64_t pt = P.n0 + i;
  const TreeDev& t = P.t;
  const int N = t.N, L = t.L;
  const size_t ws = (size_t)P.nc;
  double* w = P.work + i;
  double* nrm = w;
  double* a = w + (size_t)(3 * N) * ws;
  double* gh = w + (size_t)(6 * N) * ws;
  AdjWork Wk;
  Wk.H = gh; Wk.hs = ws;
  Wk.mu = w + (size_t)(27 * N) * ws;
  Wk.xi = w + (size_t)(30 * N) * ws;
  Wk.gab = w + (size_t)(31 * N) * ws;
  Wk.direct = w + (size_t)(33 * N) * ws;
  Wk.ws = ws;
  double* gw = w + (size_t)(33 * N + L) * ws;
  double* phv = w + (size_t)(33 * N + 2 * L) * ws;
  // orientation: normals and shape functions
  const double l1 = P.lam[2 * pt], l2 = P.lam[2 * pt + 1];
  point_normals(t, l1, l2, nrm, ws);
  const double v[3] = {l1 - l2, 3.0 * (1.0 - l1 - l2), 2.0 * l1 + 4.0 * l2 - 2.0};
  double ph[6] = {0, 0, 0, 0, 0, 0};
  if (t.M == 3) {
    ph[0] = v[0]; ph[1] = v[1]; ph[2] = v[2];
  } else if (t.M == 4) {
    const double b = v[0] * v[1] * v[2];
    ph[0] = v[0] - 9.0 * b; ph[1] = v[1] - 9.0 * b; ph[2] = v[2] - 9.0 * b; ph[3] = 27.0 * b;
  } else {
    ph[0] = v[0] * (2.0 * v[0] - 1.0); ph[1] = v[1] * (2.0 * v[1] - 1.0); ph[2] = v[2] * (2.0 * v[2] - 1.0);
    ph[3] = 4.0 * v[0] * v[1]; ph[4] = 4.0 * v[0] * v[2]; ph[5] = 4.0 * v[1] * v[2];
  }
  for (int m = 0; m < 6; ++m) phv[(size_t)m * ws] = ph[m];
  // converged jumps (paper ordering in the state -> heap order here)
  const int nzf = 6 * t.nz;
  for (int f = 0; f < 3 * N; ++f) {
    const int node = f / 3, c = f - 3 * node;
    const int lvl = 32 - __clz(node + 1);
    const int j = CMP ? node : (1 << t.K) - 3 * (1 << (lvl - 1)) + node + 1;
    a[(size_t)f * ws] = P.state_out[(size_t)(nzf + 3 * j + c) * P.n + pt];
  }
  double Eloc[6];
  local_strain(P.Q + 9 * pt, P.En + 6 * pt, P.dE + 6 * pt, Eloc);
  PointArrays A{};
  A.nrm = nrm; A.ns = ws; A.nrmf = nullptr;
  A.a = a; A.a_out = a; A.as = ws; A.paper = false;
  A.z = P.state_in + pt; A.zs = (size_t)P.n;
  // condensation at the converged jumps: H of every laminate and the tangent
  Sub<double> root;
  double r2;
  GH<double> g{gh, ws, gh};
  if (CMP) tree_pass_c<double, true>(t, Eloc, A, g, false, 1.0, root, r2, nullptr);
  else tree_pass<double, true>(t, Eloc, A, g, false, 1.0, root, r2, nullptr);
  // loss gradient into the local frame: sigma_glob = R sigma_loc  =>  g_loc = R^T g_glob
  double R[6][6], gl[6];
  mandel_rotation(P.Q + 9 * pt, R);
#pragma unroll
  for (int J = 0; J < 6; ++J) {
    double s = 0.0;
#pragma unroll
    for (int I = 0; I < 6; ++I) s += R[I][J] * P.g_stress[6 * pt + I];
    gl[J] = s;
  }
  if (CMP) {
    adjoint_pass_c(t, Eloc, gl, phv, ws, A, Wk);
    adjoint_weights_c(t, t.wl, t.wsum, Wk, gw, ws);
  } else {
    adjoint_pass(t, Eloc, gl, phv, ws, A, Wk);
    adjoint_weights(t, t.wl, t.wsum, Wk, gw, ws);
  }
  if (P.g_E) {   // dL/dE = C^T g (C symmetric), rotated back
    double ge[6];
#pragma unroll
    for (int I = 0; I < 6; ++I) {
      double s = 0.0;
#pragma unroll
      for (int J = 0; J < 6; ++J) s += root.C[sidx(I, J)] * gl[J];
      ge[I] = s;
    }
#pragma unroll
    for (int I = 0; I < 6; ++I) {
      double s = 0.0;
#pragma unroll
      for (int J = 0; J < 6; ++J) s += R[I][J] * ge[J];
      P.g_E[6 * pt + I] = s;
    }
  }
}

// Sums the per-point gradients of a chunk into the parameter gradients (added to
// g_p, g_q, g_w in the paper's ordering): one CTA per parameter, fixed-order
// reduction, so results are repeatable bit for bit.
__global__ void __launch_bounds__(256) k_grad_reduce(TreeDev t, int64_t nc, const double* __restrict__ work,
                                                     double* g_p, double* g_q, double* g_w) {
  const int r = blockIdx.x;
  const int N = t.N, M = t.M, L = t.L;
  const size_t ws = (size_t)nc;
  const double* base;
  const double* fac = nullptr;
  double* out;
  if (r < 2 * N * M) {
    const int which = r / (N * M), rr = r % (N * M), node = rr / M, m = rr % M;
    base = work + (size_t)(31 * N + which * N + node) * ws;
    fac = work + (size_t)(33 * N + 2 * L + m) * ws;
    const int lvl = 32 - __clz(node + 1);
    const int j = t.pidx ? t.pidx[node] : (1 << t.K) - 3 * (1 << (lvl - 1)) + node + 1;
    out = (which ? g_q : g_p) + j * M + m;
  } else {
    const int l = r - 2 * N * M;
    base = work + (size_t)(33 * N + L + l) * ws;
    out = g_w + l;
  }
  double s = 0.0;
  for (int64_t i = threadIdx.x; i < nc; i += blockDim.x) s += fac ? base[i] * fac[i] : base[i];
  __shared__ double red[256];
  red[threadIdx.x] = s;
  __syncthreads();
  for (int h = blockDim.x / 2; h > 0; h >>= 1) {
    if ((int)threadIdx.x < h) red[threadIdx.x] += red[threadIdx.x + h];
    __syncthreads();
  }
  if (threadIdx.x == 0) *out += red[0];
}

// Tangent seeds (trees of elastic phases): one warp per point of a chunk, in the work layout
// of k_grad plus the stiffness adjoints (grad_fields_tangent).  The lanes share each level of
// the tree (tangent_level_fwd / _rev), with a warp barrier between levels: the batches of the
// offline training (a few thousand samples) then keep the GPU's FP64 pipes busy, where one
// thread per point left most of them idle.  After k_grad (stress seeds) the normals and
// shape-function values are in the work array and the tangent's terms are added; alone (init)
// the kernel computes them and starts the per-laminate and per-leaf terms at zero.  The weight
// gradient is then (re)assembled from all terms by lane 0.
struct GradTParams {
  TreeDev t;
  int64_t n, n0, nc;
  const double *lam, *Q, *g_tangent;
  double* g_E;
  double* work;
  int init;
};

template <bool CMP>
__global__ void __launch_bounds__(128) k_grad_tangent(GradTParams P) {
  const int64_t i = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;   // this warp's point
  const int lane = threadIdx.x & 31;
  if (i >= P.nc) return;   // the whole warp
  const int64_t pt = P.n0 + i;
  const TreeDev& t = P.t;
  const int N = t.N, L = t.L;
  const size_t ws = (size_t)P.nc;
  double* w = P.work + i;
  double* nrm = w;
  double* Cst = w + (size_t)(6 * N) * ws;                       // the g, H field of k_grad: stiffnesses
  double* Gst = w + grad_fields(N, L) * ws;                     // stiffness adjoints
  AdjWork Wk;
  Wk.H = nullptr; Wk.hs = ws;
  Wk.mu = w + (size_t)(27 * N) * ws;
  Wk.xi = w + (size_t)(30 * N) * ws;
  Wk.gab = w + (size_t)(31 * N) * ws;
  Wk.direct = w + (size_t)(33 * N) * ws;
  Wk.ws = ws;
  double* gw = w + (size_t)(33 * N + L) * ws;
  double* phv = w + (size_t)(33 * N + 2 * L) * ws;   // shape-function values (k_grad writes them too)
  if (P.init) {
    const double l1 = P.lam[2 * pt], l2 = P.lam[2 * pt + 1];
    point_normals(t, l1, l2, nrm, ws, lane, 32);
    if (lane == 0) {
      const double v[3] = {l1 - l2, 3.0 * (1.0 - l1 - l2), 2.0 * l1 + 4.0 * l2 - 2.0};
      double ph[6] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
      if (t.M == 3) {
        ph[0] = v[0]; ph[1] = v[1]; ph[2] = v[2];
      } else if (t.M == 4) {
        const double b = v[0] * v[1] * v[2];
        ph[0] = v[0] - 9.0 * b; ph[1] = v[1] - 9.0 * b; ph[2] = v[2] - 9.0 * b; ph[3] = 27.0 * b;
      } else {
        ph[0] = v[0] * (2.0 * v[0] - 1.0); ph[1] = v[1] * (2.0 * v[1] - 1.0); ph[2] = v[2] * (2.0 * v[2] - 1.0);
        ph[3] = 4.0 * v[0] * v[1]; ph[4] = 4.0 * v[0] * v[2]; ph[5] = 4.0 * v[1] * v[2];
      }
      for (int m = 0; m < 6; ++m) phv[(size_t)m * ws] = ph[m];
      if (P.g_E)   // the tangent of elastic phases does not depend on the macro strain
        for (int I = 0; I < 6; ++I) P.g_E[6 * pt + I] = 0.0;
    }
    for (int k = lane; k < 2 * N; k += 32) Wk.gab[(size_t)k * ws] = 0.0;
    for (int k = lane; k < N; k += 32) Wk.xi[(size_t)k * ws] = 0.0;
    for (int l = lane; l < L; l += 32) Wk.direct[(size_t)l * ws] = 0.0;
  }
  if (lane == 0) {
    // the seed in the local frame: C_glob = R C_loc R^T  =>  Gb_loc = R^T G R, symmetrised
    double R[6][6];
    mandel_rotation(P.Q + 9 * pt, R);
    const double* G = P.g_tangent + 36 * pt;
    double RG[6][6];
    for (int P2 = 0; P2 < 6; ++P2)
      for (int J = 0; J < 6; ++J) {
        double v = 0.0;
        for (int I = 0; I < 6; ++I) v += R[I][P2] * G[6 * I + J];
        RG[P2][J] = v;
      }
    const int root = tangent_root(t, CMP);
    for (int I = 0; I < 6; ++I)
      for (int J = I; J < 6; ++J) {
        double a = 0.0, b = 0.0;
        for (int K2 = 0; K2 < 6; ++K2) { a += RG[I][K2] * R[K2][J]; b += RG[J][K2] * R[K2][I]; }
        Gst[(size_t)(21 * root + sidx(I, J)) * ws] = 0.5 * (a + b);
      }
  }
  double Cph[2][21];
  phase_stiffnesses(t, Cph);
  PointArrays A{};
  A.nrm = nrm; A.ns = ws;
  __syncwarp();
  for (int lvl = t.K; lvl >= 1; --lvl) {
    tangent_level_fwd(t, CMP, lvl, lane, 32, A, Cph, Cst, ws);
    __syncwarp();
  }
  for (int lvl = 1; lvl <= t.K; ++lvl) {
    tangent_level_rev(t, CMP, lvl, lane, 32, phv, ws, A, Cph, Cst, Gst, Wk);
    __syncwarp();
  }
  if (lane == 0) {
    if (CMP) adjoint_weights_c(t, t.wl, t.wsum, Wk, gw, ws);
    else adjoint_weights(t, t.wl, t.wsum, Wk, gw, ws);
  }
}

int64_t div_up(int64_t a, int64_t b) { return (a + b - 1) / b; }

// parameters of a tree description in heap order (array index = heap number - 1)
void heap_params(const dmn_tree_desc& d, double* ph, double* qh) {
  const int K = d.K, M = d.M;
  for (int k = 1; k <= K; ++k)
    for (int i = 1; i <= (1 << (k - 1)); ++i) {
      const int j = (1 << K) - (1 << k) + (i - 1);  // paper ordering
      const int hn = (1 << (k - 1)) + i - 2;       // array index (heap number - 1)
      for (int m = 0; m < M; ++m) { ph[hn * M + m] = d.p[j * M + m]; qh[hn * M + m] = d.q[j * M + m]; }
    }
}

const char* check_tree(const dmn_tree_desc& d, bool allow_zero = false) {
  if (d.K < 1 || d.K > KMAX) return "K must be in 1..8";
  if (d.M != 3 && d.M != 4 && d.M != 6) return "M must be 3, 4 or 6";
  if (!d.p || !d.q || !d.w) return "p, q, w must be non-NULL";
  const int N = (1 << d.K) - 1, L = 1 << d.K;
  double wsum = 0.0;
  for (int l = 0; l < L; ++l) {
    if (!std::isfinite(d.w[l]) || !(allow_zero ? d.w[l] >= 0.0 : d.w[l] > 0.0))
      return allow_zero ? "leaf weights must be finite and >= 0" : "leaf weights must be finite and > 0";
    wsum += d.w[l];
  }
  if (!(wsum > 0.0)) return "leaf weights must not all be zero";
  for (int j = 0; j < N * d.M; ++j)
    if (!std::isfinite(d.p[j]) || !std::isfinite(d.q[j])) return "p, q must be finite";
  return nullptr;
}

// Tree compression (Sec. 3.1): leaves of weight zero are removed, a laminate
// with one weightless subtree is replaced by the other subtree, one with two is
// removed.  The remaining laminates are numbered in the paper's order (level K
// first, root last) -- the numbering of their jumps in the state -- and the
// compressed tree is described by traversal tables (see TreeDev).  With all
// weights positive the result is the full tree in table form.
struct CmpTree {
  int N = 0, Lc = 0, nz = 0;
  std::vector<double> p, q, c;   // p, q [N][M]; c = c1 [N], c2 [N], sc [N], leaf weights [L], 1 / (c1 c2) [N]
  std::vector<float> cf;         // c1f [N], c2f [N], c12f [N], scf [N], 1 / (c1 c2) [N]
  std::vector<int> tab;          // lf [Lc] (4 ints each), pre [N], post [N], paper index [N], children [2 N],
                                 // the laminate at each heap position [2^K - 1], leaf children's state slots [2 N]
};

void build_compressed(const dmn_tree_desc& d, const bool inelastic[2], CmpTree& B) {
  const int K = d.K, M = d.M, N = (1 << K) - 1, L = 1 << K;
  double ws = 0.0;
  for (int l = 0; l < L; ++l) ws += d.w[l];
  // heap numbering 1..N for laminates, N+1..N+L for leaves; children of h: 2h, 2h+1
  std::vector<double> W(2 * N + 2, 0.0);
  for (int l = 0; l < L; ++l) W[N + 1 + l] = d.w[l] / ws;
  for (int h = N; h >= 1; --h) W[h] = W[2 * h] + W[2 * h + 1];
  std::vector<int> cid(N + 1, -1);
  std::vector<int> paper_of;    // paper index of each kept laminate
  for (int k = K; k >= 1; --k)
    for (int i = 1; i <= (1 << (k - 1)); ++i) {
      const int h = (1 << (k - 1)) + i - 1;
      if (W[2 * h] > 0.0 && W[2 * h + 1] > 0.0) {
        cid[h] = (int)paper_of.size();
        paper_of.push_back((1 << K) - (1 << k) + (i - 1));
      }
    }
  const int Nc = (int)paper_of.size();
  B.N = Nc;
  B.p.resize((size_t)Nc * M); B.q.resize((size_t)Nc * M);
  B.c.assign(4 * (size_t)Nc + L, 0.0); B.cf.assign(5 * (size_t)Nc, 0.0f);
  for (int c = 0; c < Nc; ++c)
    for (int m = 0; m < M; ++m) { B.p[c * M + m] = d.p[paper_of[c] * M + m]; B.q[c * M + m] = d.q[paper_of[c] * M + m]; }
  for (int h = 1; h <= N; ++h) {
    const int c = cid[h];
    if (c < 0) continue;
    const double c1 = W[2 * h] / W[h], c2 = 1.0 - c1;
    B.c[c] = c1; B.c[Nc + c] = c2; B.c[2 * Nc + c] = W[h] * c1 * c2;
    B.cf[c] = (float)c1; B.cf[Nc + c] = (float)c2; B.cf[2 * Nc + c] = (float)(c1 * c2);
    B.cf[3 * Nc + c] = (float)B.c[2 * Nc + c];
    B.c[3 * Nc + L + c] = 1.0 / (c1 * c2);
    B.cf[4 * Nc + c] = (float)(1.0 / (c1 * c2));
  }
  for (int l = 0; l < L; ++l) B.c[3 * Nc + l] = W[N + 1 + l];
  std::vector<int> lf, pre, post;
  B.nz = 0;
  // depth-first walk of the compressed tree: `top` is the depth where the
  // current descent started, `depth` the depth in the compressed tree
  struct Walk {
    const std::vector<double>& W; const std::vector<int>& cid; const bool* inel; int N;
    std::vector<int>& lf; std::vector<int>& pre; std::vector<int>& post; int& nz;
    void go(int h, int depth, int top) {
      if (!(W[h] > 0.0)) return;
      if (h > N) {                                     // a leaf
        const int l = h - N - 1, ph = l & 1;
        const int slot = inel[ph] ? nz++ : -1;
        lf.insert(lf.end(), {top, depth - top, 0, (l << 12) | ((slot + 1) << 2) | (ph << 1)});
        return;
      }
      if (cid[h] < 0) {                                // one weightless side: pass the other through
        go(W[2 * h] > 0.0 ? 2 * h : 2 * h + 1, depth, top);
        return;
      }
      pre.push_back(cid[h]);
      go(2 * h, depth + 1, top);
      go(2 * h + 1, depth + 1, depth + 1);
      post.push_back(cid[h]);
      lf[lf.size() - 2] += 1;                          // completed right after the last leaf
    }
  } walk{W, cid, inelastic, N, lf, pre, post, B.nz};
  walk.go(1, 0, 0);
  const int Lc = (int)lf.size() / 4;
  for (int l = 0; l + 1 < Lc; ++l)   // two sibling leaves: the left completes nothing, the right descends nothing
    if (lf[4 * l + 2] == 0 && lf[4 * (l + 1) + 1] == 0) lf[4 * l + 3] |= 1;
  B.Lc = Lc;
  B.tab = lf;
  B.tab.insert(B.tab.end(), pre.begin(), pre.end());
  B.tab.insert(B.tab.end(), post.begin(), post.end());
  B.tab.insert(B.tab.end(), paper_of.begin(), paper_of.end());
  // children of every kept laminate, laminates passed through skipped: a kept laminate's
  // number, or -1 - phase for a leaf
  std::vector<int> kids(2 * (size_t)Nc, 0);
  auto stand_in = [&](int x) {
    while (x <= N && cid[x] < 0) x = W[2 * x] > 0.0 ? 2 * x : 2 * x + 1;
    return x > N ? -1 - ((x - N - 1) & 1) : cid[x];
  };
  for (int h = 1; h <= N; ++h)
    if (cid[h] >= 0) { kids[2 * cid[h]] = stand_in(2 * h); kids[2 * cid[h] + 1] = stand_in(2 * h + 1); }
  B.tab.insert(B.tab.end(), kids.begin(), kids.end());
  for (int h = 1; h <= N; ++h) B.tab.push_back(cid[h]);   // heap position h - 1: its laminate or -1
  // the state slot of every child that is a leaf (the slots of the leaf table, in leaf order)
  std::vector<int> slot_of(L, -1), kslot(2 * (size_t)Nc, -1);
  for (int l = 0; l < Lc; ++l) slot_of[lf[4 * l + 3] >> 12] = ((lf[4 * l + 3] >> 2) & 1023) - 1;
  for (int h = 1; h <= N; ++h)
    if (cid[h] >= 0)
      for (int side = 0; side < 2; ++side) {
        int x = 2 * h + side;
        while (x <= N && cid[x] < 0) x = W[2 * x] > 0.0 ? 2 * x : 2 * x + 1;
        if (x > N) kslot[2 * cid[h] + side] = slot_of[x - N - 1];
      }
  B.tab.insert(B.tab.end(), kslot.begin(), kslot.end());
}

bool has_zero_weight(const dmn_tree_desc& d) {
  for (int l = 0; l < (1 << d.K); ++l)
    if (d.w[l] == 0.0) return true;
  return false;
}

}  // namespace

// ============================================================================
// C ABI

namespace {

// the all-FP32 first stage: on by default in the mixed forms, on request in the FP64 form; never
// with the line search or the extrapolated start
bool first_stage_on(const dmn_options& o) {
  const bool want = o.first_stage == 1 || (o.first_stage == 0 && o.precision != DMN_PREC_F64);
  return want && !o.line_search && !o.predictor;
}

// the warp organisation: for the paper's start (heap or compressed trees), always on request, by default
// (unless the first stage was asked for) for calls of at most warp_auto_points_per_sm points per SM.
// Below that the thread-per-point kernel leaves SMs idle or nearly so.  At depth 8 on 152 SMs,
// FP64: one point per warp is 20x faster than one point per thread at 1024 points; four points per
// warp (8 lanes each) 9.9x at 4096, 1.85x at 32768, 1.36x at 65536, 1.12x at 131072.  FP32
// condensation: one point per warp 6.2x at 1024, two per warp 4.7x at 4096, 1.48x at 32768, even
// at about 45000.
int warp_auto_points_per_sm(const dmn_handle* h) { return h->opt.precision == DMN_PREC_F64 ? 1024 : 256; }
bool warp_possible(const dmn_handle* h) {
  if (h->opt.warp_per_point < 0 || h->opt.predictor) return false;
  for (const Tree& t : h->trees)
    if (t.N < 1) return false;   // a compressed tree reduced to one leaf: no laminate to hold the result
  return true;
}
bool warp_on(const dmn_handle* h, int64_t n) {
  return warp_possible(h) && (h->opt.warp_per_point == 1 ||
                              (h->opt.first_stage != 1 && n <= (int64_t)warp_auto_points_per_sm(h) * h->n_sm));
}
// lanes per point of the warp organisation: the option's, else by the call's size: 32 while there
// are few points per SM (latency), then fewer (fewer idle lanes on the upper levels): 8 for the
// FP64 condensation, 16 for the FP32 one (whose FP64 work is a smaller part)
int warp_lanes_for(const dmn_handle* h, int64_t n) {
  if (h->opt.warp_lanes) return h->opt.warp_lanes;
  if (n <= 16 * (int64_t)h->n_sm) return 32;
  return h->opt.precision == DMN_PREC_F64 ? 8 : 16;
}

// Per-slot scratch and counters of one work set (per-point buffers come with the first update).
cudaError_t alloc_ws(const dmn_handle* h, WorkSet& w) {
  // per slot: normals + one or two jump buffers (FP64); one or two g, H buffers + FP32 normals
  const size_t sd = h->opt.line_search ? 9 : 6, stt = h->opt.line_search ? 45 : 24;
  cudaError_t e = cudaMalloc(&w.scr_d, sizeof(double) * (size_t)(sd * h->N_max) * h->nslots);
  if (e == cudaSuccess) e = cudaMalloc(&w.scr_t, sizeof(double) * (size_t)(stt * h->N_max) * h->nslots);
  if (e == cudaSuccess) e = cudaMalloc(&w.counter, sizeof(unsigned long long) * 32);
  if (e == cudaSuccess && first_stage_on(h->opt)) {
    w.nslots_s = (int64_t)h->n_sm * h->opt.stage_ctas_per_sm * 128;
    e = cudaMalloc(&w.scr_s, sizeof(float) * (size_t)(27 * h->N_max) * w.nslots_s);
  }
  if (e == cudaSuccess && warp_possible(h)) {
    // one slot per group of the smallest size the handle may use
    w.nwarps_w = (int64_t)h->n_sm * WARP_CTAS_PER_SM * 128 / (h->opt.warp_lanes ? h->opt.warp_lanes : WARP_MIN_LANES);
    // FP64 slots where an FP64 pass runs in them (the FP64 form's Newton, the mixed form's final sweep)
    const size_t per = h->opt.precision == DMN_PREC_MIXED_F32_TANGENT ? warp_slot_doubles<float>(h->N_max)
                                                                     : warp_slot_doubles<double>(h->N_max);
    e = cudaMalloc(&w.scr_w, sizeof(double) * per * (size_t)w.nwarps_w);
  }
  return e;
}

void free_ws(WorkSet& w) {
  cudaFree(w.scr_d); cudaFree(w.scr_t); cudaFree(w.scr_s); cudaFree(w.scr_w); cudaFree(w.counter); cudaFree(w.nbuf);
  cudaFree(w.perm);
  w = WorkSet();
}

void free_pipe(HostPipe& p) {
  for (int b = 0; b < 2; ++b) {
    cudaFree(p.buf[b]);
    if (p.comp[b]) cudaStreamDestroy(p.comp[b]);
    if (p.h2d[b]) cudaEventDestroy(p.h2d[b]);
    if (p.done[b]) cudaEventDestroy(p.done[b]);
    if (p.d2h[b]) cudaEventDestroy(p.d2h[b]);
  }
  if (p.up) cudaStreamDestroy(p.up);
  if (p.down) cudaStreamDestroy(p.down);
  if (p.start) cudaEventDestroy(p.start);
  p = HostPipe();
}

// Newton kernel variant for the launch shape: register cap by resident CTAs, line search.
template <typename T, bool CMP, bool PRED>
void launch_newton_p(const NewtonParams<T>& P, bool ls, int minb, unsigned grid, int block, cudaStream_t s) {
  if (ls) k_newton<T, 2, true, CMP, PRED><<<grid, block, 0, s>>>(P);
  else if (minb == 2) k_newton<T, 2, false, CMP, PRED><<<grid, block, 0, s>>>(P);
  else if (minb == 3) k_newton<T, 3, false, CMP, PRED><<<grid, block, 0, s>>>(P);
  else k_newton<T, 4, false, CMP, PRED><<<grid, block, 0, s>>>(P);
}
// the first stage's kernel: ctas resident CTAs of 128 threads per SM (registers capped to fit)
template <bool CMP>
void launch_stage(const StageParams& P, int ctas, unsigned grid, cudaStream_t s) {
  if (ctas <= 2) k_stage32<2, CMP><<<grid, 128, 0, s>>>(P);
  else if (ctas == 3) k_stage32<3, CMP><<<grid, 128, 0, s>>>(P);
  else if (ctas == 4) k_stage32<4, CMP><<<grid, 128, 0, s>>>(P);
  else if (ctas <= 6) k_stage32<6, CMP><<<grid, 128, 0, s>>>(P);
  else k_stage32<8, CMP><<<grid, 128, 0, s>>>(P);
}

template <typename T, bool CMP>
void launch_newton(const NewtonParams<T>& P, bool ls, int minb, unsigned grid, int block, cudaStream_t s) {
  if (P.predictor) launch_newton_p<T, CMP, true>(P, ls, minb, grid, block, s);
  else launch_newton_p<T, CMP, false>(P, ls, minb, grid, block, s);
}

// One update on work set w and stream s (the body of dmn_update; arguments checked by the caller).
// n_call is the size of the whole call (the sum of its chunks for dmn_update_host): it alone
// chooses between the warp and the thread-per-point organisation, so that a call's points get
// the same kernel whatever its chunks.
int update_on(dmn_handle* h, WorkSet& w, int64_t n, int64_t n_call, const int32_t* tree_id, const double* lam,
              const double* Q, const double* E_n, const double* dE, const double* state_in, double* state_out,
              double* stress, double* tangent, int32_t* iters, int32_t* status, cudaStream_t s) {
  cudaError_t e;
  const int NM = h->N_max;
  const bool sort = tree_id && h->trees.size() > 1;
  if (n > w.nbuf_cap) {
    e = cudaStreamSynchronize(s);
    if (e == cudaSuccess) {
      cudaFree(w.nbuf); cudaFree(w.perm);
      w.nbuf = nullptr; w.perm = nullptr; w.nbuf_cap = 0;
    }
    if (e == cudaSuccess) e = cudaMalloc(&w.nbuf, sizeof(double) * (size_t)(3 * NM + 6) * n);
    if (e == cudaSuccess) e = cudaMalloc(&w.perm, sizeof(int64_t) * (size_t)n);
    if (e != cudaSuccess) return cuda_fail(h, e, "dmn_update: per-point buffer");
    w.nbuf_cap = n;
  }
  Forest F;
  F.n = (int)h->trees.size();
  for (int k = 0; k < F.n; ++k) F.t[k] = tree_dev(h->trees[k]);
  const unsigned g1 = (unsigned)div_up(n, 128);
  cudaEvent_t* ev = nullptr;
  if (h->profiling) {
    if (h->events_used == h->events.size()) {
      std::array<cudaEvent_t, 5> a;
      for (auto& x : a) {
        e = cudaEventCreate(&x);
        if (e != cudaSuccess) return cuda_fail(h, e, "dmn_update: profiling event");
      }
      h->events.push_back(a);
    }
    ev = h->events[h->events_used++].data();
    cudaEventRecord(ev[0], s);
  }
  // counters: [0] work, [1..9] points per tree, [10..18] cursors, [19] first stage, [20] warp sweep
  e = cudaMemsetAsync(w.counter, 0, sizeof(unsigned long long) * 32, s);
  if (e != cudaSuccess) return cuda_fail(h, e, "dmn_update: counter reset");
  const int64_t* perm = nullptr;
  if (sort) {
    k_tree_count<<<g1, 128, 0, s>>>(n, tree_id, F.n, w.counter + 1);
    k_tree_offsets<<<1, 1, 0, s>>>(F.n, w.counter + 1, w.counter + 10);
    k_tree_scatter<<<g1, 128, 0, s>>>(n, tree_id, F.n, w.counter + 10, w.perm);
    perm = w.perm;
  }
  k_prepare<<<g1, 128, 0, s>>>(F, n, tree_id, perm, lam, Q, E_n, dE, w.nbuf, NM);
  if (ev) cudaEventRecord(ev[1], s);
  const unsigned grid = (unsigned)(h->n_sm * h->opt.ctas_per_sm);
  const bool mixed = h->opt.precision != DMN_PREC_F64;
  const bool sweep = h->opt.precision == DMN_PREC_MIXED;   // FP64 final sweep for stress and tangent
  const int threads_per_sm = h->opt.block * h->opt.ctas_per_sm;
  const int minb = threads_per_sm > 384 ? 4 : threads_per_sm > 256 ? 3 : 2;
  const bool ls = h->opt.line_search != 0;
  const int block = h->opt.block;
  const bool warp = warp_on(h, n_call) && w.scr_w;
  const bool stage = first_stage_on(h->opt) && !warp;   // a small batch goes straight to the warp kernel
  const unsigned wgrid = (unsigned)(h->n_sm * WARP_CTAS_PER_SM);
  const int lanes = warp ? warp_lanes_for(h, n_call) : 32;
  unsigned long long* passes = h->profiling ? h->d_passes : nullptr;
  if (stage) {   // counter [19]: the first stage's work counter
    // its corrections count against max_iter: the FP64-residual iteration keeps at least one
    const int max32 = std::max(0, std::min(STAGE_MAX_ITER, h->opt.max_iter - 1));
    StageParams SP{F, n, w.nslots_s, NM, tree_id, perm, state_in, state_out, iters, w.nbuf, w.scr_s,
                   w.counter + 19, STAGE_TOL, max32, passes};
    const unsigned sgrid = (unsigned)(h->n_sm * h->opt.stage_ctas_per_sm);
    if (h->cmp) launch_stage<true>(SP, h->opt.stage_ctas_per_sm, sgrid, s);
    else launch_stage<false>(SP, h->opt.stage_ctas_per_sm, sgrid, s);
  }
  if (ev) cudaEventRecord(ev[2], s);
  if (!mixed) {
    NewtonParams<double> P{F, n, h->nslots, NM, tree_id, perm, state_in, state_out, stress, tangent, iters, status,
                           w.nbuf, w.scr_d, (double*)w.scr_t, w.counter, h->opt.tol, h->opt.max_iter, 1,
                           h->opt.predictor, dE, stage ? state_out : nullptr, passes ? passes + 1 : nullptr,
                           stage ? 1 : 0};
    if (warp && h->cmp) launch_warp<double, true>(P, ls, lanes, wgrid, w.scr_w, s);
    else if (warp) launch_warp<double, false>(P, ls, lanes, wgrid, w.scr_w, s);
    else if (h->cmp) launch_newton<double, true>(P, ls, minb, grid, block, s);
    else launch_newton<double, false>(P, ls, minb, grid, block, s);
  } else {
    NewtonParams<float> P{F, n, h->nslots, NM, tree_id, perm, state_in, state_out, stress, tangent, iters, status,
                          w.nbuf, w.scr_d, (float*)w.scr_t, w.counter, h->opt.tol, h->opt.max_iter, sweep ? 0 : 1,
                          h->opt.predictor, dE, stage ? state_out : nullptr, passes ? passes + 1 : nullptr, 0};
    if (warp && h->cmp) launch_warp<float, true>(P, ls, lanes, wgrid, w.scr_w, s);
    else if (warp) launch_warp<float, false>(P, ls, lanes, wgrid, w.scr_w, s);
    else if (h->cmp) launch_newton<float, true>(P, ls, minb, grid, block, s);
    else launch_newton<float, false>(P, ls, minb, grid, block, s);
  }
  if (ev) cudaEventRecord(ev[3], s);
  FinalParams FP{F, n, NM, tree_id, perm, Q, state_in, state_out, stress, tangent, status, w.nbuf};
  if (sweep && warp) {   // the FP64 sweep in the warp organisation (counter [20]), then k_final rotates
    NewtonParams<double> SP{F, n, h->nslots, NM, tree_id, perm, state_in, state_out, stress, tangent, iters, status,
                            w.nbuf, w.scr_d, (double*)w.scr_t, w.counter + 20, h->opt.tol, h->opt.max_iter, 1, 0,
                            dE, nullptr, nullptr, 0};
    const int swl = h->opt.warp_lanes ? h->opt.warp_lanes : (n_call <= 16 * (int64_t)h->n_sm ? 32 : 8);
    if (h->cmp) launch_sweep_warp<true>(SP, swl, wgrid, w.scr_w, s);
    else launch_sweep_warp<false>(SP, swl, wgrid, w.scr_w, s);
    if (h->cmp) k_final<false, true><<<g1, 128, 0, s>>>(FP);
    else k_final<false, false><<<g1, 128, 0, s>>>(FP);
  } else if (sweep) {
    if (h->cmp) k_final<true, true><<<g1, 128, 0, s>>>(FP);
    else k_final<true, false><<<g1, 128, 0, s>>>(FP);
  } else {
    if (h->cmp) k_final<false, true><<<g1, 128, 0, s>>>(FP);
    else k_final<false, false><<<g1, 128, 0, s>>>(FP);
  }
  if (ev) cudaEventRecord(ev[4], s);
  e = cudaGetLastError();
  return e == cudaSuccess ? DMN_OK : cuda_fail(h, e, "dmn_update: launch");
}

// Device buffers of one dmn_update_host stage, carved out of one allocation.
struct StageView {
  int32_t *tid, *iters, *status;
  double *lam, *Q, *E_n, *dE, *state_in, *state_out, *stress, *tangent;
};

size_t stage_layout(int64_t cap, int64_t S, char* base, StageView* v) {
  size_t off = 0;
  auto take = [&](size_t bytes) {
    char* p = base ? base + off : nullptr;
    off += (bytes + 255) & ~size_t(255);
    return p;
  };
  const size_t c = (size_t)cap;
  StageView t;
  t.tid = (int32_t*)take(4 * c);
  t.iters = (int32_t*)take(4 * c);
  t.status = (int32_t*)take(4 * c);
  t.lam = (double*)take(16 * c);
  t.Q = (double*)take(72 * c);
  t.E_n = (double*)take(48 * c);
  t.dE = (double*)take(48 * c);
  t.stress = (double*)take(48 * c);
  t.tangent = (double*)take(288 * c);
  t.state_in = (double*)take(8 * c * (size_t)S);
  t.state_out = (double*)take(8 * c * (size_t)S);
  if (v) *v = t;
  return off;
}

// Streams, events, the second work set and stage buffers for chunks of `cap` points.
cudaError_t pipe_ready(dmn_handle* h, int64_t cap) {
  HostPipe& P = h->hp;
  cudaError_t e = cudaSuccess;
  if (!P.up) {
    e = cudaStreamCreateWithFlags(&P.up, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&P.down, cudaStreamNonBlocking);
    for (int b = 0; b < 2 && e == cudaSuccess; ++b) {
      e = cudaStreamCreateWithFlags(&P.comp[b], cudaStreamNonBlocking);
      if (e == cudaSuccess) e = cudaEventCreateWithFlags(&P.h2d[b], cudaEventDisableTiming);
      if (e == cudaSuccess) e = cudaEventCreateWithFlags(&P.done[b], cudaEventDisableTiming);
      if (e == cudaSuccess) e = cudaEventCreateWithFlags(&P.d2h[b], cudaEventDisableTiming);
    }
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&P.start, cudaEventDisableTiming);
    if (e != cudaSuccess) { free_pipe(P); return e; }
  }
  if (!h->ws[1].scr_d) {
    e = alloc_ws(h, h->ws[1]);
    if (e != cudaSuccess) { free_ws(h->ws[1]); return e; }
  }
  if (cap > P.cap) {
    for (int b = 0; b < 2; ++b) { cudaFree(P.buf[b]); P.buf[b] = nullptr; }
    P.cap = 0;
    const size_t bytes = stage_layout(cap, h->S_max, nullptr, nullptr);
    for (int b = 0; b < 2 && e == cudaSuccess; ++b) e = cudaMalloc(&P.buf[b], bytes);
    if (e != cudaSuccess) {
      for (int b = 0; b < 2; ++b) { cudaFree(P.buf[b]); P.buf[b] = nullptr; }
      return e;
    }
    P.cap = cap;
  }
  return e;
}

}  // namespace

extern "C" {

int dmn_create(const dmn_tree_desc* trees, int32_t n_trees, const dmn_options* opt, dmn_handle** out) {
  if (!out) return fail(nullptr, DMN_ERR_ARG, "dmn_create: out is NULL");
  *out = nullptr;
  g_create_error.clear();
  if (!trees || n_trees < 1 || n_trees > DMN_MAX_TREES)
    return fail(nullptr, DMN_ERR_ARG, "dmn_create: n_trees must be in 1..8 and trees non-NULL");
  std::vector<Tree> tv(n_trees);
  std::vector<CmpTree> cv(n_trees);
  int N_max = 0;
  int64_t S_max = 0;
  bool cmp = false;
  for (int k = 0; k < n_trees; ++k) {
    if (const char* m = check_tree(trees[k], true)) return fail(nullptr, DMN_ERR_ARG, std::string("dmn_create: ") + m);
    cmp = cmp || has_zero_weight(trees[k]);
  }
  for (int k = 0; k < n_trees; ++k) {
    const dmn_tree_desc& d = trees[k];
    Tree& t = tv[k];
    t.K = d.K; t.M = d.M; t.N = (1 << d.K) - 1; t.L = 1 << d.K;
    int n_inel_phase = 0;
    for (int f = 0; f < 2; ++f) {
      if (const char* m = make_phase(d.phase[f], t.ph[f]))
        return fail(nullptr, DMN_ERR_ARG, std::string("dmn_create: ") + m);
      n_inel_phase += d.phase[f].kind != DMN_PHASE_ELASTIC;
    }
    t.z_both = n_inel_phase == 2;
    t.nz = n_inel_phase * (t.L / 2);
    if (cmp) {   // every tree of the handle is walked by tables
      const bool inel[2] = {d.phase[0].kind != DMN_PHASE_ELASTIC, d.phase[1].kind != DMN_PHASE_ELASTIC};
      build_compressed(d, inel, cv[k]);
      t.cmp = 1;
      t.alive.resize(t.L);
      for (int l = 0; l < t.L; ++l) t.alive[l] = d.w[l] > 0.0;
      t.N = cv[k].N;
      t.Lc = cv[k].Lc;
      t.nz = cv[k].nz;
    }
    t.S = 6 * t.nz + 3 * t.N;
    N_max = std::max(N_max, t.N);
    S_max = std::max<int64_t>(S_max, t.S);
  }

  dmn_options o;
  o.tol = 1e-12; o.max_iter = 50; o.precision = DMN_PREC_F64; o.block = 128; o.ctas_per_sm = 0; o.line_search = 0;
  o.predictor = 0; o.first_stage = 0; o.stage_ctas_per_sm = 0; o.warp_per_point = 0;
  if (opt) {
    if (opt->tol > 0.0) o.tol = opt->tol;
    if (opt->max_iter > 0) o.max_iter = opt->max_iter;
    o.precision = opt->precision;
    if (opt->block > 0) o.block = opt->block;
    if (opt->ctas_per_sm > 0) o.ctas_per_sm = opt->ctas_per_sm;
    o.line_search = opt->line_search;
    o.predictor = opt->predictor;
    o.first_stage = opt->first_stage;
    o.stage_ctas_per_sm = opt->stage_ctas_per_sm;
    o.warp_per_point = opt->warp_per_point;
    o.warp_lanes = opt->warp_lanes;
  }
  if (o.warp_per_point < -1 || o.warp_per_point > 1)
    return fail(nullptr, DMN_ERR_ARG, "dmn_create: warp_per_point must be -1, 0 or 1");
  if (o.warp_lanes != 0 && o.warp_lanes != 8 && o.warp_lanes != 16 && o.warp_lanes != 32)
    return fail(nullptr, DMN_ERR_ARG, "dmn_create: warp_lanes must be 0, 8, 16 or 32");
  if (o.first_stage < -1 || o.first_stage > 1)
    return fail(nullptr, DMN_ERR_ARG, "dmn_create: first_stage must be -1, 0 or 1");
  if (o.stage_ctas_per_sm == 0) o.stage_ctas_per_sm = STAGE_CTAS_DEFAULT;
  if (o.stage_ctas_per_sm != 2 && o.stage_ctas_per_sm != 3 && o.stage_ctas_per_sm != 4 && o.stage_ctas_per_sm != 6 &&
      o.stage_ctas_per_sm != 8)
    return fail(nullptr, DMN_ERR_ARG, "dmn_create: stage_ctas_per_sm must be 0, 2, 3, 4, 6 or 8");
  if (o.line_search != 0 && o.line_search != 1) return fail(nullptr, DMN_ERR_ARG, "dmn_create: line_search must be 0 or 1");
  if (o.predictor != 0 && o.predictor != 1) return fail(nullptr, DMN_ERR_ARG, "dmn_create: predictor must be 0 or 1");
  if (o.predictor) {   // the last update's jump change and strain increment follow the jumps
    S_max = 0;
    for (Tree& t : tv) {
      t.S += 3 * t.N + 6;
      S_max = std::max<int64_t>(S_max, t.S);
    }
  }
  // the line-search kernel keeps two buffers per lane and is built for 256 threads per SM
  if (o.line_search && o.ctas_per_sm <= 0) o.ctas_per_sm = 256 / o.block;
  if (o.precision != DMN_PREC_F64 && o.precision != DMN_PREC_MIXED && o.precision != DMN_PREC_MIXED_F32_TANGENT)
    return fail(nullptr, DMN_ERR_ARG, "dmn_create: unknown precision");
  if (o.block % 32 != 0 || o.block > 128)
    return fail(nullptr, DMN_ERR_ARG, "dmn_create: block must be a multiple of 32 and at most 128");
  // default occupancy: the FP64 form is bound by the FP64 pipe from 256 threads per SM on;
  // the FP32 form hides latency with 512
  if (o.ctas_per_sm <= 0) o.ctas_per_sm = (o.precision != DMN_PREC_F64 ? 512 : 384) / o.block;
  if (o.block * o.ctas_per_sm > (o.line_search ? 256 : 512))
    return fail(nullptr, DMN_ERR_ARG, "dmn_create: block * ctas_per_sm must be at most 512 threads per SM "
                                      "(256 with the line search)");

  dmn_handle* h = new dmn_handle();
  h->trees = tv;
  h->cmp = cmp;
  h->N_max = std::max(N_max, 1);
  h->S_max = S_max;
  h->opt = o;
  cudaError_t e = cudaGetDevice(&h->device);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&h->n_sm, cudaDevAttrMultiProcessorCount, h->device);
  if (e != cudaSuccess) { delete h; return cuda_fail(nullptr, e, "dmn_create: device query"); }

  double* d_w = nullptr;
  e = cudaMalloc(&d_w, sizeof(double) * (1 << KMAX));
  for (int k = 0; k < n_trees && e == cudaSuccess; ++k) {
    const dmn_tree_desc& d = trees[k];
    Tree& T = h->trees[k];
    const int N = T.N, M = T.M, L = T.L;
    T.wsum = 0.0;
    for (int l = 0; l < L; ++l) T.wsum += d.w[l];
    if (T.cmp) {   // host-built parameters in the compressed numbering, and the tables
      const CmpTree& B = cv[k];
      const size_t np = std::max<size_t>(B.p.size(), 1), nc = B.c.size(), nf = std::max<size_t>(B.cf.size(), 1);
      e = cudaMalloc(&T.d_p, sizeof(double) * np);
      if (e == cudaSuccess) e = cudaMalloc(&T.d_q, sizeof(double) * np);
      if (e == cudaSuccess) e = cudaMalloc(&T.d_c, sizeof(double) * nc);
      if (e == cudaSuccess) e = cudaMalloc(&T.d_cf, sizeof(float) * nf);
      if (e == cudaSuccess) e = cudaMalloc(&T.d_tab, sizeof(int) * B.tab.size());
      if (e == cudaSuccess && !B.p.empty())
        e = cudaMemcpy(T.d_p, B.p.data(), sizeof(double) * B.p.size(), cudaMemcpyHostToDevice);
      if (e == cudaSuccess && !B.q.empty())
        e = cudaMemcpy(T.d_q, B.q.data(), sizeof(double) * B.q.size(), cudaMemcpyHostToDevice);
      if (e == cudaSuccess) e = cudaMemcpy(T.d_c, B.c.data(), sizeof(double) * nc, cudaMemcpyHostToDevice);
      if (e == cudaSuccess && !B.cf.empty())
        e = cudaMemcpy(T.d_cf, B.cf.data(), sizeof(float) * B.cf.size(), cudaMemcpyHostToDevice);
      if (e == cudaSuccess) e = cudaMemcpy(T.d_tab, B.tab.data(), sizeof(int) * B.tab.size(), cudaMemcpyHostToDevice);
      continue;
    }
    std::vector<double> ph(N * M), qh(N * M);
    heap_params(d, ph.data(), qh.data());
    e = cudaMalloc(&T.d_p, sizeof(double) * N * M);
    if (e == cudaSuccess) e = cudaMalloc(&T.d_q, sizeof(double) * N * M);
    if (e == cudaSuccess) e = cudaMalloc(&T.d_c, sizeof(double) * (4 * N + L));
    if (e == cudaSuccess) e = cudaMalloc(&T.d_cf, sizeof(float) * 5 * N);
    if (e == cudaSuccess) e = cudaMemcpy(T.d_p, ph.data(), sizeof(double) * N * M, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(T.d_q, qh.data(), sizeof(double) * N * M, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(d_w, d.w, sizeof(double) * L, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) {
      k_setup_tree<<<1, 1>>>(T.K, d_w, T.d_c, T.d_cf);
      e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
  }
  cudaFree(d_w);
  h->nslots = (int64_t)h->n_sm * o.ctas_per_sm * o.block;
  if (e == cudaSuccess) e = alloc_ws(h, h->ws[0]);
  if (e != cudaSuccess) {
    dmn_destroy(h);
    return cuda_fail(nullptr, e, "dmn_create");
  }
  *out = h;
  return DMN_OK;
}

void dmn_destroy(dmn_handle* h) {
  if (!h) return;
  cudaDeviceSynchronize();
  for (auto& a : h->events)
    for (auto& x : a) cudaEventDestroy(x);
  for (auto& t : h->trees) { cudaFree(t.d_p); cudaFree(t.d_q); cudaFree(t.d_c); cudaFree(t.d_cf); cudaFree(t.d_tab); }
  for (auto& w : h->ws) free_ws(w);
  free_pipe(h->hp);
  cudaFree(h->gwork);
  cudaFree(h->d_passes);
  delete h;
}

int64_t dmn_state_size(const dmn_handle* h, int32_t tree_id) {
  if (!h) return -1;
  if (tree_id == -1) return h->S_max;
  if (tree_id < 0 || tree_id >= (int)h->trees.size()) return -1;
  return h->trees[tree_id].S;
}

int dmn_update_lanes_per_point(const dmn_handle* h, int64_t n) {
  if (!h || n < 0) return -1;
  return warp_on(h, n) ? warp_lanes_for(h, n) : 1;
}

int dmn_profile_enable(dmn_handle* h, int32_t enable) {
  if (!h) return fail(nullptr, DMN_ERR_ARG, "dmn_profile_enable: NULL handle");
  if (enable) {
    cudaError_t e = cudaSuccess;
    if (!h->d_passes) e = cudaMalloc(&h->d_passes, 2 * sizeof(unsigned long long));
    if (e == cudaSuccess) e = cudaMemset(h->d_passes, 0, 2 * sizeof(unsigned long long));
    if (e != cudaSuccess) return cuda_fail(h, e, "dmn_profile_enable");
    h->events_used = 0;
  }
  h->profiling = enable != 0;
  return DMN_OK;
}

int dmn_profile_read_stages(dmn_handle* h, double ms[4], int64_t passes[2], int64_t* updates) {
  if (!h) return fail(nullptr, DMN_ERR_ARG, "dmn_profile_read_stages: NULL handle");
  if (!ms || !updates) return fail(h, DMN_ERR_ARG, "dmn_profile_read_stages: NULL output");
  ms[0] = ms[1] = ms[2] = ms[3] = 0.0;
  for (size_t i = 0; i < h->events_used; ++i) {
    const auto& a = h->events[i];
    cudaError_t e = cudaEventSynchronize(a[4]);
    if (e != cudaSuccess) return cuda_fail(h, e, "dmn_profile_read_stages");
    for (int k = 0; k < 4; ++k) {
      float t = 0.f;
      e = cudaEventElapsedTime(&t, a[k], a[k + 1]);
      if (e != cudaSuccess) return cuda_fail(h, e, "dmn_profile_read_stages");
      ms[k] += t;
    }
  }
  if (passes) {
    unsigned long long c[2] = {0, 0};
    if (h->d_passes) {
      cudaError_t e = cudaDeviceSynchronize();
      if (e == cudaSuccess) e = cudaMemcpy(c, h->d_passes, sizeof c, cudaMemcpyDeviceToHost);
      if (e != cudaSuccess) return cuda_fail(h, e, "dmn_profile_read_stages");
    }
    passes[0] = (int64_t)c[0];
    passes[1] = (int64_t)c[1];
  }
  *updates = (int64_t)h->events_used;
  return DMN_OK;
}

int dmn_profile_read(dmn_handle* h, double ms[3], int64_t* updates) {
  if (!h) return fail(nullptr, DMN_ERR_ARG, "dmn_profile_read: NULL handle");
  if (!ms || !updates) return fail(h, DMN_ERR_ARG, "dmn_profile_read: NULL output");
  double m4[4];
  const int rc = dmn_profile_read_stages(h, m4, nullptr, updates);
  if (rc != DMN_OK) return rc;
  ms[0] = m4[0]; ms[1] = m4[1] + m4[2]; ms[2] = m4[3];
  return DMN_OK;
}

const char* dmn_last_error(const dmn_handle* h) { return h ? h->err.c_str() : g_create_error.c_str(); }

int dmn_interp_orientation(dmn_handle* h, int64_t n, const double* A2, double* lam, double* Q, void* stream) {
  if (!h) return fail(nullptr, DMN_ERR_ARG, "dmn_interp_orientation: NULL handle");
  if (n < 0) return fail(h, DMN_ERR_ARG, "dmn_interp_orientation: n < 0");
  if (n == 0) return DMN_OK;
  if (!A2 || !lam || !Q) return fail(h, DMN_ERR_ARG, "dmn_interp_orientation: NULL array");
  cudaStream_t s = (cudaStream_t)stream;
  k_interp<<<(unsigned)div_up(n, 128), 128, 0, s>>>(n, A2, lam, Q);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? DMN_OK : cuda_fail(h, e, "dmn_interp_orientation");
}

int dmn_update(dmn_handle* h, int64_t n, const int32_t* tree_id, const double* lam, const double* Q,
               const double* E_n, const double* dE, const double* state_in, double* state_out, double* stress,
               double* tangent, int32_t* iters, int32_t* status, void* stream) {
  if (!h) return fail(nullptr, DMN_ERR_ARG, "dmn_update: NULL handle");
  if (n < 0) return fail(h, DMN_ERR_ARG, "dmn_update: n < 0");
  if (n == 0) return DMN_OK;
  if (!lam || !Q || !E_n || !dE || !state_in || !state_out || !stress || !tangent || !iters || !status)
    return fail(h, DMN_ERR_ARG, "dmn_update: NULL array");
  if (state_in == state_out) return fail(h, DMN_ERR_ARG, "dmn_update: state_in and state_out must differ");
  return update_on(h, h->ws[0], n, n, tree_id, lam, Q, E_n, dE, state_in, state_out, stress, tangent, iters, status,
                   (cudaStream_t)stream);
}

int dmn_update_host(dmn_handle* h, int64_t n, const int32_t* tree_id, const double* lam, const double* Q,
                    const double* E_n, const double* dE, const double* state_in, double* state_out, double* stress,
                    double* tangent, int32_t* iters, int32_t* status, int64_t chunk, void* stream) {
  if (!h) return fail(nullptr, DMN_ERR_ARG, "dmn_update_host: NULL handle");
  if (n < 0) return fail(h, DMN_ERR_ARG, "dmn_update_host: n < 0");
  if (n == 0) return DMN_OK;
  if (!lam || !Q || !E_n || !dE || !state_in || !state_out || !stress || !tangent || !iters || !status)
    return fail(h, DMN_ERR_ARG, "dmn_update_host: NULL array");
  if (chunk <= 0) chunk = 2 * h->nslots;
  chunk = std::min(chunk, n);
  cudaStream_t s = (cudaStream_t)stream;
  // the stage buffers may still be read by the copies of an earlier call that failed
  HostPipe& P = h->hp;
  if (P.up && chunk > P.cap) {
    cudaError_t e = cudaSuccess;
    for (cudaStream_t x : {P.up, P.comp[0], P.comp[1], P.down})
      if (e == cudaSuccess) e = cudaStreamSynchronize(x);
    if (e != cudaSuccess) return cuda_fail(h, e, "dmn_update_host: pipeline");
  }
  cudaError_t e = pipe_ready(h, chunk);
  if (e != cudaSuccess) return cuda_fail(h, e, "dmn_update_host: pipeline buffers");
  StageView v[2];
  for (int b = 0; b < 2; ++b) stage_layout(P.cap, h->S_max, P.buf[b], &v[b]);
  const int64_t S = h->S_max;
  const size_t host_pitch = sizeof(double) * (size_t)n;
  // work already queued on the caller's stream (an update on work set 0) comes first
  e = cudaEventRecord(P.start, s);
  for (cudaStream_t x : {P.up, P.comp[0], P.comp[1]})
    if (e == cudaSuccess) e = cudaStreamWaitEvent(x, P.start, 0);
  int rc = e == cudaSuccess ? DMN_OK : cuda_fail(h, e, "dmn_update_host: stream order");
  const auto H2D = cudaMemcpyHostToDevice, D2H = cudaMemcpyDeviceToHost;
  for (int64_t j = 0, n0 = 0; rc == DMN_OK && n0 < n; ++j, n0 += chunk) {
    const int b = (int)(j & 1);
    const int64_t c = std::min(chunk, n - n0);
    const size_t c8 = sizeof(double) * (size_t)c;
    const StageView& V = v[b];
    // inputs of chunk j, once the update of chunk j - 2 (same stage) has read its own
    if (j >= 2) e = cudaStreamWaitEvent(P.up, P.done[b], 0);
    if (e == cudaSuccess && tree_id) e = cudaMemcpyAsync(V.tid, tree_id + n0, 4 * (size_t)c, H2D, P.up);
    if (e == cudaSuccess) e = cudaMemcpyAsync(V.lam, lam + 2 * n0, 2 * c8, H2D, P.up);
    if (e == cudaSuccess) e = cudaMemcpyAsync(V.Q, Q + 9 * n0, 9 * c8, H2D, P.up);
    if (e == cudaSuccess) e = cudaMemcpyAsync(V.E_n, E_n + 6 * n0, 6 * c8, H2D, P.up);
    if (e == cudaSuccess) e = cudaMemcpyAsync(V.dE, dE + 6 * n0, 6 * c8, H2D, P.up);
    if (e == cudaSuccess) e = cudaMemcpy2DAsync(V.state_in, c8, state_in + n0, host_pitch, c8, (size_t)S, H2D, P.up);
    if (e == cudaSuccess) e = cudaEventRecord(P.h2d[b], P.up);
    // the update, once its inputs are in and the outputs of chunk j - 2 are out
    if (e == cudaSuccess) e = cudaStreamWaitEvent(P.comp[b], P.h2d[b], 0);
    if (e == cudaSuccess && j >= 2) e = cudaStreamWaitEvent(P.comp[b], P.d2h[b], 0);
    // a point of an unknown tree leaves its state_out untouched: give it state_in, so that
    // the copy-out returns the point's state unchanged rather than stale stage contents
    if (e == cudaSuccess && tree_id)
      e = cudaMemcpyAsync(V.state_out, V.state_in, c8 * (size_t)S, cudaMemcpyDeviceToDevice, P.comp[b]);
    if (e != cudaSuccess) { rc = cuda_fail(h, e, "dmn_update_host: copy in"); break; }
    rc = update_on(h, h->ws[b], c, n, tree_id ? V.tid : nullptr, V.lam, V.Q, V.E_n, V.dE, V.state_in, V.state_out,
                   V.stress, V.tangent, V.iters, V.status, P.comp[b]);
    if (rc != DMN_OK) break;
    e = cudaEventRecord(P.done[b], P.comp[b]);
    // outputs of chunk j
    if (e == cudaSuccess) e = cudaStreamWaitEvent(P.down, P.done[b], 0);
    if (e == cudaSuccess) e = cudaMemcpyAsync(stress + 6 * n0, V.stress, 6 * c8, D2H, P.down);
    if (e == cudaSuccess) e = cudaMemcpyAsync(tangent + 36 * n0, V.tangent, 36 * c8, D2H, P.down);
    if (e == cudaSuccess) e = cudaMemcpyAsync(iters + n0, V.iters, 4 * (size_t)c, D2H, P.down);
    if (e == cudaSuccess) e = cudaMemcpyAsync(status + n0, V.status, 4 * (size_t)c, D2H, P.down);
    if (e == cudaSuccess)
      e = cudaMemcpy2DAsync(state_out + n0, host_pitch, V.state_out, c8, c8, (size_t)S, D2H, P.down);
    if (e == cudaSuccess) e = cudaEventRecord(P.d2h[b], P.down);
    if (e != cudaSuccess) rc = cuda_fail(h, e, "dmn_update_host: copy out");
  }
  // the host arrays are in use until every copy has ended: wait for all four streams
  for (cudaStream_t x : {P.up, P.comp[0], P.comp[1], P.down}) {
    e = cudaStreamSynchronize(x);
    if (e != cudaSuccess && rc == DMN_OK) rc = cuda_fail(h, e, "dmn_update_host: pipeline");
  }
  return rc;
}

int dmn_set_params(dmn_handle* h, int32_t tree_id, const double* p, const double* q, const double* w) {
  if (!h) return fail(nullptr, DMN_ERR_ARG, "dmn_set_params: NULL handle");
  if (tree_id < 0 || tree_id >= (int)h->trees.size()) return fail(h, DMN_ERR_ARG, "dmn_set_params: bad tree_id");
  Tree& T = h->trees[tree_id];
  dmn_tree_desc d;
  d.K = T.K; d.M = T.M; d.p = p; d.q = q; d.w = w;
  if (const char* m = check_tree(d, h->cmp)) return fail(h, DMN_ERR_ARG, std::string("dmn_set_params: ") + m);
  if (h->cmp) {   // same compressed structure: new parameters in its numbering
    for (int l = 0; l < T.L; ++l)
      if ((w[l] > 0.0) != (T.alive.empty() ? true : T.alive[l] != 0))
        return fail(h, DMN_ERR_ARG, "dmn_set_params: the set of zero leaf weights changed (another compressed "
                                    "tree); create a new handle");
    const bool inel[2] = {T.ph[0].kind != 0, T.ph[1].kind != 0};
    CmpTree B;
    build_compressed(d, inel, B);
    cudaError_t e = cudaDeviceSynchronize();
    if (e == cudaSuccess && !B.p.empty())
      e = cudaMemcpy(T.d_p, B.p.data(), sizeof(double) * B.p.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess && !B.q.empty())
      e = cudaMemcpy(T.d_q, B.q.data(), sizeof(double) * B.q.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(T.d_c, B.c.data(), sizeof(double) * B.c.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess && !B.cf.empty())
      e = cudaMemcpy(T.d_cf, B.cf.data(), sizeof(float) * B.cf.size(), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return cuda_fail(h, e, "dmn_set_params");
    T.wsum = 0.0;
    for (int l = 0; l < T.L; ++l) T.wsum += w[l];
    return DMN_OK;
  }
  std::vector<double> ph(T.N * T.M), qh(T.N * T.M);
  heap_params(d, ph.data(), qh.data());
  cudaError_t e = cudaDeviceSynchronize();
  double* d_w = nullptr;
  if (e == cudaSuccess) e = cudaMalloc(&d_w, sizeof(double) * T.L);
  if (e == cudaSuccess) e = cudaMemcpy(T.d_p, ph.data(), sizeof(double) * T.N * T.M, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(T.d_q, qh.data(), sizeof(double) * T.N * T.M, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(d_w, w, sizeof(double) * T.L, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) {
    k_setup_tree<<<1, 1>>>(T.K, d_w, T.d_c, T.d_cf);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  cudaFree(d_w);
  if (e != cudaSuccess) return cuda_fail(h, e, "dmn_set_params");
  T.wsum = 0.0;
  for (int l = 0; l < T.L; ++l) T.wsum += w[l];
  return DMN_OK;
}

int dmn_grad(dmn_handle* h, int64_t n, const int32_t* tree_id, const double* lam, const double* Q, const double* E_n,
             const double* dE, const double* state_in, const double* state_out, const double* g_stress,
             const double* g_tangent, double* g_p, double* g_q, double* g_w, double* g_E, void* stream) {
  if (!h) return fail(nullptr, DMN_ERR_ARG, "dmn_grad: NULL handle");
  if (n < 0) return fail(h, DMN_ERR_ARG, "dmn_grad: n < 0");
  if (tree_id || h->trees.size() != 1) return fail(h, DMN_ERR_ARG, "dmn_grad: one tree only (tree_id must be NULL)");
  if (!g_stress && !g_tangent) return fail(h, DMN_ERR_ARG, "dmn_grad: g_stress and g_tangent are both NULL");
  const Tree& T = h->trees[0];
  const TreeDev td = tree_dev(T);
  if (g_tangent && (td.ph[0].kind != DMN_PHASE_ELASTIC || td.ph[1].kind != DMN_PHASE_ELASTIC))
    return fail(h, DMN_ERR_ARG, "dmn_grad: tangent seeds need a tree of elastic phases");
  if (n == 0) return DMN_OK;
  if (!lam || !Q || !g_p || !g_q || !g_w || (g_stress && (!E_n || !dE || !state_in || !state_out)))
    return fail(h, DMN_ERR_ARG, "dmn_grad: NULL array");
  cudaStream_t s = (cudaStream_t)stream;
  const int64_t chunk = std::min<int64_t>(n, 65536);   // few points per chunk leave the adjoint latency-bound
  const size_t fields = g_tangent ? grad_fields_tangent(T.N, T.L) : grad_fields(T.N, T.L);
  const int64_t need = (int64_t)(fields * (size_t)chunk);   // doubles
  cudaError_t e;
  if (need > h->gwork_cap) {
    e = cudaStreamSynchronize(s);
    if (e == cudaSuccess) { cudaFree(h->gwork); h->gwork = nullptr; h->gwork_cap = 0; }
    if (e == cudaSuccess) e = cudaMalloc(&h->gwork, sizeof(double) * (size_t)need);
    if (e != cudaSuccess) return cuda_fail(h, e, "dmn_grad: work buffer");
    h->gwork_cap = need;
  }
  const int n_params = 2 * T.N * T.M + T.L;
  for (int64_t n0 = 0; n0 < n; n0 += chunk) {
    const int64_t nc = std::min(chunk, n - n0);
    const unsigned grid = (unsigned)div_up(nc, 128);
    if (g_stress) {
      GradParams P{td, n, n0, nc, lam, Q, E_n, dE, state_in, state_out, g_stress, g_E, h->gwork};
      if (h->cmp) k_grad<true><<<grid, 128, 0, s>>>(P);
      else k_grad<false><<<grid, 128, 0, s>>>(P);
    }
    if (g_tangent) {
      GradTParams P{td, n, n0, nc, lam, Q, g_tangent, g_E, h->gwork, g_stress ? 0 : 1};
      const unsigned wgrid = (unsigned)div_up(32 * nc, 128);   // a warp per point
      if (h->cmp) k_grad_tangent<true><<<wgrid, 128, 0, s>>>(P);
      else k_grad_tangent<false><<<wgrid, 128, 0, s>>>(P);
    }
    k_grad_reduce<<<n_params, 256, 0, s>>>(td, nc, h->gwork, g_p, g_q, g_w);
  }
  e = cudaGetLastError();
  return e == cudaSuccess ? DMN_OK : cuda_fail(h, e, "dmn_grad: launch");
}

}  // extern "C"

// ============================================================================
// Update without any allocation (dmn_update_noalloc).
//
// Some callers cannot allocate device memory: code that runs where every byte of
// the device is handed out by someone else's pool or arena, or under policies that
// forbid cudaMalloc after start-up.  For them the update below keeps its whole work
// space -- tree parameters, the work counter and the per-lane scratch of the
// persistent Newton kernel -- in one file-scope device array of fixed size,
// DMN_NOALLOC_BYTES.  Every GPU that loads this library holds that array until the
// process exits.  The caller passes inputs and outputs as for dmn_update.

namespace {

constexpr size_t DMN_NOALLOC_BYTES = size_t(64) << 20;  // 64 MiB
constexpr size_t NOALLOC_PARAM_DOUBLES = 6144;          // p, q, w, c, cf for K <= 8, M <= 6
constexpr int NOALLOC_BLOCK = 128;

// [0, 256): work counter; [256, 256 + 8 * NOALLOC_PARAM_DOUBLES): tree parameters;
// the rest: per-lane scratch (normals, jumps, g and H of every laminate).
static __device__ __align__(256) unsigned char g_noalloc_scratch[DMN_NOALLOC_BYTES];

// Tree parameters passed by value as a kernel argument (26.5 KB at K = 8, M = 6, within
// the 32,764 bytes a kernel's arguments may take), so that nothing the call leaves queued
// refers to host memory once it has returned.
struct NoAllocUpload {
  int nm, L;
  double p[NMAX * 6], q[NMAX * 6];
  double w[1 << KMAX];
};
static_assert(sizeof(NoAllocUpload) <= 32764, "kernel argument too large");

__global__ void k_noalloc_upload(NoAllocUpload u, double* __restrict__ d_p, double* __restrict__ d_q,
                                 double* __restrict__ d_w) {
  for (int i = threadIdx.x; i < u.nm; i += blockDim.x) { d_p[i] = u.p[i]; d_q[i] = u.q[i]; }
  for (int i = threadIdx.x; i < u.L; i += blockDim.x) d_w[i] = u.w[i];
}

struct NoAllocParams {
  TreeDev t;
  int64_t n, nslots;
  const double *lam, *Q, *En, *dE, *state_in;
  double *state_out, *stress, *tangent;
  int32_t *iters, *status;
  double* slots;  // per-lane scratch, field-major over lanes
  unsigned long long* counter;
  double tol;
  int max_iter;
};

// FP64 Newton kernel of dmn_update, with the orientation normals, the local
// strain, the rotation of the results and the new leaf states computed by the
// lane that owns the point (no per-point buffers).
__global__ void __launch_bounds__(NOALLOC_BLOCK) k_newton_noalloc(NoAllocParams P) {
  const int64_t slot = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int lane = threadIdx.x & 31;
  const TreeDev& t = P.t;
  const int N = t.N;
  double* my_nrm = P.slots + slot;
  PointArrays A{};
  A.nrm = my_nrm; A.ns = (size_t)P.nslots;
  A.nrmf = nullptr;
  A.a = P.slots + (size_t)(3 * N) * P.nslots + slot; A.as = (size_t)P.nslots;
  A.a_out = A.a;
  A.paper = false;
  A.z = nullptr; A.zs = (size_t)P.n;
  GH<double> gh{P.slots + (size_t)(6 * N) * P.nslots + slot, (size_t)P.nslots,
                P.slots + (size_t)(6 * N) * P.nslots + slot};
  const int nzf = 6 * t.nz;
  int64_t pt = -1;
  int it = 0;
  double Eloc[6];
  for (;;) {
    const bool need = pt < 0;
    const unsigned mask = __ballot_sync(0xffffffffu, need);
    if (mask) {
      const int leader = __ffs(mask) - 1;
      unsigned long long base = 0;
      if (lane == leader) base = atomicAdd(P.counter, (unsigned long long)__popc(mask));
      base = __shfl_sync(0xffffffffu, base, leader);
      if (need) {
        pt = (int64_t)(base + __popc(mask & ((1u << lane) - 1u)));
        if (pt < P.n) {
          local_strain(P.Q + 9 * pt, P.En + 6 * pt, P.dE + 6 * pt, Eloc);
          point_normals(t, P.lam[2 * pt], P.lam[2 * pt + 1], my_nrm, A.ns);
          for (int f = 0; f < 3 * N; ++f) {
            const int node = f / 3, c = f - 3 * node;
            const int lvl = 32 - __clz(node + 1);
            const int j = (1 << t.K) - 3 * (1 << (lvl - 1)) + node + 1;
            A.a[(size_t)f * A.as] = P.state_in[(size_t)(nzf + 3 * j + c) * P.n + pt];
          }
          A.z = P.state_in + pt;
          it = 0;
        }
      }
    }
    const bool active = pt >= 0 && pt < P.n;
    if (!__any_sync(0xffffffffu, active)) break;
    if (!active) continue;
    Sub<double> root;
    double r2;
    tree_pass<double, true>(t, Eloc, A, gh, it > 0, 1.0, root, r2, nullptr);
    const double rn = sqrt(r2);
    double sn2 = 0.0;
#pragma unroll
    for (int I = 0; I < 6; ++I) sn2 += root.sb[I] * root.sb[I];
    const double sn = sqrt(sn2);
    int st = -1;
    if (!isfinite(rn) || !isfinite(sn)) st = DMN_STATUS_NONFINITE;
    else if (rn <= P.tol * (double)N * sn) st = DMN_STATUS_OK;
    else if (it >= P.max_iter) st = DMN_STATUS_MAXITER;
    if (st < 0) { ++it; continue; }
    const bool bad = st == DMN_STATUS_NONFINITE;
    const double qnan = __longlong_as_double(0x7ff8000000000000LL);
    for (int f = 0; f < 3 * N; ++f) {
      const int node = f / 3, c = f - 3 * node;
      const int lvl = 32 - __clz(node + 1);
      const int j = (1 << t.K) - 3 * (1 << (lvl - 1)) + node + 1;
      P.state_out[(size_t)(nzf + 3 * j + c) * P.n + pt] = bad ? qnan : A.a[(size_t)f * A.as];
    }
    P.iters[pt] = it;
    P.status[pt] = st;
    if (bad) {
      for (int I = 0; I < 6; ++I) P.stress[6 * pt + I] = qnan;
      for (int I = 0; I < 36; ++I) P.tangent[36 * pt + I] = qnan;
    } else {
      write_stress_tangent<double>(P.Q + 9 * pt, root.sb, root.C, P.stress + 6 * pt, P.tangent + 36 * pt);
    }
    write_leaf_states(t, Eloc, A, P.state_out + pt, (size_t)P.n, bad);
    pt = -1;
  }
}

}  // namespace

extern "C" int dmn_update_noalloc(const dmn_tree_desc* tree, const dmn_options* opt, int64_t n, const double* lam,
                                  const double* Q, const double* E_n, const double* dE, const double* state_in,
                                  double* state_out, double* stress, double* tangent, int32_t* iters,
                                  int32_t* status, void* stream) {
  if (!tree) return fail(nullptr, DMN_ERR_ARG, "dmn_update_noalloc: tree is NULL");
  const dmn_tree_desc& d = *tree;
  if (const char* m = check_tree(d)) return fail(nullptr, DMN_ERR_ARG, std::string("dmn_update_noalloc: ") + m);
  if (n < 0) return fail(nullptr, DMN_ERR_ARG, "dmn_update_noalloc: n < 0");
  const int K = d.K, M = d.M, N = (1 << K) - 1, L = 1 << K;
  double tol = 1e-12;
  int max_iter = 50;
  if (opt) {
    if (opt->precision != DMN_PREC_F64)
      return fail(nullptr, DMN_ERR_ARG, "dmn_update_noalloc: only the FP64 form is available without allocation");
    if (opt->predictor != 0)
      return fail(nullptr, DMN_ERR_ARG, "dmn_update_noalloc: the extrapolated start is not available without allocation");
    if (opt->line_search != 0)
      return fail(nullptr, DMN_ERR_ARG, "dmn_update_noalloc: the line search is not available without allocation");
    if (opt->tol > 0.0) tol = opt->tol;
    if (opt->max_iter > 0) max_iter = opt->max_iter;
  }
  TreeDev td{};
  td.K = K; td.M = M; td.N = N; td.L = L;
  int n_inel = 0;
  for (int f = 0; f < 2; ++f) {
    if (const char* m = make_phase(d.phase[f], td.ph[f]))
      return fail(nullptr, DMN_ERR_ARG, std::string("dmn_update_noalloc: ") + m);
    n_inel += d.phase[f].kind != DMN_PHASE_ELASTIC;
  }
  td.z_both = n_inel == 2;
  td.nz = n_inel * (L / 2);
  // sizes against the fixed work space: parameters, then whole CTAs of lane scratch
  const size_t param_doubles = (size_t)2 * N * M + (size_t)L + 4 * (size_t)N + (size_t)L + (5 * (size_t)N + 1) / 2;
  const size_t lane_bytes = sizeof(double) * (size_t)27 * N;
  const size_t avail = DMN_NOALLOC_BYTES - 256 - sizeof(double) * NOALLOC_PARAM_DOUBLES;
  const int64_t nslots = (int64_t)(avail / lane_bytes) / NOALLOC_BLOCK * NOALLOC_BLOCK;
  if (param_doubles > NOALLOC_PARAM_DOUBLES || nslots < NOALLOC_BLOCK)
    return fail(nullptr, DMN_ERR_ARG, "dmn_update_noalloc: tree too large for the 64 MiB static work space");
  if (n == 0) return DMN_OK;
  if (!lam || !Q || !E_n || !dE || !state_in || !state_out || !stress || !tangent || !iters || !status)
    return fail(nullptr, DMN_ERR_ARG, "dmn_update_noalloc: NULL array");
  if (state_in == state_out) return fail(nullptr, DMN_ERR_ARG, "dmn_update_noalloc: state_in and state_out must differ");

  // device address of the static work space on the current device, looked up on every call
  // (cheap; a reset device may load the module at another address).  The first call on a
  // device also loads the module, which is why it must come before any stream capture.
  void* ptr = nullptr;
  cudaError_t e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
  if (e != cudaSuccess) return cuda_fail(nullptr, e, "dmn_update_noalloc: cudaGetSymbolAddress");
  unsigned char* base = (unsigned char*)ptr;
  unsigned long long* counter = (unsigned long long*)base;
  double* prm = (double*)(base + 256);
  double* d_p = prm;
  double* d_q = d_p + N * M;
  double* d_w = d_q + N * M;
  double* d_c = d_w + L;
  float* d_cf = (float*)(d_c + 4 * N + L);
  double* slots = (double*)(base + 256 + sizeof(double) * NOALLOC_PARAM_DOUBLES);

  // parameters in heap order, handed to the device by value as a kernel argument
  NoAllocUpload up;
  up.nm = N * M;
  up.L = L;
  heap_params(d, up.p, up.q);
  for (int l = 0; l < L; ++l) up.w[l] = d.w[l];
  cudaStream_t s = (cudaStream_t)stream;
  k_noalloc_upload<<<1, 256, 0, s>>>(up, d_p, d_q, d_w);
  k_setup_tree<<<1, 1, 0, s>>>(K, d_w, d_c, d_cf);
  // the counter keeps the previous call's value: clear it
  e = cudaMemsetAsync(counter, 0, sizeof(unsigned long long), s);
  if (e != cudaSuccess) return cuda_fail(nullptr, e, "dmn_update_noalloc: counter reset");
  td.p = d_p; td.q = d_q;
  td.c1 = d_c; td.c2 = d_c + N; td.sc = d_c + 2 * N;
  td.c1f = d_cf; td.c2f = d_cf + N; td.c12f = d_cf + 2 * N; td.scf = d_cf + 3 * N;
  td.wl = d_c + 3 * N;
  td.ic12 = d_c + 3 * N + L; td.ic12f = d_cf + 4 * N;
  td.wsum = 0.0;
  for (int l = 0; l < L; ++l) td.wsum += d.w[l];
  NoAllocParams P{td, n, nslots, lam, Q, E_n, dE, state_in, state_out, stress, tangent, iters, status, slots,
                  counter, tol, max_iter};
  k_newton_noalloc<<<(unsigned)(nslots / NOALLOC_BLOCK), NOALLOC_BLOCK, 0, s>>>(P);
  e = cudaGetLastError();
  return e == cudaSuccess ? DMN_OK : cuda_fail(nullptr, e, "dmn_update_noalloc: launch");
}
