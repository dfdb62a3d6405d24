// Small-strain hexahedral FE operator and Jacobi-PCG (include/fe.h): the
// macroscopic side of an FE-DMN run, whose Gauss points get stress and
// algorithmic tangent from dmn_update (Sec. 5).
//
// Layout.  Per Gauss point the mesh stores the 24 shape-function gradients
// dN_a/dx_i and det(J), field-major ([25][n_gp], coalesced by Gauss point).
// The operator kernels run one thread per Gauss point; the 8 Gauss points of
// an element are 8 consecutive lanes of a warp, so the element sums of B^T s
// are butterfly shuffles inside those 8 lanes, after which lane g writes the
// three entries of node g to an element vector [n_elem][24].  A second kernel
// sums, per node, the entries of its elements in a fixed order (node-to-element
// lists built at mesh creation): no atomics, and results that do not depend on
// scheduling.  Reductions for the CG (dot products) likewise use per-block
// partial sums and one final block in a fixed order.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <string>
#include <vector>

#include "../../include/fe.h"

namespace {

thread_local std::string g_fe_create_error;

constexpr int GF = 25;             // fields per Gauss point: 24 gradients + det(J)
constexpr int TPB = 256;           // threads per block of the operator kernels
constexpr int RED_BLOCKS = 608;    // partial sums per reduction (<= 1024)
constexpr double RS2 = 0.70710678118654752440;  // 1 / sqrt(2)
enum { S_RZ = 0, S_PQ = 1, S_RZN = 2, S_RR = 3, S_BB = 4, S_OUT = 5, N_SCAL = 8 };

}  // namespace

struct fe_mesh {
  int64_t n_nodes = 0, n_elem = 0, n_gp = 0;
  int32_t* conn = nullptr;     // dev [n_elem][8]
  double* G = nullptr;         // dev [25][n_gp]
  int32_t* nptr = nullptr;     // dev [n_nodes + 1]: node-to-element list offsets
  int32_t* nadj = nullptr;     // dev [8 n_elem]: 8 e + a for every element e with node a = that node
  double* fe = nullptr;        // dev [n_elem][24] element vectors
  float* G32 = nullptr;        // dev [25][n_gp]: FP32 copy of G (fe_pcg_f32, made on first use)
  float* C32 = nullptr;        // dev [36][n_gp]: FP32 tangents, field-major (fe_pcg_f32)
  float* fe32 = nullptr;       // dev [n_elem][24] FP32 element vectors (fe_pcg_f32)
  double* part = nullptr;      // dev [2][RED_BLOCKS] partial sums
  double* scal = nullptr;      // dev [N_SCAL] CG scalars
  double* h_scal = nullptr;    // pinned host copy of scal
  double *r = nullptr, *z = nullptr, *p = nullptr, *q = nullptr;  // dev [n_dofs] CG vectors
  double volume = 0.0;
  std::string err;
};

namespace {

int fail(fe_mesh* m, int code, const std::string& msg) {
  if (m) m->err = msg; else g_fe_create_error = msg;
  return code;
}

int cuda_fail(fe_mesh* m, cudaError_t e, const char* what) {
  return fail(m, -2, std::string(what) + ": " + cudaGetErrorString(e));
}

// natural coordinates of the hexahedron's nodes
constexpr int XI[8][3] = {{-1, -1, -1}, {1, -1, -1}, {1, 1, -1}, {-1, 1, -1},
                          {-1, -1, 1},  {1, -1, 1},  {1, 1, 1},  {-1, 1, 1}};

// Gradients dN_a/dx of Gauss point g of an element with node coordinates x [8][3];
// returns det(J) (the integration weight, Gauss weights being 1).
double gauss_point_gradients(const double x[8][3], int g, double grad[8][3]) {
  const double gp = 1.0 / std::sqrt(3.0);
  const double s[3] = {(g & 1) ? gp : -gp, (g & 2) ? gp : -gp, (g & 4) ? gp : -gp};
  double dn[8][3];
  for (int a = 0; a < 8; ++a) {
    const double f[3] = {1.0 + XI[a][0] * s[0], 1.0 + XI[a][1] * s[1], 1.0 + XI[a][2] * s[2]};
    dn[a][0] = 0.125 * XI[a][0] * f[1] * f[2];
    dn[a][1] = 0.125 * XI[a][1] * f[0] * f[2];
    dn[a][2] = 0.125 * XI[a][2] * f[0] * f[1];
  }
  double J[3][3] = {{0}};   // J[i][k] = dx_i / dxi_k
  for (int a = 0; a < 8; ++a)
    for (int i = 0; i < 3; ++i)
      for (int k = 0; k < 3; ++k) J[i][k] += x[a][i] * dn[a][k];
  const double det = J[0][0] * (J[1][1] * J[2][2] - J[1][2] * J[2][1]) -
                     J[0][1] * (J[1][0] * J[2][2] - J[1][2] * J[2][0]) +
                     J[0][2] * (J[1][0] * J[2][1] - J[1][1] * J[2][0]);
  double Ji[3][3];   // inverse: Ji[k][i] = dxi_k / dx_i
  Ji[0][0] = (J[1][1] * J[2][2] - J[1][2] * J[2][1]) / det;
  Ji[0][1] = (J[0][2] * J[2][1] - J[0][1] * J[2][2]) / det;
  Ji[0][2] = (J[0][1] * J[1][2] - J[0][2] * J[1][1]) / det;
  Ji[1][0] = (J[1][2] * J[2][0] - J[1][0] * J[2][2]) / det;
  Ji[1][1] = (J[0][0] * J[2][2] - J[0][2] * J[2][0]) / det;
  Ji[1][2] = (J[0][2] * J[1][0] - J[0][0] * J[1][2]) / det;
  Ji[2][0] = (J[1][0] * J[2][1] - J[1][1] * J[2][0]) / det;
  Ji[2][1] = (J[0][1] * J[2][0] - J[0][0] * J[2][1]) / det;
  Ji[2][2] = (J[0][0] * J[1][1] - J[0][1] * J[1][0]) / det;
  for (int a = 0; a < 8; ++a)
    for (int i = 0; i < 3; ++i)
      grad[a][i] = dn[a][0] * Ji[0][i] + dn[a][1] * Ji[1][i] + dn[a][2] * Ji[2][i];
  return det;
}

// ---------------------------------------------------------------------------
// Operator kernels: one thread per Gauss point.

struct GPView {
  const double* G;
  int64_t n_gp;
};

__device__ __forceinline__ void load_grad(const GPView& V, int64_t gp, double g[8][3], double& w) {
#pragma unroll
  for (int a = 0; a < 8; ++a)
#pragma unroll
    for (int i = 0; i < 3; ++i) g[a][i] = V.G[(size_t)(3 * a + i) * V.n_gp + gp];
  w = V.G[(size_t)24 * V.n_gp + gp];
}

// Mandel strain of the element displacement ue [8][3]
__device__ __forceinline__ void strain_of(const double g[8][3], const double ue[8][3], double eps[6]) {
  double d[3][3] = {{0}};   // d[i][j] = du_i / dx_j
#pragma unroll
  for (int a = 0; a < 8; ++a)
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int j = 0; j < 3; ++j) d[i][j] += ue[a][i] * g[a][j];
  eps[0] = d[0][0];
  eps[1] = d[1][1];
  eps[2] = d[2][2];
  eps[3] = (d[1][2] + d[2][1]) * RS2;
  eps[4] = (d[0][2] + d[2][0]) * RS2;
  eps[5] = (d[0][1] + d[1][0]) * RS2;
}

// ws = w (s11, s22, s33, s23/sqrt2, s13/sqrt2, s12/sqrt2): the weighted stress with the
// Mandel shear factor folded in, so that B^T s w of node a is three 3-term dot products
__device__ __forceinline__ void weighted_stress(const double s[6], double w, double ws[6]) {
  ws[0] = w * s[0]; ws[1] = w * s[1]; ws[2] = w * s[2];
  const double wr = w * RS2;
  ws[3] = wr * s[3]; ws[4] = wr * s[4]; ws[5] = wr * s[5];
}

// w B^T s for node a from the weighted stress ws: three force components
__device__ __forceinline__ void bt_apply(const double ga[3], const double ws[6], double out[3]) {
  out[0] = ga[0] * ws[0] + ga[2] * ws[4] + ga[1] * ws[5];
  out[1] = ga[1] * ws[1] + ga[2] * ws[3] + ga[0] * ws[5];
  out[2] = ga[2] * ws[2] + ga[1] * ws[3] + ga[0] * ws[4];
}

// Sums v over the 8 lanes of this Gauss point's element (all lanes of the warp call it).
__device__ __forceinline__ double elem_sum(double v) {
  v += __shfl_xor_sync(0xffffffffu, v, 1);
  v += __shfl_xor_sync(0xffffffffu, v, 2);
  v += __shfl_xor_sync(0xffffffffu, v, 4);
  return v;
}

// Sums the element vector fe [8][3] over the element's 8 Gauss points (lanes);
// lane g writes the three entries of node g to the element vector out [n_elem][24].
__device__ __forceinline__ void store_element(int64_t e, int g, bool valid, double fe[8][3], double* out) {
  double mine[3] = {0.0, 0.0, 0.0};
#pragma unroll
  for (int a = 0; a < 8; ++a)
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      const double s = elem_sum(fe[a][i]);
      if (a == g) mine[i] = s;
    }
  if (valid) {
#pragma unroll
    for (int i = 0; i < 3; ++i) out[24 * e + 3 * g + i] = mine[i];
  }
}

// f[node] = sum of the element-vector entries of the node, in list order.
__global__ void __launch_bounds__(256) k_gather_nodes(int64_t n_nodes, const int32_t* __restrict__ nptr,
                                                      const int32_t* __restrict__ nadj, const double* __restrict__ fe,
                                                      double* __restrict__ f) {
  const int64_t nd = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (nd >= n_nodes) return;
  double s0 = 0.0, s1 = 0.0, s2 = 0.0;
  for (int k = nptr[nd]; k < nptr[nd + 1]; ++k) {
    const double* x = fe + 3 * (int64_t)nadj[k];   // 24 e + 3 a
    s0 += x[0]; s1 += x[1]; s2 += x[2];
  }
  f[3 * nd] = s0; f[3 * nd + 1] = s1; f[3 * nd + 2] = s2;
}

__device__ __forceinline__ void gather_element(const int32_t* conn, int64_t e, const double* u, double ue[8][3]) {
#pragma unroll
  for (int a = 0; a < 8; ++a) {
    const int64_t node = conn[8 * e + a];
#pragma unroll
    for (int i = 0; i < 3; ++i) ue[a][i] = u[3 * node + i];
  }
}

__global__ void __launch_bounds__(TPB) k_strain(GPView V, const int32_t* __restrict__ conn,
                                                const double* __restrict__ u, double* __restrict__ E) {
  const int64_t gp = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (gp >= V.n_gp) return;
  double g[8][3], w, ue[8][3], eps[6];
  load_grad(V, gp, g, w);
  gather_element(conn, gp >> 3, u, ue);
  strain_of(g, ue, eps);
#pragma unroll
  for (int I = 0; I < 6; ++I) E[6 * gp + I] = eps[I];
}

__global__ void __launch_bounds__(TPB) k_force(GPView V, const double* __restrict__ sig, double* __restrict__ fe_out) {
  const int64_t gp = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const bool valid = gp < V.n_gp;
  double fe[8][3];
  if (valid) {
    double g[8][3], w, s[6], ws[6];
    load_grad(V, gp, g, w);
#pragma unroll
    for (int I = 0; I < 6; ++I) s[I] = sig[6 * gp + I];
    weighted_stress(s, w, ws);
#pragma unroll
    for (int a = 0; a < 8; ++a) bt_apply(g[a], ws, fe[a]);
  } else {
#pragma unroll
    for (int a = 0; a < 8; ++a) fe[a][0] = fe[a][1] = fe[a][2] = 0.0;
  }
  store_element(gp >> 3, (int)(gp & 7), valid, fe, fe_out);
}

__global__ void __launch_bounds__(TPB) k_apply(GPView V, const int32_t* __restrict__ conn,
                                               const double* __restrict__ C, const double* __restrict__ v,
                                               double* __restrict__ fe_out) {
  const int64_t gp = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const bool valid = gp < V.n_gp;
  double fe[8][3];
  if (valid) {
    double g[8][3], w, ve[8][3], eps[6], tau[6];
    load_grad(V, gp, g, w);
    gather_element(conn, gp >> 3, v, ve);
    strain_of(g, ve, eps);
    const double* c = C + 36 * gp;
#pragma unroll
    for (int I = 0; I < 6; ++I) {
      double t = 0.0;
#pragma unroll
      for (int J = 0; J < 6; ++J) t += c[6 * I + J] * eps[J];
      tau[I] = t;
    }
    double ws[6];
    weighted_stress(tau, w, ws);
#pragma unroll
    for (int a = 0; a < 8; ++a) bt_apply(g[a], ws, fe[a]);
  } else {
#pragma unroll
    for (int a = 0; a < 8; ++a) fe[a][0] = fe[a][1] = fe[a][2] = 0.0;
  }
  store_element(gp >> 3, (int)(gp & 7), valid, fe, fe_out);
}

// b_{a,i}^T C b_{a,i} w for every dof of the element, with b_{a,i} the Mandel strain of a unit
// displacement of dof (a, i)
__global__ void __launch_bounds__(TPB) k_diag(GPView V, const double* __restrict__ C, double* __restrict__ fe_out) {
  const int64_t gp = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const bool valid = gp < V.n_gp;
  double fe[8][3];
  if (valid) {
    double g[8][3], w;
    load_grad(V, gp, g, w);
    double c[36];
#pragma unroll
    for (int k = 0; k < 36; ++k) c[k] = C[36 * gp + k];
#pragma unroll
    for (int a = 0; a < 8; ++a)
#pragma unroll
      for (int i = 0; i < 3; ++i) {
        double b[6] = {0, 0, 0, 0, 0, 0};
        b[i] = g[a][i];
        if (i == 0) { b[4] = g[a][2] * RS2; b[5] = g[a][1] * RS2; }
        if (i == 1) { b[3] = g[a][2] * RS2; b[5] = g[a][0] * RS2; }
        if (i == 2) { b[3] = g[a][1] * RS2; b[4] = g[a][0] * RS2; }
        double s = 0.0;
#pragma unroll
        for (int I = 0; I < 6; ++I) {
          double t = 0.0;
#pragma unroll
          for (int J = 0; J < 6; ++J) t += c[6 * I + J] * b[J];
          s += b[I] * t;
        }
        fe[a][i] = w * s;
      }
  } else {
#pragma unroll
    for (int a = 0; a < 8; ++a) fe[a][0] = fe[a][1] = fe[a][2] = 0.0;
  }
  store_element(gp >> 3, (int)(gp & 7), valid, fe, fe_out);
}

// ---------------------------------------------------------------------------
// FP32 operator (fe_pcg_f32): the same products in single precision, from field-major
// FP32 copies of G and C; element sums in FP32, node sums in FP64.

__global__ void __launch_bounds__(256) k_to_f32(int64_t n, const double* __restrict__ a, float* __restrict__ b) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    b[i] = (float)a[i];
}

// C [n_gp][36] (FP64, point-major) -> C32 [36][n_gp] (FP32, field-major)
__global__ void __launch_bounds__(256) k_pack_c(int64_t n_gp, const double* __restrict__ C, float* __restrict__ C32) {
  const int64_t gp = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (gp >= n_gp) return;
#pragma unroll
  for (int k = 0; k < 36; ++k) C32[(size_t)k * n_gp + gp] = (float)C[36 * gp + k];
}

__device__ __forceinline__ float elem_sum_f(float v) {
  v += __shfl_xor_sync(0xffffffffu, v, 1);
  v += __shfl_xor_sync(0xffffffffu, v, 2);
  v += __shfl_xor_sync(0xffffffffu, v, 4);
  return v;
}

__global__ void __launch_bounds__(TPB) k_apply32(int64_t n_gp, const float* __restrict__ G32,
                                                 const int32_t* __restrict__ conn, const float* __restrict__ C32,
                                                 const double* __restrict__ v, float* __restrict__ fe_out) {
  const int64_t gp = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const bool valid = gp < n_gp;
  const float rs2 = 0.70710678f;
  float fe[8][3];
  if (valid) {
    float g[8][3];
#pragma unroll
    for (int a = 0; a < 8; ++a)
#pragma unroll
      for (int i = 0; i < 3; ++i) g[a][i] = G32[(size_t)(3 * a + i) * n_gp + gp];
    const float w = G32[(size_t)24 * n_gp + gp];
    float d[3][3] = {{0.f, 0.f, 0.f}, {0.f, 0.f, 0.f}, {0.f, 0.f, 0.f}};
    const int64_t e = gp >> 3;
#pragma unroll
    for (int a = 0; a < 8; ++a) {
      const int64_t node = conn[8 * e + a];
#pragma unroll
      for (int i = 0; i < 3; ++i) {
        const float ui = (float)v[3 * node + i];
#pragma unroll
        for (int j = 0; j < 3; ++j) d[i][j] += ui * g[a][j];
      }
    }
    const float eps[6] = {d[0][0], d[1][1], d[2][2], (d[1][2] + d[2][1]) * rs2, (d[0][2] + d[2][0]) * rs2,
                          (d[0][1] + d[1][0]) * rs2};
    float ws[6];
#pragma unroll
    for (int I = 0; I < 6; ++I) {
      float t = 0.f;
#pragma unroll
      for (int J = 0; J < 6; ++J) t += C32[(size_t)(6 * I + J) * n_gp + gp] * eps[J];
      ws[I] = (I < 3 ? w : w * rs2) * t;
    }
#pragma unroll
    for (int a = 0; a < 8; ++a) {
      fe[a][0] = g[a][0] * ws[0] + g[a][2] * ws[4] + g[a][1] * ws[5];
      fe[a][1] = g[a][1] * ws[1] + g[a][2] * ws[3] + g[a][0] * ws[5];
      fe[a][2] = g[a][2] * ws[2] + g[a][1] * ws[3] + g[a][0] * ws[4];
    }
  } else {
#pragma unroll
    for (int a = 0; a < 8; ++a) fe[a][0] = fe[a][1] = fe[a][2] = 0.f;
  }
  const int gl = (int)(gp & 7);
  float mine[3] = {0.f, 0.f, 0.f};
#pragma unroll
  for (int a = 0; a < 8; ++a)
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      const float sm = elem_sum_f(fe[a][i]);
      if (a == gl) mine[i] = sm;
    }
  if (valid) {
#pragma unroll
    for (int i = 0; i < 3; ++i) fe_out[24 * (gp >> 3) + 3 * gl + i] = mine[i];
  }
}

__global__ void __launch_bounds__(256) k_gather_nodes32(int64_t n_nodes, const int32_t* __restrict__ nptr,
                                                        const int32_t* __restrict__ nadj, const float* __restrict__ fe,
                                                        double* __restrict__ f) {
  const int64_t nd = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (nd >= n_nodes) return;
  double s0 = 0.0, s1 = 0.0, s2 = 0.0;
  for (int k = nptr[nd]; k < nptr[nd + 1]; ++k) {
    const float* x = fe + 3 * (int64_t)nadj[k];
    s0 += (double)x[0]; s1 += (double)x[1]; s2 += (double)x[2];
  }
  f[3 * nd] = s0; f[3 * nd + 1] = s1; f[3 * nd + 2] = s2;
}

// ---------------------------------------------------------------------------
// Vector kernels and reductions (grid RED_BLOCKS x TPB, grid-stride).

__device__ __forceinline__ double block_sum(double v, double* sh) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
  __syncthreads();
  if (lane == 0) sh[wid] = v;
  __syncthreads();
  v = (threadIdx.x < (blockDim.x >> 5)) ? sh[threadIdx.x] : 0.0;
  if (wid == 0)
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// part[block] = sum of w a b over this block's stride (w may be NULL)
__global__ void __launch_bounds__(TPB) k_dot_part(int64_t n, const double* __restrict__ a,
                                                  const double* __restrict__ b, const double* __restrict__ w,
                                                  double* __restrict__ part) {
  __shared__ double sh[TPB / 32];
  double s = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)TPB + threadIdx.x; i < n; i += (int64_t)gridDim.x * TPB)
    s += (w ? w[i] : 1.0) * a[i] * b[i];
  s = block_sum(s, sh);
  if (threadIdx.x == 0) part[blockIdx.x] = s;
}

// out[k] = sum of part[k * nb .. k * nb + nb - 1] for k < nk, in a fixed order (one block of 1024);
// with rotate, scal[S_RZ] takes scal[S_RZN] first (the CG's r.z of the previous iteration)
__global__ void k_reduce(const double* __restrict__ part, int nb, int nk, double* scal, int slot0, int rotate) {
  __shared__ double sh[32];
  if (rotate && threadIdx.x == 0) scal[S_RZ] = scal[S_RZN];
  for (int k = 0; k < nk; ++k) {
    double v = (threadIdx.x < nb) ? part[k * nb + threadIdx.x] : 0.0;
    v = block_sum(v, sh);
    if (threadIdx.x == 0) scal[slot0 + k] = v;
    __syncthreads();
  }
}

__global__ void __launch_bounds__(TPB) k_axpy(int64_t n, double alpha, const double* __restrict__ x,
                                              const double* __restrict__ w, double* __restrict__ y) {
  for (int64_t i = blockIdx.x * (int64_t)TPB + threadIdx.x; i < n; i += (int64_t)gridDim.x * TPB)
    y[i] += alpha * (w ? w[i] : 1.0) * x[i];
}

// CG start: r = free b, x = 0, z = r / diag, p = z; partials of r.z and r.r
__global__ void __launch_bounds__(TPB) k_pcg_init(int64_t n, const double* __restrict__ fr,
                                                  const double* __restrict__ diag, const double* __restrict__ b,
                                                  double* __restrict__ x, double* __restrict__ r,
                                                  double* __restrict__ z, double* __restrict__ p,
                                                  double* __restrict__ part) {
  __shared__ double sh[TPB / 32];
  double rz = 0.0, rr = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)TPB + threadIdx.x; i < n; i += (int64_t)gridDim.x * TPB) {
    const double ri = fr[i] * b[i];
    const double zi = (fr[i] != 0.0 && diag[i] > 0.0) ? ri / diag[i] : 0.0;
    x[i] = 0.0; r[i] = ri; z[i] = zi; p[i] = zi;
    rz += ri * zi; rr += ri * ri;
  }
  rz = block_sum(rz, sh);
  __syncthreads();
  rr = block_sum(rr, sh);
  if (threadIdx.x == 0) { part[blockIdx.x] = rz; part[gridDim.x + blockIdx.x] = rr; }
}

// x += alpha p, r -= alpha free q, z = r / diag with alpha = r.z / p.q; partials of r.z, r.r
__global__ void __launch_bounds__(TPB) k_pcg_update(int64_t n, const double* __restrict__ fr,
                                                    const double* __restrict__ diag, const double* __restrict__ scal,
                                                    const double* __restrict__ p, const double* __restrict__ q,
                                                    double* __restrict__ x, double* __restrict__ r,
                                                    double* __restrict__ z, double* __restrict__ part) {
  __shared__ double sh[TPB / 32];
  const double pq = scal[S_PQ];
  const double alpha = pq > 0.0 ? scal[S_RZ] / pq : 0.0;
  double rz = 0.0, rr = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)TPB + threadIdx.x; i < n; i += (int64_t)gridDim.x * TPB) {
    x[i] += alpha * p[i];
    const double ri = r[i] - alpha * fr[i] * q[i];
    const double zi = (fr[i] != 0.0 && diag[i] > 0.0) ? ri / diag[i] : 0.0;
    r[i] = ri; z[i] = zi;
    rz += ri * zi; rr += ri * ri;
  }
  rz = block_sum(rz, sh);
  __syncthreads();
  rr = block_sum(rr, sh);
  if (threadIdx.x == 0) { part[blockIdx.x] = rz; part[gridDim.x + blockIdx.x] = rr; }
}

// p = z + beta p, beta = r.z (new) / r.z (old)
__global__ void __launch_bounds__(TPB) k_pcg_dir(int64_t n, const double* __restrict__ scal,
                                                 const double* __restrict__ z, double* __restrict__ p) {
  const double rz = scal[S_RZ];
  const double beta = rz > 0.0 ? scal[S_RZN] / rz : 0.0;
  for (int64_t i = blockIdx.x * (int64_t)TPB + threadIdx.x; i < n; i += (int64_t)gridDim.x * TPB)
    p[i] = z[i] + beta * p[i];
}

unsigned op_grid(const fe_mesh* m) { return (unsigned)((m->n_gp + TPB - 1) / TPB); }
unsigned node_grid(const fe_mesh* m) { return (unsigned)((m->n_nodes + 255) / 256); }

GPView view(const fe_mesh* m) { return GPView{m->G, m->n_gp}; }

}  // namespace

namespace {

// Jacobi-PCG on the free dofs (fe_pcg, fe_pcg_f32).  f32: the products K p in FP32.
int pcg_run(fe_mesh* m, bool f32, const char* who, const double* C, const double* free, const double* diag,
            const double* b, double* x, double rtol, int32_t max_iter, int32_t* iters, double* rel_res,
            void* stream) {
  if (!m) return fail(nullptr, -1, std::string(who) + ": NULL mesh");
  if (!C || !free || !diag || !b || !x) return fail(m, -1, std::string(who) + ": NULL array");
  if (!(rtol > 0.0) || max_iter < 1) return fail(m, -1, std::string(who) + ": need rtol > 0 and max_iter >= 1");
  cudaStream_t s = (cudaStream_t)stream;
  const int64_t n = 3 * m->n_nodes;
  cudaError_t e = cudaSuccess;
  if (f32) {
    if (!m->G32) {
      e = cudaMalloc(&m->G32, sizeof(float) * GF * m->n_gp);
      if (e == cudaSuccess) e = cudaMalloc(&m->C32, sizeof(float) * 36 * m->n_gp);
      if (e == cudaSuccess) e = cudaMalloc(&m->fe32, sizeof(float) * 24 * m->n_elem);
      if (e == cudaSuccess) {
        k_to_f32<<<RED_BLOCKS, 256, 0, s>>>((int64_t)GF * m->n_gp, m->G, m->G32);
        e = cudaGetLastError();
      }
      if (e != cudaSuccess) {
        cudaFree(m->G32); cudaFree(m->C32); cudaFree(m->fe32);
        m->G32 = nullptr; m->C32 = nullptr; m->fe32 = nullptr;
        return cuda_fail(m, e, who);
      }
    }
    k_pack_c<<<(unsigned)((m->n_gp + 255) / 256), 256, 0, s>>>(m->n_gp, C, m->C32);
  }
  const int CHECK = 8;   // iterations between convergence checks on the host
  k_pcg_init<<<RED_BLOCKS, TPB, 0, s>>>(n, free, diag, b, x, m->r, m->z, m->p, m->part);
  k_reduce<<<1, 1024, 0, s>>>(m->part, RED_BLOCKS, 2, m->scal, S_RZN, 0);   // r.z -> RZN, r.r -> RR
  e = cudaMemcpyAsync(m->h_scal, m->scal, sizeof(double) * N_SCAL, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_fail(m, e, who);
  const double bnorm = std::sqrt(m->h_scal[S_RR]);
  int it = 0;
  double res = 0.0;
  if (bnorm > 0.0) {
    res = 1.0;
    while (it < max_iter) {
      const int todo = std::min(CHECK, max_iter - it);
      for (int k = 0; k < todo; ++k) {
        if (f32) {
          k_apply32<<<op_grid(m), TPB, 0, s>>>(m->n_gp, m->G32, m->conn, m->C32, m->p, m->fe32);
          k_gather_nodes32<<<node_grid(m), 256, 0, s>>>(m->n_nodes, m->nptr, m->nadj, m->fe32, m->q);
        } else {
          k_apply<<<op_grid(m), TPB, 0, s>>>(view(m), m->conn, C, m->p, m->fe);
          k_gather_nodes<<<node_grid(m), 256, 0, s>>>(m->n_nodes, m->nptr, m->nadj, m->fe, m->q);
        }
        k_dot_part<<<RED_BLOCKS, TPB, 0, s>>>(n, m->p, m->q, free, m->part);
        k_reduce<<<1, 1024, 0, s>>>(m->part, RED_BLOCKS, 1, m->scal, S_PQ, 1);
        k_pcg_update<<<RED_BLOCKS, TPB, 0, s>>>(n, free, diag, m->scal, m->p, m->q, x, m->r, m->z, m->part);
        k_reduce<<<1, 1024, 0, s>>>(m->part, RED_BLOCKS, 2, m->scal, S_RZN, 0);
        k_pcg_dir<<<RED_BLOCKS, TPB, 0, s>>>(n, m->scal, m->z, m->p);
      }
      it += todo;
      e = cudaGetLastError();
      if (e == cudaSuccess) e = cudaMemcpyAsync(m->h_scal, m->scal, sizeof(double) * N_SCAL, cudaMemcpyDeviceToHost, s);
      if (e == cudaSuccess) e = cudaStreamSynchronize(s);
      if (e != cudaSuccess) return cuda_fail(m, e, who);
      res = std::sqrt(std::max(m->h_scal[S_RR], 0.0)) / bnorm;
      if (!(res > rtol)) break;   // converged (or NaN: stop and report it)
    }
  } else {
    e = cudaMemsetAsync(x, 0, sizeof(double) * n, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(m, e, who);
  }
  if (iters) *iters = it;
  if (rel_res) *rel_res = res;
  return 0;
}

}  // namespace

extern "C" {

int fe_mesh_create(int64_t n_nodes, int64_t n_elem, const double* xyz, const int32_t* conn, fe_mesh** out) {
  if (!out) return fail(nullptr, -1, "fe_mesh_create: out is NULL");
  *out = nullptr;
  g_fe_create_error.clear();
  if (n_nodes < 8 || n_elem < 1 || !xyz || !conn)
    return fail(nullptr, -1, "fe_mesh_create: need n_nodes >= 8, n_elem >= 1 and non-NULL arrays");
  if (n_nodes > (int64_t)1 << 31 || n_elem > ((int64_t)1 << 31) / 8)
    return fail(nullptr, -1, "fe_mesh_create: mesh too large for 32-bit node and Gauss-point indices");
  const int64_t n_gp = 8 * n_elem;
  std::vector<double> G((size_t)GF * n_gp);
  double vol = 0.0;
  for (int64_t e = 0; e < n_elem; ++e) {
    double x[8][3];
    for (int a = 0; a < 8; ++a) {
      const int32_t nd = conn[8 * e + a];
      if (nd < 0 || nd >= n_nodes) return fail(nullptr, -1, "fe_mesh_create: node index out of range");
      for (int i = 0; i < 3; ++i) x[a][i] = xyz[3 * (int64_t)nd + i];
    }
    for (int g = 0; g < 8; ++g) {
      double grad[8][3];
      const double det = gauss_point_gradients(x, g, grad);
      if (!(det > 0.0)) {
        char msg[160];
        std::snprintf(msg, sizeof msg, "fe_mesh_create: element %lld has det(J) = %g <= 0 at Gauss point %d",
                      (long long)e, det, g);
        return fail(nullptr, -1, msg);
      }
      const int64_t gp = 8 * e + g;
      for (int a = 0; a < 8; ++a)
        for (int i = 0; i < 3; ++i) G[(size_t)(3 * a + i) * n_gp + gp] = grad[a][i];
      G[(size_t)24 * n_gp + gp] = det;
      vol += det;
    }
  }
  // node-to-element lists (counting sort of the connectivity), entries 8 e + a in element order
  std::vector<int32_t> nptr(n_nodes + 1, 0), nadj((size_t)8 * n_elem);
  for (int64_t k = 0; k < 8 * n_elem; ++k) ++nptr[conn[k] + 1];
  for (int64_t nd = 0; nd < n_nodes; ++nd) nptr[nd + 1] += nptr[nd];
  {
    std::vector<int32_t> cur(nptr.begin(), nptr.end() - 1);
    for (int64_t k = 0; k < 8 * n_elem; ++k) nadj[cur[conn[k]]++] = (int32_t)k;
  }
  fe_mesh* m = new fe_mesh();
  m->n_nodes = n_nodes; m->n_elem = n_elem; m->n_gp = n_gp; m->volume = vol;
  const size_t nd = (size_t)3 * n_nodes;
  cudaError_t e = cudaMalloc(&m->conn, sizeof(int32_t) * 8 * n_elem);
  if (e == cudaSuccess) e = cudaMalloc(&m->G, sizeof(double) * G.size());
  if (e == cudaSuccess) e = cudaMalloc(&m->nptr, sizeof(int32_t) * nptr.size());
  if (e == cudaSuccess) e = cudaMalloc(&m->nadj, sizeof(int32_t) * nadj.size());
  if (e == cudaSuccess) e = cudaMalloc(&m->fe, sizeof(double) * 24 * n_elem);
  if (e == cudaSuccess) e = cudaMalloc(&m->part, sizeof(double) * 2 * RED_BLOCKS);
  if (e == cudaSuccess) e = cudaMalloc(&m->scal, sizeof(double) * N_SCAL);
  if (e == cudaSuccess) e = cudaHostAlloc(&m->h_scal, sizeof(double) * N_SCAL, cudaHostAllocDefault);
  for (double** v : {&m->r, &m->z, &m->p, &m->q})
    if (e == cudaSuccess) e = cudaMalloc(v, sizeof(double) * nd);
  if (e == cudaSuccess) e = cudaMemcpy(m->conn, conn, sizeof(int32_t) * 8 * n_elem, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(m->G, G.data(), sizeof(double) * G.size(), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(m->nptr, nptr.data(), sizeof(int32_t) * nptr.size(), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(m->nadj, nadj.data(), sizeof(int32_t) * nadj.size(), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemset(m->scal, 0, sizeof(double) * N_SCAL);
  if (e != cudaSuccess) {
    fe_mesh_destroy(m);
    return cuda_fail(nullptr, e, "fe_mesh_create");
  }
  *out = m;
  return 0;
}

void fe_mesh_destroy(fe_mesh* m) {
  if (!m) return;
  cudaDeviceSynchronize();
  cudaFree(m->conn); cudaFree(m->G); cudaFree(m->part); cudaFree(m->scal);
  cudaFree(m->nptr); cudaFree(m->nadj); cudaFree(m->fe);
  cudaFree(m->G32); cudaFree(m->C32); cudaFree(m->fe32);
  cudaFree(m->r); cudaFree(m->z); cudaFree(m->p); cudaFree(m->q);
  if (m->h_scal) cudaFreeHost(m->h_scal);
  delete m;
}

int64_t fe_num_gauss_points(const fe_mesh* m) { return m ? m->n_gp : -1; }
int64_t fe_num_dofs(const fe_mesh* m) { return m ? 3 * m->n_nodes : -1; }
double fe_volume(const fe_mesh* m) { return m ? m->volume : 0.0; }

const char* fe_last_error(const fe_mesh* m) { return m ? m->err.c_str() : g_fe_create_error.c_str(); }

int fe_strain(fe_mesh* m, const double* u, double* E, void* stream) {
  if (!m) return fail(nullptr, -1, "fe_strain: NULL mesh");
  if (!u || !E) return fail(m, -1, "fe_strain: NULL array");
  k_strain<<<op_grid(m), TPB, 0, (cudaStream_t)stream>>>(view(m), m->conn, u, E);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? 0 : cuda_fail(m, e, "fe_strain");
}

int fe_internal_force(fe_mesh* m, const double* sigma, double* f, void* stream) {
  if (!m) return fail(nullptr, -1, "fe_internal_force: NULL mesh");
  if (!sigma || !f) return fail(m, -1, "fe_internal_force: NULL array");
  cudaStream_t s = (cudaStream_t)stream;
  k_force<<<op_grid(m), TPB, 0, s>>>(view(m), sigma, m->fe);
  k_gather_nodes<<<node_grid(m), 256, 0, s>>>(m->n_nodes, m->nptr, m->nadj, m->fe, f);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? 0 : cuda_fail(m, e, "fe_internal_force");
}

int fe_apply_tangent(fe_mesh* m, const double* C, const double* v, double* Kv, void* stream) {
  if (!m) return fail(nullptr, -1, "fe_apply_tangent: NULL mesh");
  if (!C || !v || !Kv) return fail(m, -1, "fe_apply_tangent: NULL array");
  if (v == Kv) return fail(m, -1, "fe_apply_tangent: v and Kv must differ");
  cudaStream_t s = (cudaStream_t)stream;
  k_apply<<<op_grid(m), TPB, 0, s>>>(view(m), m->conn, C, v, m->fe);
  k_gather_nodes<<<node_grid(m), 256, 0, s>>>(m->n_nodes, m->nptr, m->nadj, m->fe, Kv);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? 0 : cuda_fail(m, e, "fe_apply_tangent");
}

int fe_tangent_diagonal(fe_mesh* m, const double* C, double* diag, void* stream) {
  if (!m) return fail(nullptr, -1, "fe_tangent_diagonal: NULL mesh");
  if (!C || !diag) return fail(m, -1, "fe_tangent_diagonal: NULL array");
  cudaStream_t s = (cudaStream_t)stream;
  k_diag<<<op_grid(m), TPB, 0, s>>>(view(m), C, m->fe);
  k_gather_nodes<<<node_grid(m), 256, 0, s>>>(m->n_nodes, m->nptr, m->nadj, m->fe, diag);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? 0 : cuda_fail(m, e, "fe_tangent_diagonal");
}

int fe_dot(fe_mesh* m, const double* a, const double* b, const double* free, double* out, void* stream) {
  if (!m) return fail(nullptr, -1, "fe_dot: NULL mesh");
  if (!a || !b || !out) return fail(m, -1, "fe_dot: NULL array");
  cudaStream_t s = (cudaStream_t)stream;
  const int64_t n = 3 * m->n_nodes;
  k_dot_part<<<RED_BLOCKS, TPB, 0, s>>>(n, a, b, free, m->part);
  k_reduce<<<1, 1024, 0, s>>>(m->part, RED_BLOCKS, 1, m->scal, S_OUT, 0);
  cudaError_t e = cudaMemcpyAsync(m->h_scal + S_OUT, m->scal + S_OUT, sizeof(double), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_fail(m, e, "fe_dot");
  *out = m->h_scal[S_OUT];
  return 0;
}

int fe_axpy(fe_mesh* m, double alpha, const double* x, const double* free, double* y, void* stream) {
  if (!m) return fail(nullptr, -1, "fe_axpy: NULL mesh");
  if (!x || !y) return fail(m, -1, "fe_axpy: NULL array");
  k_axpy<<<RED_BLOCKS, TPB, 0, (cudaStream_t)stream>>>(3 * m->n_nodes, alpha, x, free, y);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? 0 : cuda_fail(m, e, "fe_axpy");
}

int fe_pcg(fe_mesh* m, const double* C, const double* free, const double* diag, const double* b, double* x,
           double rtol, int32_t max_iter, int32_t* iters, double* rel_res, void* stream) {
  return pcg_run(m, false, "fe_pcg", C, free, diag, b, x, rtol, max_iter, iters, rel_res, stream);
}

int fe_pcg_f32(fe_mesh* m, const double* C, const double* free, const double* diag, const double* b, double* x,
               double rtol, int32_t max_iter, int32_t* iters, double* rel_res, void* stream) {
  return pcg_run(m, true, "fe_pcg_f32", C, free, diag, b, x, rtol, max_iter, iters, rel_res, stream);
}

}  // extern "C"
