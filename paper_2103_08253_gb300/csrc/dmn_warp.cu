// The warp organisation of the Newton iteration (small calls): k_newton_warp and its launch.  The
// per-laminate arithmetic is that of csrc/dmn_device.cuh, shared with the thread-per-point kernels
// of csrc/dmn.cu; its own translation unit so that the two compile in parallel.
#include <cuda_runtime.h>

#include "../../include/dmn.h"
#include "dmn_device.cuh"
#include "dmn_launch.cuh"

namespace dmn {

template <typename T, bool LS, int G, bool CMP>
__global__ void __launch_bounds__(128) k_newton_warp(NewtonParams<T> P, double* scratch) {
  static_assert(G == 8 || G == 16 || G == 32, "8, 16 or 32 lanes per point");
  const int64_t grp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) / G;
  const int lane = threadIdx.x % G;
  const unsigned gmask = G == 32 ? 0xffffffffu : ((1u << G) - 1u) << ((threadIdx.x & 31) / G * G);
  const int NM = P.N_max;
  double* base = scratch + (size_t)grp * warp_slot_doubles<T>(NM);
  double* abuf[2] = {base, base + 3 * NM};
  double* ein = base + 6 * NM;
  double* sbv = base + 12 * NM;
  double* nrm = base + 18 * NM;
  double* le = base + 21 * NM;
  T* tb = reinterpret_cast<T*>(base + 27 * NM);
  T* gbuf[2] = {tb, tb + 21 * NM};
  T* dein = tb + 42 * NM;
  T* dcv = tb + 48 * NM;
  float* nrmf = reinterpret_cast<float*>(tb + 75 * NM);
  PointArrays A{};
  A.nrm = nrm; A.ns = 1; A.nrmf = nrmf;
  A.as = 1; A.paper = false;
  A.zs = (size_t)P.n;
  const double qnan = __longlong_as_double(0x7ff8000000000000LL);
  unsigned long long npass = 0;
  // the group's point and its Newton state
  int64_t pt = -1;
  int tr = 0, it0 = 0, it = 0, cur = 0, halvings = 0;
  bool first = true;
  T step = (T)1;
  double rn_acc = 0.0, Eloc[6];
  Sub<T> root, root_acc;
  // the next point of a known tree for this group (points of unknown trees are reported on the
  // way); false once the counter is exhausted
  auto take = [&]() -> bool {
    for (;;) {
      unsigned long long i = 0;
      if (lane == 0) i = atomicAdd(P.counter, 1ull);
      i = __shfl_sync(gmask, i, 0, G);
      if (i >= (unsigned long long)P.n) return false;
      point_of(P.perm, P.tid, P.F.n, (int64_t)i, pt, tr);
      if (tr < P.F.n) break;
      if (lane == 0) {   // unknown tree: report and take the next point
        P.iters[pt] = 0;
        P.status[pt] = DMN_STATUS_BAD_TREE;
        for (int I = 0; I < 6; ++I) P.stress[6 * pt + I] = qnan;
        for (int I = 0; I < 36; ++I) P.tangent[36 * pt + I] = qnan;
      }
    }
    const TreeDev& t = P.F.t[tr];
    const int nzf = 6 * t.nz;
#pragma unroll
    for (int I = 0; I < 6; ++I) Eloc[I] = P.nbuf[(size_t)(3 * NM + I) * P.n + pt];
    for (int f = lane; f < 3 * t.N; f += G) {   // jumps: heap order here, paper order in the state
      const int node = f / 3, c = f - 3 * node;
      const int lvl = 32 - __clz(node + 1);
      const int j = CMP ? node : (1 << t.K) - 3 * (1 << (lvl - 1)) + node + 1;
      abuf[0][f] = (P.a_start ? P.a_start : P.state_in)[(size_t)(nzf + 3 * j + c) * P.n + pt];
      const double nv = P.nbuf[(size_t)f * P.n + pt];
      nrm[f] = nv;
      if (sizeof(T) == 4) nrmf[f] = narrow_rn(nv);
    }
    it0 = P.a_start ? P.iters[pt] : 0;
    it = 0; cur = 0; halvings = 0; first = true; step = (T)1; rn_acc = 0.0;
    __syncwarp(gmask);
    return true;
  };
  bool have = take();
  while (__any_sync(0xffffffffu, have)) {
    if (!have) continue;
    const TreeDev& t = P.F.t[tr];
    A.z = P.state_in + pt;
    WarpSlot<T> W{abuf[cur], abuf[LS ? 1 - cur : cur], gbuf[cur], gbuf[LS ? 1 - cur : cur], ein, dein, sbv, dcv, NM,
                  le};
    ++npass;
    double r2 = warp_tree_pass<T, CMP>(t, Eloc, A, W, !first, step, lane, G, gmask);
#pragma unroll
    for (int o = G / 2; o > 0; o >>= 1) r2 += __shfl_xor_sync(gmask, r2, o, G);
    warp_sub_load<T>(W, CMP ? t.N - 1 : 0, root);
    __syncwarp(gmask);
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
      else if (it >= P.max_iter - it0) st = DMN_STATUS_MAXITER;
      if (st < 0) { ++it; continue; }
    } else {
      const bool accepted = first || rn < rn_acc;
      if (accepted) {
        first = false;
        cur = 1 - cur;
        rn_acc = rn;
        root_acc = root;
        step = (T)1;
        halvings = 0;
        if (!isfinite(rn) || !isfinite(sn)) st = DMN_STATUS_NONFINITE;
        else if (rn <= P.tol * (double)t.N * sn && it >= P.min_corr) st = DMN_STATUS_OK;
        else if (it >= P.max_iter - it0) st = DMN_STATUS_MAXITER;
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
    // finished point: jumps (paper ordering), counters, and without a final sweep the local-frame
    // stress and packed tangent for k_final to rotate
    const int nzf = 6 * t.nz;
    const double* afin = abuf[cur];
    for (int f = lane; f < 3 * t.N; f += G) {
      const int node = f / 3, c = f - 3 * node;
      const int lvl = 32 - __clz(node + 1);
      const int j = CMP ? node : (1 << t.K) - 3 * (1 << (lvl - 1)) + node + 1;
      P.state_out[(size_t)(nzf + 3 * j + c) * P.n + pt] = st == DMN_STATUS_NONFINITE ? qnan : afin[f];
    }
    if (lane == 0) {
      P.iters[pt] = it + it0;
      P.status[pt] = st;
      if (P.write_outputs) {
        for (int I = 0; I < 6; ++I) P.stress[6 * pt + I] = root.sb[I];
        for (int k = 0; k < 21; ++k) P.tangent[36 * pt + k] = widen(root.C[k]);
      }
    }
    __syncwarp(gmask);
    have = take();
  }
  if (lane == 0 && P.passes && npass) atomicAdd(P.passes, npass);
}

template <typename T, bool CMP>
void launch_warp(const NewtonParams<T>& P, bool ls, int lanes, unsigned grid, double* scr, cudaStream_t s) {
  if (lanes == 8) {
    if (ls) k_newton_warp<T, true, 8, CMP><<<grid, 128, 0, s>>>(P, scr);
    else k_newton_warp<T, false, 8, CMP><<<grid, 128, 0, s>>>(P, scr);
  } else if (lanes == 16) {
    if (ls) k_newton_warp<T, true, 16, CMP><<<grid, 128, 0, s>>>(P, scr);
    else k_newton_warp<T, false, 16, CMP><<<grid, 128, 0, s>>>(P, scr);
  } else {
    if (ls) k_newton_warp<T, true, 32, CMP><<<grid, 128, 0, s>>>(P, scr);
    else k_newton_warp<T, false, 32, CMP><<<grid, 128, 0, s>>>(P, scr);
  }
}

// The mixed form's FP64 final sweep in the warp organisation: one FP64 pass per point at its converged
// jumps (state_out), no correction applied, the root's stress and packed tangent (local frame) written
// for k_final<false> to rotate; that kernel then writes the leaf states.  Points whose Newton iteration
// was not finite, or whose tree is unknown, are left to k_final and to the Newton kernel's report.  The
// groups run side by side as in k_newton_warp; the scratch slots are sized for FP64.
template <bool CMP, int G>
__global__ void __launch_bounds__(128) k_sweep_warp(NewtonParams<double> P, double* scratch) {
  const int64_t grp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) / G;
  const int lane = threadIdx.x % G;
  const unsigned gmask = G == 32 ? 0xffffffffu : ((1u << G) - 1u) << ((threadIdx.x & 31) / G * G);
  const int NM = P.N_max;
  double* base = scratch + (size_t)grp * warp_slot_doubles<double>(NM);
  double* av = base;
  double* ein = base + 6 * NM;
  double* sbv = base + 12 * NM;
  double* nrm = base + 18 * NM;
  double* le = base + 21 * NM;
  double* tb = base + 27 * NM;
  double* gbuf = tb;             // written by the pass, not read: no correction is applied
  double* dein = tb + 42 * NM;
  double* dcv = tb + 48 * NM;
  PointArrays A{};
  A.nrm = nrm; A.ns = 1; A.nrmf = nullptr;
  A.as = 1; A.paper = false;
  A.zs = (size_t)P.n;
  int64_t pt = -1;
  int tr = 0;
  double Eloc[6];
  auto take = [&]() -> bool {
    for (;;) {
      unsigned long long i = 0;
      if (lane == 0) i = atomicAdd(P.counter, 1ull);
      i = __shfl_sync(gmask, i, 0, G);
      if (i >= (unsigned long long)P.n) return false;
      point_of(P.perm, P.tid, P.F.n, (int64_t)i, pt, tr);
      if (tr < P.F.n && P.status[pt] != DMN_STATUS_NONFINITE) break;
    }
    const TreeDev& t = P.F.t[tr];
    const int nzf = 6 * t.nz;
#pragma unroll
    for (int I = 0; I < 6; ++I) Eloc[I] = P.nbuf[(size_t)(3 * NM + I) * P.n + pt];
    for (int f = lane; f < 3 * t.N; f += G) {   // jumps: heap order here, paper order in the state
      const int node = f / 3, c = f - 3 * node;
      const int lvl = 32 - __clz(node + 1);
      const int j = CMP ? node : (1 << t.K) - 3 * (1 << (lvl - 1)) + node + 1;
      av[f] = P.state_out[(size_t)(nzf + 3 * j + c) * P.n + pt];
      nrm[f] = P.nbuf[(size_t)f * P.n + pt];
    }
    __syncwarp(gmask);
    return true;
  };
  bool have = take();
  while (__any_sync(0xffffffffu, have)) {
    if (!have) continue;
    const TreeDev& t = P.F.t[tr];
    A.z = P.state_in + pt;
    WarpSlot<double> W{av, av, gbuf, gbuf, ein, dein, sbv, dcv, NM, le};
    warp_tree_pass<double, CMP>(t, Eloc, A, W, false, 1.0, lane, G, gmask);
    Sub<double> root;
    warp_sub_load<double>(W, CMP ? t.N - 1 : 0, root);
    if (lane == 0) {
      for (int I = 0; I < 6; ++I) P.stress[6 * pt + I] = root.sb[I];
      for (int k = 0; k < 21; ++k) P.tangent[36 * pt + k] = root.C[k];
    }
    __syncwarp(gmask);
    have = take();
  }
}

template <bool CMP>
void launch_sweep_warp(const NewtonParams<double>& P, int lanes, unsigned grid, double* scr, cudaStream_t s) {
  if (lanes == 8) k_sweep_warp<CMP, 8><<<grid, 128, 0, s>>>(P, scr);
  else if (lanes == 16) k_sweep_warp<CMP, 16><<<grid, 128, 0, s>>>(P, scr);
  else k_sweep_warp<CMP, 32><<<grid, 128, 0, s>>>(P, scr);
}

template void launch_sweep_warp<false>(const NewtonParams<double>&, int, unsigned, double*, cudaStream_t);
template void launch_sweep_warp<true>(const NewtonParams<double>&, int, unsigned, double*, cudaStream_t);
template void launch_warp<double, false>(const NewtonParams<double>&, bool, int, unsigned, double*, cudaStream_t);
template void launch_warp<double, true>(const NewtonParams<double>&, bool, int, unsigned, double*, cudaStream_t);
template void launch_warp<float, false>(const NewtonParams<float>&, bool, int, unsigned, double*, cudaStream_t);
template void launch_warp<float, true>(const NewtonParams<float>&, bool, int, unsigned, double*, cudaStream_t);

}  // namespace dmn
