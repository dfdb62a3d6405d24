// Launch parameters shared by the translation units of the DMN library (csrc/dmn.cu, the C ABI and
// the thread-per-point kernels; csrc/dmn_warp.cu, the warp organisation): the trees of a handle,
// the Newton kernels' parameters, and the warp organisation's scratch and launch.
#pragma once
#include <cuda_runtime.h>
#include <cstddef>
#include <cstdint>

#include "../../include/dmn.h"
#include "dmn_device.cuh"

namespace dmn {

// All trees of a handle, passed by value to the kernels.
struct Forest {
  TreeDev t[DMN_MAX_TREES];
  int n;
};

// point handled by thread/work item i and its tree (n_trees = invalid)
__device__ __forceinline__ void point_of(const int64_t* perm, const int32_t* tid, int n_trees, int64_t i,
                                         int64_t& p, int& tree) {
  p = perm ? perm[i] : i;
  const int t = tid ? tid[p] : 0;
  tree = (t >= 0 && t < n_trees) ? t : n_trees;
}

template <typename T>
struct NewtonParams {
  Forest F;
  int64_t n, nslots;
  int N_max;
  const int32_t* tid;
  const int64_t* perm;
  const double* state_in;
  double *state_out, *stress, *tangent;
  int32_t *iters, *status;
  const double* nbuf;
  double* scr_d;
  T* scr_t;
  unsigned long long* counter;
  double tol;
  int max_iter;
  int write_outputs;  // no final sweep: stress and tangent (local frame) come from the converged Newton pass
  int predictor;      // extrapolated start; the state carries the last jump change and strain increment
  const double* dE;   // [n][6] strain increments (global frame), read with the extrapolated start
  const double* a_start;  // the jumps to start from (state layout), or NULL for those of state_in; with the
                          // first stage these are its jumps in state_out, and iters holds its corrections
  unsigned long long* passes;  // profiling: tree passes of all points added here, or NULL
  int min_corr;       // corrections before the criterion may end the iteration (1 for the FP64 form after
                      // the first stage: one quadratic step from the FP32 iterate, so that the accepted
                      // iterate is as far inside the criterion as in the plain FP64 iteration)
};

// Small calls: one point per group of G lanes of a warp (G = 32, 16 or 8; the paper's start; heap
// trees or compressed ones), the group's lanes sharing each level of the tree (warp_tree_pass).
// The Newton loop is k_newton's.  The warp's groups run their passes side by side: every iteration
// of the warp's loop is one pass of every group that holds a point, so the groups' lanes stay
// together (the pass's instructions are the same for every point); a group whose point is done
// writes it out and takes the next one from the work counter.  Each group owns a block of scratch
// (warp_slot_doubles<T>(N) doubles) holding its point's jumps, g, H, level hand-over and subtree
// results, in two buffers where the line search needs them.
template <typename T>
__host__ __device__ inline size_t warp_slot_doubles(int N) {
  // jumps 2 x 3N, ein 6N, sb 6N, normals 3N, leaf-child strains 6N (FP64); g, H 2 x 21N, dein 6N,
  // ds + C 27N (T); FP32 normals 3N
  const size_t d = (size_t)27 * N, tt = (size_t)75 * N * sizeof(T), f = (size_t)3 * N * sizeof(float);
  return d + (tt + f + sizeof(double) - 1) / sizeof(double);
}
constexpr int WARP_CTAS_PER_SM = 2;   // 128-thread CTAs: 8 warps per SM
constexpr int WARP_MIN_LANES = 8;     // the smallest group: the scratch holds 32 / 8 = 4 slots per warp

// k_newton_warp<T, LS, lanes, CMP> on `grid` CTAs of 128 threads (csrc/dmn_warp.cu); `scr` holds
// grid * 128 / lanes slots of warp_slot_doubles<T>(P.N_max) doubles
template <typename T, bool CMP>
void launch_warp(const NewtonParams<T>& P, bool ls, int lanes, unsigned grid, double* scr, cudaStream_t s);
// k_sweep_warp<CMP, lanes>: the mixed form's FP64 final sweep in the warp organisation (csrc/dmn_warp.cu);
// `scr` holds grid * 128 / lanes slots of warp_slot_doubles<double>(P.N_max) doubles
template <bool CMP>
void launch_sweep_warp(const NewtonParams<double>& P, int lanes, unsigned grid, double* scr, cudaStream_t s);

}  // namespace dmn
