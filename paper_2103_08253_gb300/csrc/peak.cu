// Sustained FP64 / FP32 FMA throughput of the current GPU (include/dmn_peak.h).
#include <cuda_runtime.h>

#include <string>

#include "dmn.h"
#include "dmn_peak.h"

// defined in dmn.cu: the message returned by dmn_last_error(NULL)
void dmn_set_create_error(const std::string& msg);

namespace {

constexpr int PEAK_MAX_CHAINS = 8;

// Each thread of the first `active` lanes of every warp runs CH independent chains
// x <- x a + b (a slightly below 1 keeps the values bounded); the other lanes skip the loop.
// The sum written at the end keeps the chains live.
template <typename T, int CH>
__global__ void __launch_bounds__(128) k_fma_peak(T* __restrict__ out, int iters, int active, T a, T b) {
  T x[CH];
#pragma unroll
  for (int c = 0; c < CH; ++c) x[c] = (T)(threadIdx.x + c) * (T)1e-3;
  if ((int)(threadIdx.x & 31) < active) {
#pragma unroll 4
    for (int i = 0; i < iters; ++i)
#pragma unroll
      for (int c = 0; c < CH; ++c) x[c] = fma(x[c], a, b);
  }
  T s = (T)0;
#pragma unroll
  for (int c = 0; c < CH; ++c) s += x[c];
  out[(size_t)blockIdx.x * blockDim.x + threadIdx.x] = s;
}

int peak_fail(cudaError_t e, const char* what) {
  dmn_set_create_error(std::string("dmn_fma_throughput: ") + what + ": " + cudaGetErrorString(e));
  return DMN_ERR_CUDA;
}

template <typename T, int CH>
cudaError_t launch(unsigned grid, int block, cudaStream_t s, T* out, int iters, int active) {
  k_fma_peak<T, CH><<<grid, block, 0, s>>>(out, iters, active, (T)0.999999, (T)1e-7);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_ch(int chains, unsigned grid, int block, cudaStream_t s, T* out, int iters, int active) {
  switch (chains) {
    case 1: return launch<T, 1>(grid, block, s, out, iters, active);
    case 2: return launch<T, 2>(grid, block, s, out, iters, active);
    case 4: return launch<T, 4>(grid, block, s, out, iters, active);
    default: return launch<T, 8>(grid, block, s, out, iters, active);
  }
}

template <typename T>
int measure(int wps, int chains, int active, double seconds, double* gflops, double* ms_out, cudaStream_t s) {
  int dev = 0, nsm = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return peak_fail(e, "device query");
  const int block = wps >= 4 ? 128 : 32 * wps;
  const unsigned grid = (unsigned)(nsm * (wps * 32 / block));
  const size_t threads = (size_t)grid * block;
  T* out = nullptr;
  e = cudaMalloc(&out, threads * sizeof(T));
  if (e != cudaSuccess) return peak_fail(e, "cudaMalloc");
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  // calibration: iterations for about 20 ms per launch
  int iters = (1 << 14) / chains;
  float ms = 0.0f;
  if (e == cudaSuccess) e = launch_ch<T>(chains, grid, block, s, out, iters, active);   // warm-up
  if (e == cudaSuccess) e = cudaEventRecord(e0, s);
  if (e == cudaSuccess) e = launch_ch<T>(chains, grid, block, s, out, iters, active);
  if (e == cudaSuccess) e = cudaEventRecord(e1, s);
  if (e == cudaSuccess) e = cudaEventSynchronize(e1);
  if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
  if (e == cudaSuccess && ms > 0.0f) {
    const double scale = 20.0 / (double)ms;
    const double it = (double)iters * (scale > 1.0 ? scale : 1.0);
    iters = it > 1e8 ? 100000000 : (int)it;
  }
  int launches = (int)(seconds * 1000.0 / 20.0);
  if (launches < 1) launches = 1;
  if (e == cudaSuccess) e = cudaEventRecord(e0, s);
  for (int k = 0; k < launches && e == cudaSuccess; ++k) e = launch_ch<T>(chains, grid, block, s, out, iters, active);
  if (e == cudaSuccess) e = cudaEventRecord(e1, s);
  if (e == cudaSuccess) e = cudaEventSynchronize(e1);
  if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaFree(out);
  if (e != cudaSuccess) return peak_fail(e, "timed launches");
  const double lanes = (double)threads / 32.0 * active;
  const double flops = 2.0 * chains * (double)iters * lanes * launches;
  *gflops = flops / (ms * 1e-3) * 1e-9;
  *ms_out = ms;
  return DMN_OK;
}

}  // namespace

extern "C" int dmn_fma_throughput(int32_t kind, int32_t warps_per_sm, int32_t chains, int32_t active_lanes,
                                  double seconds, double* gflops, double* ms, void* stream) {
  if (!gflops || !ms || !(seconds > 0.0) || warps_per_sm < 1 || warps_per_sm > 64 ||
      (warps_per_sm > 4 && warps_per_sm % 4 != 0) || (chains != 1 && chains != 2 && chains != 4 && chains != 8) ||
      active_lanes < 1 || active_lanes > 32) {
    dmn_set_create_error("dmn_fma_throughput: invalid argument");
    return DMN_ERR_ARG;
  }
  cudaStream_t s = (cudaStream_t)stream;
  if (kind == DMN_PEAK_FP64_FMA) return measure<double>(warps_per_sm, chains, active_lanes, seconds, gflops, ms, s);
  if (kind == DMN_PEAK_FP32_FMA) return measure<float>(warps_per_sm, chains, active_lanes, seconds, gflops, ms, s);
  dmn_set_create_error("dmn_fma_throughput: unknown kind");
  return DMN_ERR_ARG;
}

extern "C" int dmn_peak_gflops(int32_t kind, double seconds, double* gflops, double* ms, void* stream) {
  if (!gflops || !ms || !(seconds > 0.0)) {
    dmn_set_create_error("dmn_peak_gflops: NULL output or seconds <= 0");
    return DMN_ERR_ARG;
  }
  if (kind != DMN_PEAK_FP64_FMA && kind != DMN_PEAK_FP32_FMA) {
    dmn_set_create_error("dmn_peak_gflops: unknown kind");
    return DMN_ERR_ARG;
  }
  return dmn_fma_throughput(kind, 64, PEAK_MAX_CHAINS, 32, seconds, gflops, ms, stream);
}
