// FP64 FMA throughput of the current device, measured (gbs_fp64_peak).
//
// On GB300 the FP64 pipe, not HBM, bounds several solve-phase kernels
// (a 4x4 FP64 block costs 16 DFMA per 128 bytes).  Their roofline needs the
// device's real DFMA rate rather than a figure derived from assumed unit
// counts: this kernel issues only independent DFMA chains from every
// resident warp and times them with CUDA events.
//
// The chains take all three operands from per-thread registers, as the
// solve's products do (acc += a * x).  Chains whose multiplier and addend
// are kernel parameters (a = a * m + c) measured 1.006-1.056 TFLOP/s on
// GB300 against 1.195 with register operands, so they would understate the
// rate the kernels can reach.
#include <cuda_runtime.h>

#include <algorithm>
#include <string>

#include "../../include/gbstokes.h"
#include "device.hpp"

namespace gbs {

extern thread_local std::string g_err;

namespace {

constexpr int PEAK_THREADS = 256;
constexpr int PEAK_CHAINS = 8;   // independent FMA chains per thread (latency cover)

// Each thread runs PEAK_CHAINS chains acc_q <- u_q * v_(q+w mod Q) + acc_q
// for `iters` rounds of 16, rotating u between rounds (register moves
// only).  u and v come from the thread index, so nothing folds into
// constants; the values stay finite, and the result is stored only if it
// takes an impossible value, which keeps the chains live.
__global__ void __launch_bounds__(PEAK_THREADS)
    k_dfma_peak(int iters, double* __restrict__ sink) {
  double acc[PEAK_CHAINS], u[PEAK_CHAINS], v[PEAK_CHAINS];
#pragma unroll
  for (int q = 0; q < PEAK_CHAINS; ++q) {
    acc[q] = 0.0;
    u[q] = 1.0 + (double)((threadIdx.x + q) & 255) * 1e-3;
    v[q] = 1.0 - (double)((threadIdx.x + 3 * q + 1) & 255) * 1e-4;
  }
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int w = 0; w < 16; ++w)
#pragma unroll
      for (int q = 0; q < PEAK_CHAINS; ++q)
        acc[q] = fma(u[q], v[(q + w) & (PEAK_CHAINS - 1)], acc[q]);
    const double t = u[0];
#pragma unroll
    for (int q = 0; q < PEAK_CHAINS - 1; ++q) u[q] = u[q + 1];
    u[PEAK_CHAINS - 1] = t;
  }
  double s = 0.0;
#pragma unroll
  for (int q = 0; q < PEAK_CHAINS; ++q) s += acc[q];
  if (s == -1.0) sink[0] = s;
}

}  // namespace
}  // namespace gbs

using namespace gbs;

extern "C" gbs_status gbs_fp64_peak(double* tflops, int32_t* sms, double* sink_dev,
                                    void* stream) {
  g_err.clear();
  if (!tflops || !sms || !sink_dev) {
    g_err = "gbs_fp64_peak: null argument";
    return GBS_ERR_INVALID;
  }
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  int dev = 0, nsm = 0, per_sm = 0;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  auto fail = [&](cudaError_t e) {
    g_err = std::string("gbs_fp64_peak: ") + cudaGetErrorString(e);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    return GBS_ERR_CUDA;
  };
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  if (e == cudaSuccess)
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_dfma_peak, PEAK_THREADS, 0);
  if (e != cudaSuccess) return fail(e);
  if (e == cudaSuccess) e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  if (e != cudaSuccess) return fail(e);
  const int blocks = std::max(1, per_sm) * nsm;
  const int iters = 1024;
  float best = 0.f;
  for (int rep = 0; rep < 6; ++rep) {   // the first two warm the clocks up
    cudaEventRecord(e0, s);
    k_dfma_peak<<<blocks, PEAK_THREADS, 0, s>>>(iters, sink_dev);
    cudaEventRecord(e1, s);
    e = cudaEventSynchronize(e1);
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e != cudaSuccess) return fail(e);
    count_launch();
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    if (rep >= 2 && (best == 0.f || ms < best)) best = ms;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  const double fmas = (double)blocks * PEAK_THREADS * iters * 16.0 * PEAK_CHAINS;
  *tflops = 2.0 * fmas / (best * 1e-3) / 1e12;
  *sms = nsm;
  return GBS_OK;
}
