// Allocation-free variant of the FP64 block SpMV with fused dot products.
//
// The regular entry points keep their reduction scratch (per-CTA partial
// sums and a completion counter) inside a hierarchy handle that
// gbs_build_hierarchy allocates.  Some callers cannot allocate device
// memory at the point where they need this operation: code that runs
// while a CUDA graph is being captured (cudaMalloc is not a capturable
// operation), applications whose memory manager owns the whole device and
// forbids allocations behind its back, and real-time loops that must not
// hit the allocator's latency or failure modes.  gbs_spmv_dots_noalloc
// serves them: the caller passes the matrix and the vectors in device
// memory, and the scratch is a fixed file-scope __device__ array that
// exists once per GPU for the life of the process.
#include <cuda_runtime.h>

#include <cstdint>
#include <mutex>
#include <string>

#include "../../include/gbstokes.h"
#include "device.hpp"
#include "outer.cuh"

namespace gbs {

// Partial sums of the reduction: two doubles per CTA of the fixed grid,
// followed by the completion counter (the last 8 bytes).
constexpr int NOALLOC_CTAS = OUTER_N_BLOCKS;
constexpr int NOALLOC_DOUBLES = 2 * NOALLOC_CTAS + 1;
static __device__ __align__(256) double g_noalloc_scratch[NOALLOC_DOUBLES];

extern thread_local std::string g_err;

namespace {

constexpr int kMaxDevices = 64;
std::mutex g_mu;
double* g_scratch_addr[kMaxDevices] = {nullptr};

// Device address of the scratch array for the current device.  In host
// code g_noalloc_scratch names a host-side stand-in, not device memory, so
// the address must come from cudaGetSymbolAddress with the device current.
cudaError_t scratch_for_current_device(double** out) {
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_scratch_addr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    g_scratch_addr[dev] = static_cast<double*>(p);
  }
  *out = g_scratch_addr[dev];
  return cudaSuccess;
}

bool aligned16(const void* p) { return reinterpret_cast<uintptr_t>(p) % 16 == 0; }

}  // namespace

}  // namespace gbs

using namespace gbs;

extern "C" gbs_status gbs_spmv_dots_noalloc(int32_t n_brows, int32_t n_bcols, int32_t bdim,
                                            int64_t nnzb, const int32_t* row_ptr,
                                            const int32_t* col_idx, const double* vals,
                                            const double* x, double* y, const double* w,
                                            double* dots, void* stream) {
  g_err.clear();
  if (n_brows < 0 || n_bcols < 0 || nnzb < 0 || bdim < 1 || bdim > 4) {
    g_err = "gbs_spmv_dots_noalloc: bad dimensions (need n_brows, n_bcols, nnzb >= 0, bdim 1..4)";
    return GBS_ERR_INVALID;
  }
  if (nnzb > INT32_MAX || (int64_t)n_brows * bdim > INT32_MAX ||
      (int64_t)n_bcols * bdim > INT32_MAX) {
    g_err = "gbs_spmv_dots_noalloc: size beyond the maximum (nnzb and n*bdim must fit in int32)";
    return GBS_ERR_INVALID;
  }
  if (!row_ptr || !dots || (nnzb > 0 && (!col_idx || !vals)) ||
      ((n_brows > 0 || n_bcols > 0) && (!x || !y))) {
    g_err = "gbs_spmv_dots_noalloc: null pointer";
    return GBS_ERR_INVALID;
  }
  if (!aligned16(vals) || !aligned16(x) || !aligned16(y) || (w && !aligned16(w)) ||
      reinterpret_cast<uintptr_t>(dots) % 8 != 0) {
    g_err = "gbs_spmv_dots_noalloc: vals, x, y, w must be 16-byte aligned and dots 8-byte aligned";
    return GBS_ERR_INVALID;
  }
  if (w == y) {
    g_err = "gbs_spmv_dots_noalloc: w must not alias y";
    return GBS_ERR_INVALID;
  }
  double* scratch = nullptr;
  cudaError_t e = scratch_for_current_device(&scratch);
  if (e != cudaSuccess) {
    g_err = std::string("gbs_spmv_dots_noalloc: cudaGetSymbolAddress failed: ") +
            cudaGetErrorString(e);
    return GBS_ERR_CUDA;
  }
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  Red R;
  R.partials = scratch;
  R.counter = reinterpret_cast<unsigned*>(scratch + 2 * NOALLOC_CTAS);
  R.sc = dots;
  // the counter must start at zero: a previous call may have been cut short
  e = cudaMemsetAsync(R.counter, 0, sizeof(double), s);
  if (e != cudaSuccess) {
    g_err = std::string("gbs_spmv_dots_noalloc: ") + cudaGetErrorString(e);
    return GBS_ERR_CUDA;
  }
  DevBsr<double> A;
  A.nbr = n_brows;
  A.nbc = n_bcols;
  A.rp = row_ptr;
  A.col = col_idx;
  A.val = vals;
#define GBS_NA(BB)                                                                           \
  k_outer_n<BB, false, SPMV_SET><<<NOALLOC_CTAS, RED_THREADS, 0, s>>>(A, x, nullptr, y, w, 1, R, \
                                                                      0, FIN_OUT, 1)
  switch (bdim) {
    case 1: GBS_NA(1); break;
    case 2: GBS_NA(2); break;
    case 3: GBS_NA(3); break;
    default: GBS_NA(4); break;
  }
#undef GBS_NA
  e = cudaPeekAtLastError();
  if (e != cudaSuccess) {
    g_err = std::string("gbs_spmv_dots_noalloc: launch failed: ") + cudaGetErrorString(e);
    return GBS_ERR_CUDA;
  }
  count_launch();
  return GBS_OK;
}
