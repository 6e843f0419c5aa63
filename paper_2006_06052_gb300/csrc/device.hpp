// Device-resident preconditioners (internal interface).
#pragma once

#include <cuda_runtime.h>

#include <memory>
#include <stdexcept>
#include <string>
#include <vector>

#include <cstdlib>

#include <nvtx3/nvToolsExt.h>

#include "setup.hpp"

namespace gbs {

struct CudaError {
  std::string msg;
};

#define GBS_CUDA(call)                                                              \
  do {                                                                              \
    cudaError_t e__ = (call);                                                       \
    if (e__ != cudaSuccess)                                                         \
      throw ::gbs::CudaError{std::string(#call) + ": " + cudaGetErrorString(e__)};  \
  } while (0)

// Kernel launches issued by this library (see gbs_kernel_launches).
void count_launch(int64_t k = 1);
int64_t launch_count();

#define GBS_LAUNCH_CHECK()               \
  do {                                   \
    GBS_CUDA(cudaPeekAtLastError());     \
    ::gbs::count_launch();               \
  } while (0)

// Owns device allocations; counts bytes.
struct Arena {
  std::vector<void*> ptrs;
  int64_t bytes = 0;
  template <class T>
  T* alloc(size_t n) {
    if (n == 0) n = 1;
    void* p = nullptr;
    cudaError_t e = cudaMalloc(&p, n * sizeof(T));
    if (e != cudaSuccess) {
      cudaGetLastError();
      throw CudaError{"cudaMalloc of " + std::to_string(n * sizeof(T)) + " bytes failed: " +
                      cudaGetErrorString(e)};
    }
    ptrs.push_back(p);
    bytes += (int64_t)(n * sizeof(T));
    return static_cast<T*>(p);
  }
  template <class T>
  T* upload(const T* h, size_t n, cudaStream_t s) {
    T* d = alloc<T>(n);
    if (n) GBS_CUDA(cudaMemcpyAsync(d, h, n * sizeof(T), cudaMemcpyHostToDevice, s));
    return d;
  }
  void release() {
    for (void* p : ptrs) cudaFree(p);
    ptrs.clear();
    bytes = 0;
  }
  ~Arena() { release(); }
};

// A preconditioner z = M^-1 r acting on FP64 outer vectors.
struct DevPrecond {
  virtual ~DevPrecond() = default;
  virtual void apply(const double* r, double* z, bool transpose, cudaStream_t s) = 0;
  virtual int64_t bytes() const = 0;
  virtual int nlevels(int which) const = 0;
  virtual int64_t level_rows(int which, int l) const = 0;
  virtual int64_t level_nnzb(int which, int l) const = 0;
  // algorithmic bytes moved by one application (from the stored sizes)
  virtual double bytes_per_apply() const = 0;
  // one level operation of AMG `which` (0 residual, 1 relaxation sweep) on
  // vectors of the hierarchy's vector type (vector_bytes() wide)
  virtual void level_op(int which, int l, int op, const void* x, const void* f, void* y,
                        cudaStream_t s) {
    (void)which; (void)l; (void)op; (void)x; (void)f; (void)y; (void)s;
    throw SetupError{"level_op is not available for this preconditioner"};
  }
  virtual int vector_bytes() const { return 8; }
  // layout A_l of AMG `which` runs in (forward): 0 block CSR, 1 scalar CSR,
  // 2 scalar slices, 3 block-row slices; +4 when the level fuses its
  // zero-guess smoothing step with the residual
  virtual int level_layout(int which, int l) const { return 0; }
};

struct PrecondOptions {
  int precision = 0;   // 0 FP64, 1 FP32, 2 BF16
  int npre = 1, npost = 1;
  bool tmaps = true;
  int level_format = 0;  // 0 automatic, 1 blocks, 2 plain scalar CSR, 3 sliced scalar CSR
  int schur_order = 0;   // 0 full (two velocity solves), 1 lower (one)
  bool schur_p_smoother = false;  // pressure solve = one smoother application (HSchur::MS)
  double* err = nullptr;          // device slot a timed-out pipelined kernel sets to 1.0
  long long wait_cycles = 1LL << 31;  // bound of a pipeline wait (SM clocks)
  int ilut_sweeps = 2;            // Jacobi sweeps per ILUT triangular solve
  double ilut_omega = 1.0;        // ILUT relaxation damping
  bool iso = true;                // store levels of multiples of I_B as S (x) I_B (iso.cuh)
};

std::unique_ptr<DevPrecond> make_amg_precond(const HAmg& H, const PrecondOptions& o,
                                             cudaStream_t s);
std::unique_ptr<DevPrecond> make_schur_precond(const HSchur& S, const HAmg& HA, const HAmg& HS,
                                               const PrecondOptions& o, cudaStream_t s);

// Per-form factories (one translation unit each).
std::unique_ptr<DevPrecond> make_amg_fp64(const HAmg&, const PrecondOptions&, cudaStream_t);
std::unique_ptr<DevPrecond> make_amg_fp32(const HAmg&, const PrecondOptions&, cudaStream_t);
std::unique_ptr<DevPrecond> make_amg_bf16(const HAmg&, const PrecondOptions&, cudaStream_t);
std::unique_ptr<DevPrecond> make_schur_fp64(const HSchur&, const HAmg&, const HAmg&,
                                            const PrecondOptions&, cudaStream_t);
std::unique_ptr<DevPrecond> make_schur_fp32(const HSchur&, const HAmg&, const HAmg&,
                                            const PrecondOptions&, cudaStream_t);
std::unique_ptr<DevPrecond> make_schur_bf16(const HSchur&, const HAmg&, const HAmg&,
                                            const PrecondOptions&, cudaStream_t);

// NVTX ranges around each Krylov phase and each V-cycle level, for
// profilers that show them; recorded only when the environment variable
// GBS_NVTX is set (to anything but 0) when the library first checks it.
inline bool nvtx_on() {
  static const bool on = [] {
    const char* e = std::getenv("GBS_NVTX");
    return e && e[0] && e[0] != '0';
  }();
  return on;
}
struct NvtxRange {
  bool on;
  explicit NvtxRange(const char* name) : on(nvtx_on()) {
    if (on) nvtxRangePushA(name);
  }
  ~NvtxRange() {
    if (on) nvtxRangePop();
  }
  NvtxRange(const NvtxRange&) = delete;
  NvtxRange& operator=(const NvtxRange&) = delete;
};

}  // namespace gbs
