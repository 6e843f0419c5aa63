// Device kernels of the solve phase (sm_103a).
//
// The solve phase is expressed, as in Section 2.3 of the paper, through a
// few bandwidth-bound primitives -- block SpMV, residual f - A x,
// relaxation x += M (f - A x), zero-guess smoothing x = M f, restriction
// and prolongation (both SpMVs), dense coarse GEMV -- over block-CSR
// matrices whose values are small dense blocks (the value types of
// Section 2.4; statically sized 3x3 blocks in Listing V3).
//
// Layout: vectors are interleaved per block row (B consecutive values);
// block values are row-major, one block after another in CSR order.
// Thread mapping: B consecutive lanes own one block row (lane r computes
// scalar row r of the block), 32/B block rows per warp, so a block row
// never straddles a warp and its B lanes can exchange values by shuffles.
// Value storage may be FP64, FP32 or BF16; accumulation is in AT (FP64 or
// FP32).  None of this uses tensor cores: every kernel here moves far
// more bytes than it does flops.
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace gbs {

template <class VT>
struct DevBsr {
  int nbr = 0, nbc = 0;
  const int* rp = nullptr;
  const int* col = nullptr;
  const VT* val = nullptr;
  const int* tmap = nullptr;  // transpose map (may be null)
};

// ---------------------------------------------------------------- conversions
__device__ __forceinline__ float to_f(float v) { return v; }
__device__ __forceinline__ float to_f(double v) { return (float)v; }
__device__ __forceinline__ float to_f(__nv_bfloat16 v) { return __bfloat162float(v); }
template <class AT, class T>
__device__ __forceinline__ AT cvt(T v);
template <> __device__ __forceinline__ double cvt<double, double>(double v) { return v; }
template <> __device__ __forceinline__ double cvt<double, float>(float v) { return (double)v; }
template <> __device__ __forceinline__ float cvt<float, float>(float v) { return v; }
template <> __device__ __forceinline__ float cvt<float, double>(double v) { return (float)v; }
template <> __device__ __forceinline__ float cvt<float, __nv_bfloat16>(__nv_bfloat16 v) {
  return __bfloat162float(v);
}
template <> __device__ __forceinline__ double cvt<double, __nv_bfloat16>(__nv_bfloat16 v) {
  return (double)__bfloat162float(v);
}

// ------------------------------------------------------------- vector loads
// Load N consecutive T values starting at p into registers (as AT),
// using 16-byte or 8-byte loads when the run is a multiple of that size
// (block rows and vector blocks are then naturally aligned).
template <int N, class T, class AT, bool NC>
__device__ __forceinline__ void load_run(const T* __restrict__ p, AT (&out)[N]) {
  constexpr int bytes = N * (int)sizeof(T);
  if constexpr (bytes % 16 == 0) {
    constexpr int V = bytes / 16;
    constexpr int PER = 16 / (int)sizeof(T);
#pragma unroll
    for (int v = 0; v < V; ++v) {
      int4 w = NC ? __ldcs(reinterpret_cast<const int4*>(p) + v)
                  : __ldg(reinterpret_cast<const int4*>(p) + v);
      T tmp[PER];
      memcpy(tmp, &w, 16);
#pragma unroll
      for (int e = 0; e < PER; ++e) out[v * PER + e] = cvt<AT>(tmp[e]);
    }
  } else if constexpr (bytes % 8 == 0) {
    constexpr int V = bytes / 8;
    constexpr int PER = 8 / (int)sizeof(T);
#pragma unroll
    for (int v = 0; v < V; ++v) {
      int2 w = NC ? __ldcs(reinterpret_cast<const int2*>(p) + v)
                  : __ldg(reinterpret_cast<const int2*>(p) + v);
      T tmp[PER];
      memcpy(tmp, &w, 8);
#pragma unroll
      for (int e = 0; e < PER; ++e) out[v * PER + e] = cvt<AT>(tmp[e]);
    }
  } else {
#pragma unroll
    for (int e = 0; e < N; ++e) out[e] = cvt<AT>(p[e]);
  }
}

// Column r of a B x B row-major block (strided; used by transposed ops).
template <int B, class T, class AT>
__device__ __forceinline__ void load_col(const T* __restrict__ blk, int r, AT (&out)[B]) {
#pragma unroll
  for (int c = 0; c < B; ++c) out[c] = cvt<AT>(blk[c * B + r]);
}

// ------------------------------------------------------------ row mapping
template <int B>
struct RowMap {
  static constexpr int RPW = 32 / B;  // block rows per warp
  int brow, r, lane, base;
  bool lane_ok;
  __device__ __forceinline__ explicit RowMap(int64_t gtid) {
    int64_t warp = gtid >> 5;
    lane = (int)(gtid & 31);
    int sub = lane / B;
    r = lane - sub * B;
    base = sub * B;
    lane_ok = sub < RPW;
    brow = (int)(warp * RPW + sub);
  }
};

template <int B>
inline int64_t row_threads(int nbr) {
  constexpr int RPW = 32 / B;
  return (int64_t)((nbr + RPW - 1) / RPW) * 32;
}

// Row r of (A x) for block row `brow` (A x or A^T x through tmap).
template <int B, bool TR, class VT, class XT, class AT>
__device__ __forceinline__ AT row_dot(const DevBsr<VT>& A, const XT* __restrict__ x, int brow,
                                      int r) {
  AT acc = AT(0);
  const int k0 = A.rp[brow], k1 = A.rp[brow + 1];
#pragma unroll 2
  for (int k = k0; k < k1; ++k) {
    const int j = __ldg(A.col + k);
    AT a[B], xv[B];
    if constexpr (!TR) {
      load_run<B, VT, AT, true>(A.val + (size_t)k * (B * B) + r * B, a);
    } else {
      const int kt = __ldg(A.tmap + k);
      load_col<B, VT, AT>(A.val + (size_t)kt * (B * B), r, a);
    }
    load_run<B, XT, AT, false>(x + (size_t)j * B, xv);
#pragma unroll
    for (int c = 0; c < B; ++c) acc += a[c] * xv[c];
  }
  return acc;
}

// ------------------------------------------------------------------ kernels
enum { SPMV_SET = 0, SPMV_RESID = 1, SPMV_ADD = 2 };

// MODE SET: y = A x;  RESID: y = f - A x;  ADD: y += A x.
template <int B, bool TR, int MODE, class VT, class XT, class YT, class AT>
__global__ void __launch_bounds__(256) k_spmv(DevBsr<VT> A, const XT* __restrict__ x,
                                              const YT* __restrict__ f, YT* __restrict__ y) {
  RowMap<B> m(blockIdx.x * (int64_t)blockDim.x + threadIdx.x);
  if (!m.lane_ok || m.brow >= A.nbr) return;
  AT acc = row_dot<B, TR, VT, XT, AT>(A, x, m.brow, m.r);
  const size_t o = (size_t)m.brow * B + m.r;
  if constexpr (MODE == SPMV_SET) y[o] = (YT)acc;
  else if constexpr (MODE == SPMV_RESID) y[o] = (YT)(cvt<AT>(f[o]) - acc);
  else y[o] = (YT)(cvt<AT>(y[o]) + acc);
}

// xo = x + M (f - A x)   (one relaxation sweep; M^T, A^T when TR).
template <int B, bool TR, class VT, class XT, class AT>
__global__ void __launch_bounds__(256) k_relax(DevBsr<VT> A, const VT* __restrict__ M,
                                               const XT* __restrict__ f,
                                               const XT* __restrict__ x, XT* __restrict__ xo) {
  RowMap<B> m(blockIdx.x * (int64_t)blockDim.x + threadIdx.x);
  const bool ok = m.lane_ok && m.brow < A.nbr;
  const size_t o = (size_t)m.brow * B + m.r;
  AT res = AT(0);
  if (ok) res = cvt<AT>(f[o]) - row_dot<B, TR, VT, XT, AT>(A, x, m.brow, m.r);
  AT rb[B];
#pragma unroll
  for (int c = 0; c < B; ++c) rb[c] = __shfl_sync(0xffffffffu, res, (m.base + c) & 31);
  if (!ok) return;
  AT mr[B];
  if constexpr (!TR) load_run<B, VT, AT, false>(M + (size_t)m.brow * (B * B) + m.r * B, mr);
  else load_col<B, VT, AT>(M + (size_t)m.brow * (B * B), m.r, mr);
  AT out = cvt<AT>(x[o]);
#pragma unroll
  for (int c = 0; c < B; ++c) out += mr[c] * rb[c];
  xo[o] = (XT)out;
}

// x = M f   (zero-guess smoothing step).
template <int B, bool TR, class VT, class XT, class AT>
__global__ void __launch_bounds__(256) k_mapply(int nbr, const VT* __restrict__ M,
                                                const XT* __restrict__ f, XT* __restrict__ x) {
  RowMap<B> m(blockIdx.x * (int64_t)blockDim.x + threadIdx.x);
  if (!m.lane_ok || m.brow >= nbr) return;
  AT mr[B], fv[B];
  if constexpr (!TR) load_run<B, VT, AT, false>(M + (size_t)m.brow * (B * B) + m.r * B, mr);
  else load_col<B, VT, AT>(M + (size_t)m.brow * (B * B), m.r, mr);
  load_run<B, XT, AT, false>(f + (size_t)m.brow * B, fv);
  AT out = AT(0);
#pragma unroll
  for (int c = 0; c < B; ++c) out += mr[c] * fv[c];
  x[(size_t)m.brow * B + m.r] = (XT)out;
}

// x = Ainv f, dense n x n row-major, one warp per row.
template <class VT, class XT, class AT>
__global__ void __launch_bounds__(256) k_gemv(int n, const VT* __restrict__ Ainv,
                                              const XT* __restrict__ f, XT* __restrict__ x) {
  const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (warp >= n) return;
  const VT* row = Ainv + (size_t)warp * n;
  AT acc = AT(0);
  for (int j = lane; j < n; j += 32) acc += cvt<AT>(row[j]) * cvt<AT>(f[j]);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if (lane == 0) x[warp] = (XT)acc;
}

template <class TI, class TO>
__global__ void k_cast(int64_t n, const TI* __restrict__ in, TO* __restrict__ out) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    out[i] = (TO)cvt<float>(in[i]);
}
template <>
__global__ void k_cast<double, double>(int64_t n, const double* __restrict__ in,
                                       double* __restrict__ out) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    out[i] = in[i];
}
template <>
__global__ void k_cast<float, double>(int64_t n, const float* __restrict__ in,
                                      double* __restrict__ out) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    out[i] = (double)in[i];
}

inline unsigned grid_for(int64_t threads, int tpb = 256) {
  int64_t g = (threads + tpb - 1) / tpb;
  return (unsigned)(g < 1 ? 1 : g);
}

}  // namespace gbs
