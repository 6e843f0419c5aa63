// Sliced scalar CSR kernels with a per-warp TMA pipeline.
//
// A scalar CSR operator whose rows come in B components per node (the
// fine level and K of a block system) is stored in slices: the rows of
// component c of 32 consecutive nodes form slice q = group * B + c,
// column-major, padded with column -1 to the slice's longest row (see
// HSell).  One warp owns one row per lane, so on the FP64 pipe -- where a
// warp instruction costs the same with idle lanes -- every lane is busy,
// and a slice's values and columns are two contiguous runs.
//
// Uniform slices (a stencil level's) need no column loads in the FP64
// direct kernels: the gather address is the row plus the column's offset,
// so the value and the x entry load together.  The staged kernels read
// the columns from shared memory, which measured faster than offsets for
// them, even with the offsets staged beside the values (C2 BF16 V-cycle:
// 181 us explicit; 190 us with staged offsets; 201 us with offsets from
// global memory).
//
// For the FP32 and BF16 forms those runs stream into shared memory by
// bulk asynchronous copies (cp.async.bulk, completion counted on an
// mbarrier).  Each warp keeps NST chunks of CW columns in flight while it
// gathers x for the chunk it is working on, so the value stream does not
// wait behind the gathers; the lanes then read their entries from shared
// memory without bank conflicts.  The FP64 form uses direct loads (see
// the direct variants below).
//
// Every wait on an mbarrier is bounded (about a second of SM clock).  On a
// timeout the warp records 1.0 in *err, waits (again bounded) for its other
// copies in flight, and stops; the host reports the flag.
#pragma once

#include <algorithm>
#include <map>
#include <mutex>
#include <utility>

#include "kernels.cuh"

namespace gbs {

// Blocks of a grid-stride launch: all that stay resident at once on this
// device (one wave, from the kernel's register and shared-memory use), at
// most cap.  A fixed 8 CTAs per SM needs <= 32 registers a thread; kernels
// above that would otherwise run a second, partial wave.
inline unsigned resident_grid(const void* fn, int cap, int threads, size_t smem) {
  static std::mutex mu;
  static std::map<std::pair<const void*, int>, int64_t> cache;   // CTAs resident per device
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return (unsigned)std::max(cap, 1);
  int64_t resident = 0;
  {
    std::lock_guard<std::mutex> lock(mu);
    const auto key = std::make_pair(fn, dev);
    const auto it = cache.find(key);
    if (it != cache.end()) {
      resident = it->second;
    } else {
      int per_sm = 0, sms = 0;
      if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, threads, smem) != cudaSuccess ||
          cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
          per_sm < 1 || sms < 1) {
        (void)cudaGetLastError();
        return (unsigned)std::max(cap, 1);
      }
      resident = (int64_t)per_sm * sms;
      cache[key] = resident;
    }
  }
  return (unsigned)std::max<int64_t>(1, std::min<int64_t>(resident, cap));
}

namespace sellp {

__device__ __forceinline__ uint32_t saddr(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void bar_init(uint64_t* b, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(saddr(b)), "r"(count) : "memory");
}
__device__ __forceinline__ void bar_init_fence() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
// Arrive once and add `bytes` to the transaction count of the current phase.
__device__ __forceinline__ void bar_arrive_tx(uint64_t* b, uint32_t bytes) {
  asm volatile(
      "{\n\t.reg .b64 st;\n\t"
      "mbarrier.arrive.expect_tx.shared::cta.b64 st, [%0], %1;\n\t}" ::"r"(saddr(b)),
      "r"(bytes)
      : "memory");
}
// Order this thread's earlier shared-memory accesses before later
// async-proxy (bulk copy) writes to the same buffer.
__device__ __forceinline__ void fence_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
// dst (shared) <- src (global), `bytes` a multiple of 16, both 16-byte aligned.
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* b) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::
          "r"(saddr(dst)),
      "l"(src), "r"(bytes), "r"(saddr(b))
      : "memory");
}
__device__ __forceinline__ bool bar_try(uint64_t* b, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(saddr(b)), "r"(parity)
      : "memory");
  return ok != 0;
}
// Non-blocking test of the phase with parity `parity`.
__device__ __forceinline__ bool bar_test(uint64_t* b, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(saddr(b)), "r"(parity)
      : "memory");
  return ok != 0;
}
constexpr long long WAIT_CYCLES = 1LL << 31;   // about a second at 2 GHz
constexpr long long WAIT_POLL = 1LL << 20;     // bounds below this poll without suspending
// Wait for the phase with parity `parity` to complete; false after `bound`
// SM clocks.  try_wait may suspend the thread for a while by itself, so a
// bound below WAIT_POLL (tests of the timeout path) polls with test_wait,
// which returns at once, and is honoured to the clock.
__device__ __forceinline__ bool bar_wait(uint64_t* b, uint32_t parity,
                                         long long bound = WAIT_CYCLES) {
  const long long t0 = clock64();
  if (bound < WAIT_POLL) {
    while (!bar_test(b, parity))
      if (clock64() - t0 > bound) return false;
    return true;
  }
  if (bar_try(b, parity)) return true;
  while (!bar_try(b, parity))
    if (clock64() - t0 > bound) return false;
  return true;
}

}  // namespace sellp

constexpr int SELL_WARPS = 8;      // warps per CTA of the pipelined kernels
constexpr int SELL_CW = 16;        // columns per pipeline stage
constexpr int SELL_NST = 2;        // stages per warp

template <class VT>
struct SellStages {
  VT val[SELL_NST][SELL_CW * 32];
  int col[SELL_NST][SELL_CW * 32];
  uint64_t bar[SELL_NST];
};
template <class VT>
constexpr size_t sell_smem_bytes() {
  return sizeof(SellStages<VT>) * SELL_WARPS;
}

// Walk the slices of this warp's units -- unit u covers slices u*U ..
// u*U + U-1; units u = warp, warp + warps, ... below nunits -- and call
// on_slice(u, s, acc) with each lane's row sum (entries in CSR column
// order) at the end of every slice.  Returns false after a timed-out wait.
template <class VT, class XT, class AT, class SliceFn>
__device__ __forceinline__ bool sell_pipe(const DevSell<VT>& A, const XT* __restrict__ x, int U,
                                          int64_t nunits, SellStages<VT>& sm, SliceFn&& on_slice) {
  using namespace sellp;
  constexpr int CW = SELL_CW, NST = SELL_NST;
  const int lane = threadIdx.x & 31;
  const int64_t w0 = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t ws = ((int64_t)gridDim.x * blockDim.x) >> 5;
  if (lane == 0) {
#pragma unroll
    for (int st = 0; st < NST; ++st) bar_init(&sm.bar[st], 1);
    bar_init_fence();
  }
  __syncwarp();
  // producer cursor: every lane tracks it, lane 0 issues the copies
  int64_t pu = w0;
  int ps = 0, pk = 0;
  auto issue = [&](int st) -> bool {
    if (pu >= nunits) return false;
    const int q = (int)(pu * U + ps);
    const int o0 = __ldg(A.off + q), w = __ldg(A.off + q + 1) - o0;
    const int nc = min(CW, w - pk);
    if (lane == 0) {
      const uint32_t vb = (uint32_t)nc * 32u * (uint32_t)sizeof(VT);
      const uint32_t cb = (uint32_t)nc * 32u * 4u;
      fence_async_smem();
      bar_arrive_tx(&sm.bar[st], vb + cb);
      if (nc > 0) {
        bulk_g2s(sm.val[st], A.val + ((size_t)o0 + pk) * 32, vb, &sm.bar[st]);
        bulk_g2s(sm.col[st], A.col + ((size_t)o0 + pk) * 32, cb, &sm.bar[st]);
      }
    }
    pk += CW;
    if (pk >= w) {
      pk = 0;
      if (++ps == U) {
        ps = 0;
        pu += ws;
      }
    }
    return true;
  };
  int issued = 0;
#pragma unroll
  for (int st = 0; st < NST; ++st)
    if (issue(st)) ++issued;
  int64_t cu = w0;
  int cs = 0, ck = 0;
  AT acc = AT(0);
  for (int it = 0; it < issued; ++it) {
    const int st = it % NST;
    const int q = (int)(cu * U + cs);
    const int o0 = __ldg(A.off + q), w = __ldg(A.off + q + 1) - o0;
    const int nc = min(CW, w - ck);
    // the decision to stop is warp-uniform: every lane takes it together
    if (!__all_sync(0xffffffffu, bar_wait(&sm.bar[st], (uint32_t)(it / NST) & 1u, A.wait))) {
      if (lane == 0 && A.err) *A.err = 1.0;
      // every copy in flight lands before the warp leaves: the drain waits
      // with the full bound whatever A.wait is
      for (int j = it; j < issued; ++j)
        (void)bar_wait(&sm.bar[j % NST], (uint32_t)(j / NST) & 1u);
      __syncwarp();
      return false;
    }
    const VT* __restrict__ sv = sm.val[st];
    const int* __restrict__ sc = sm.col[st];
    for (int k0 = 0; k0 < nc; k0 += 8) {
      int jj[8];
      VT aa[8];
      XT xx[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        jj[u] = k0 + u < nc ? sc[(k0 + u) * 32 + lane] : -1;
        aa[u] = k0 + u < nc ? sv[(k0 + u) * 32 + lane] : VT(0);
      }
#pragma unroll
      for (int u = 0; u < 8; ++u) xx[u] = jj[u] >= 0 ? __ldg(x + jj[u]) : XT(0);
#pragma unroll
      for (int u = 0; u < 8; ++u)
        if (k0 + u < nc) {
          if (jj[u] >= 0) acc += cvt<AT>(aa[u]) * cvt<AT>(xx[u]);
        }
    }
    ck += CW;
    if (ck >= w) {
      on_slice(cu, cs, acc);
      acc = AT(0);
      ck = 0;
      if (++cs == U) {
        cs = 0;
        cu += ws;
      }
    }
    __syncwarp();
    if (issue(st)) ++issued;
  }
  return true;
}

// MODE SET / RESID / ADD on a sliced operator.
template <int MODE, class VT, class XT, class YT, class AT>
__global__ void __launch_bounds__(SELL_WARPS * 32, 2)
    k_sell_spmv(DevSell<VT> A, const XT* __restrict__ x, const YT* __restrict__ f,
                YT* __restrict__ y) {
  GBS_GRID_DEP();
  extern __shared__ __align__(128) unsigned char sell_smem[];
  SellStages<VT>& sm = reinterpret_cast<SellStages<VT>*>(sell_smem)[threadIdx.x >> 5];
  const int lane = threadIdx.x & 31;
  sell_pipe<VT, XT, AT>(A, x, 1, A.nslices, sm, [&](int64_t q, int, AT acc) {
    const int64_t g = q / A.B;
    const int64_t node = sell_node(A, g, lane);
    if (node < 0) return;
    const int64_t row = node * A.B + (q - g * A.B);
    if constexpr (MODE == SPMV_SET) y[row] = (YT)acc;
    else if constexpr (MODE == SPMV_RESID) y[row] = (YT)(cvt<AT>(f[row]) - acc);
    else y[row] = (YT)(cvt<AT>(y[row]) + acc);
  });
}

// MODE SET / RESID / ADD with one unit per 32-node group: the warp walks
// the group's B slices and each lane then writes its node's B rows, B
// consecutive values, so a warp's stores cover one contiguous run (one
// slice per warp writes every B-th value: partial sectors, measured 101 us
// against 74 us for the relaxation sweep over the same C3 velocity level).
template <int B, int MODE, class VT, class XT, class YT, class AT>
__global__ void __launch_bounds__(SELL_WARPS * 32, 2)
    k_sell_spmv_g(DevSell<VT> A, const XT* __restrict__ x, const YT* __restrict__ f,
                  YT* __restrict__ y) {
  GBS_GRID_DEP();
  extern __shared__ __align__(128) unsigned char sell_smem[];
  SellStages<VT>& sm = reinterpret_cast<SellStages<VT>*>(sell_smem)[threadIdx.x >> 5];
  const int lane = threadIdx.x & 31;
  const int64_t nn = A.n / B;
  AT res[B];
  sell_pipe<VT, XT, AT>(A, x, B, (nn + 31) / 32, sm, [&](int64_t g, int c, AT acc) {
#pragma unroll
    for (int r = 0; r < B; ++r)
      if (r == c) res[r] = acc;
    if (c != B - 1) return;
    const int64_t node = sell_node(A, g, lane);
    if (node < 0) return;
    AT fv[B];
    if constexpr (MODE == SPMV_RESID) load_run<B, YT, AT, false>(f + node * B, fv);
    if constexpr (MODE == SPMV_ADD) load_run<B, YT, AT, false>(y + node * B, fv);
#pragma unroll
    for (int r = 0; r < B; ++r) {
      AT v = res[r];
      if constexpr (MODE == SPMV_RESID) v = fv[r] - v;
      if constexpr (MODE == SPMV_ADD) v = fv[r] + v;
      y[node * B + r] = (YT)v;
    }
  });
}

// xo = x + M (f - A x): one unit is a group of 32 nodes (its B slices), so
// each lane ends with the whole residual of its node for the B x B block.
template <int B, class VT, class XT, class AT, class OT = XT>
__global__ void __launch_bounds__(SELL_WARPS * 32, 2)
    k_sell_relax(DevSell<VT> A, const VT* __restrict__ M, const XT* __restrict__ f,
                 const XT* __restrict__ x, OT* __restrict__ xo) {
  GBS_GRID_DEP();
  extern __shared__ __align__(128) unsigned char sell_smem[];
  SellStages<VT>& sm = reinterpret_cast<SellStages<VT>*>(sell_smem)[threadIdx.x >> 5];
  const int lane = threadIdx.x & 31;
  const int64_t nn = A.n / B;
  AT res[B];
  sell_pipe<VT, XT, AT>(A, x, B, (nn + 31) / 32, sm, [&](int64_t g, int c, AT acc) {
#pragma unroll
    for (int r = 0; r < B; ++r)
      if (r == c) res[r] = acc;
    if (c != B - 1) return;
    const int64_t node = sell_node(A, g, lane);
    if (node < 0) return;
    AT fv[B], xv[B];
    load_run<B, XT, AT, false>(f + node * B, fv);
    load_run<B, XT, AT, false>(x + node * B, xv);
#pragma unroll
    for (int r = 0; r < B; ++r) res[r] = fv[r] - res[r];
#pragma unroll
    for (int r = 0; r < B; ++r) {
      AT mr[B];
      load_run<B, VT, AT, false>(M + node * (B * B) + r * B, mr);
      AT out = xv[r];
#pragma unroll
      for (int c2 = 0; c2 < B; ++c2) out += mr[c2] * res[c2];
      xo[node * B + r] = (OT)(XT)out;
    }
  });
}

// ---- direct variants (FP64 forms) ----
// With FP64 arithmetic the FP64 pipe, not the value stream, sets the pace
// on GB300: the staged kernels' shared memory limits a CTA pair per SM to
// 16 warps, too few to cover the pipe's latency, and they measured slower
// (C2 V-cycle 379 us staged, 358 us direct).  The direct kernels load each
// column straight from global memory, four columns in flight per lane, at
// up to 32 warps per SM.
//
// (Measured alternatives that lost: each lane loading one column's offset
// and mask once and the warp broadcasting them by shuffles, in batches of
// 8 columns -- C2 outer SpMV 43.7 us against 38.3; batches of 4 columns
// whose offset, value and x loads issue in order through volatile PTX --
// 40.3 us against 34.6 with one warp per 32-node group.)
template <class VT, class XT, class AT>
__device__ __forceinline__ AT sell_row_dot_direct(const DevSell<VT>& A, const XT* __restrict__ x, int q,
                                                  int lane, int64_t row) {
  const int k0 = __ldg(A.off + q), w = __ldg(A.off + q + 1) - k0;
  const VT* v = A.val + (size_t)k0 * 32 + lane;
  AT acc = AT(0);
  const int ci = __ldg(A.cinfo + q);
  if (ci < 0) {   // uniform slice: the gather address comes from the row
    const int2* u = A.uinfo + (-1 - ci);
#pragma unroll 4
    for (int k = 0; k < w; ++k) {
      const int2 om = __ldg(u + k);   // warp-uniform: one broadcast load
      const VT a = __ldcs(v + (size_t)k * 32);
      if (((unsigned)om.y >> lane) & 1u) acc += cvt<AT>(a) * cvt<AT>(__ldg(x + row + om.x));
    }
    return acc;
  }
  const int* c = A.col + (size_t)k0 * 32 + lane;
#pragma unroll 4
  for (int k = 0; k < w; ++k) {
    const int j = __ldcs(c + (size_t)k * 32);
    const VT a = __ldcs(v + (size_t)k * 32);
    if (j >= 0) acc += cvt<AT>(a) * cvt<AT>(__ldg(x + j));
  }
  return acc;
}
template <int MODE, class VT, class XT, class YT, class AT>
__global__ void __launch_bounds__(256, 4) k_sell_spmv_direct(DevSell<VT> A, const XT* __restrict__ x,
                                                        const YT* __restrict__ f,
                                                        YT* __restrict__ y) {
  GBS_GRID_DEP();
  const int64_t q = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  if (q >= A.nslices) return;
  const int lane = threadIdx.x & 31;
  const int g = (int)(q / A.B), c = (int)(q - (int64_t)g * A.B);
  const int64_t node = sell_node(A, g, lane);
  const int64_t row = (node < 0 ? 0 : node) * A.B + c;   // no entries in an empty lane
  const AT acc = sell_row_dot_direct<VT, XT, AT>(A, x, (int)q, lane, row);
  if (node < 0) return;
  if constexpr (MODE == SPMV_SET) y[row] = (YT)acc;
  else if constexpr (MODE == SPMV_RESID) y[row] = (YT)(cvt<AT>(f[row]) - acc);
  else y[row] = (YT)(cvt<AT>(y[row]) + acc);
}
// Direct (FP64) MODE SET / RESID / ADD with one warp per 32-node group and
// contiguous stores of each node's B rows (see k_sell_spmv_g).
template <int B, int MODE, class VT, class XT, class YT, class AT>
__global__ void __launch_bounds__(256, 4) k_sell_spmv_direct_g(DevSell<VT> A,
                                                          const XT* __restrict__ x,
                                                          const YT* __restrict__ f,
                                                          YT* __restrict__ y) {
  GBS_GRID_DEP();
  const int64_t g = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int nn = A.n / B;
  if (g * 32 >= nn) return;
  const int lane = threadIdx.x & 31;
  const int64_t node = sell_node(A, g, lane);
  const int64_t nd = node < 0 ? 0 : node;   // no entries in an empty lane
  AT res[B];
#pragma unroll
  for (int c = 0; c < B; ++c)
    res[c] = sell_row_dot_direct<VT, XT, AT>(A, x, (int)(g * B + c), lane, nd * B + c);
  if (node < 0) return;
  AT fv[B];
  if constexpr (MODE == SPMV_RESID) load_run<B, YT, AT, false>(f + node * B, fv);
  if constexpr (MODE == SPMV_ADD) load_run<B, YT, AT, false>(y + node * B, fv);
#pragma unroll
  for (int r = 0; r < B; ++r) {
    AT v = res[r];
    if constexpr (MODE == SPMV_RESID) v = fv[r] - v;
    if constexpr (MODE == SPMV_ADD) v = fv[r] + v;
    y[node * B + r] = (YT)v;
  }
}

template <int B, class VT, class XT, class AT, class OT = XT>
__global__ void __launch_bounds__(256, 4) k_sell_relax_direct(DevSell<VT> A, const VT* __restrict__ M,
                                                         const XT* __restrict__ f,
                                                         const XT* __restrict__ x,
                                                         OT* __restrict__ xo) {
  GBS_GRID_DEP();
  const int64_t g = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int nn = A.n / B;
  if (g * 32 >= nn) return;
  const int lane = threadIdx.x & 31;
  const int64_t node = sell_node(A, g, lane);
  const int64_t nd = node < 0 ? 0 : node;   // no entries in an empty lane
  AT res[B];
#pragma unroll
  for (int c = 0; c < B; ++c)
    res[c] = sell_row_dot_direct<VT, XT, AT>(A, x, (int)(g * B + c), lane, nd * B + c);
  if (node < 0) return;
  AT fv[B], xv[B];
  load_run<B, XT, AT, false>(f + node * B, fv);
  load_run<B, XT, AT, false>(x + node * B, xv);
#pragma unroll
  for (int c = 0; c < B; ++c) res[c] = fv[c] - res[c];
#pragma unroll
  for (int r = 0; r < B; ++r) {
    AT mr[B];
    load_run<B, VT, AT, false>(M + node * (B * B) + r * B, mr);
    AT out = xv[r];
#pragma unroll
    for (int c = 0; c < B; ++c) out += mr[c] * res[c];
    xo[node * B + r] = (OT)(XT)out;
  }
}
// Zero-guess pre-smoothing step fused with the residual (FP64 forms):
// x = M f and r = f - A x = f - (A M) f, with AM = A M precomputed on the
// level's slices, so no kernel has to wait for x.  One warp per 32-node
// group as in k_sell_relax_direct; each lane ends with its node's B rows
// of (A M) f and forms both outputs.
template <int B, class VT, class XT, class AT>
__global__ void __launch_bounds__(256, 4) k_sell_presmooth_direct(DevSell<VT> AM,
                                                             const VT* __restrict__ M,
                                                             const XT* __restrict__ f,
                                                             XT* __restrict__ x,
                                                             XT* __restrict__ r) {
  GBS_GRID_DEP();
  const int64_t g = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int nn = AM.n / B;
  if (g * 32 >= nn) return;
  const int lane = threadIdx.x & 31;
  const int64_t node = sell_node(AM, g, lane);
  const int64_t nd = node < 0 ? 0 : node;   // no entries in an empty lane
  AT amf[B];
#pragma unroll
  for (int c = 0; c < B; ++c)
    amf[c] = sell_row_dot_direct<VT, XT, AT>(AM, f, (int)(g * B + c), lane, nd * B + c);
  if (node < 0) return;
  AT fv[B];
  load_run<B, XT, AT, false>(f + node * B, fv);
#pragma unroll
  for (int rr = 0; rr < B; ++rr) {
    AT mr[B];
    load_run<B, VT, AT, false>(M + node * (B * B) + rr * B, mr);
    AT xo = AT(0);
#pragma unroll
    for (int c = 0; c < B; ++c) xo += mr[c] * fv[c];
    x[node * B + rr] = (XT)xo;
    r[node * B + rr] = (XT)(fv[rr] - amf[rr]);
  }
}

// Persistent pipelined launch: dynamic shared memory for the stages, as
// many CTAs as stay resident, at most cap.
template <class... KA, class... A>
inline void launch_sell(void (*fn)(KA...), size_t smem, int64_t cap, cudaStream_t s, A&&... a) {
  static std::mutex mu;
  {
    std::lock_guard<std::mutex> lock(mu);
    static std::map<const void*, bool> set;
    if (!set[(const void*)fn]) {
      // a failure here surfaces as a failed launch below
      if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) ==
          cudaSuccess)
        set[(const void*)fn] = true;
    }
  }
  const unsigned g = resident_grid((const void*)fn, (int)std::min<int64_t>(cap, 1 << 30),
                                   SELL_WARPS * 32, smem);
  ::gbs::launch_k(fn, g, SELL_WARPS * 32, smem, s, std::forward<A>(a)...);
}

}  // namespace gbs
