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

#include <cstdlib>
#include <type_traits>
#include <utility>

namespace gbs {

// ------------------------------------------- programmatic dependent launch
// The solve phase is a chain of short dependent kernels (about 40 a
// BiCGStab iteration, 80 a Schur application), and on the small and
// mixed-precision levels the gap between one kernel's last CTAs and the
// next one's first is a large part of each kernel's time.  Every kernel is
// launched with programmatic stream serialization (launch_k), so the next
// kernel in the stream may be scheduled while this one finishes; every
// kernel begins with GBS_GRID_DEP: griddepcontrol.wait, which returns once
// the preceding grid has completed and its writes are visible (at once when
// there is none), so no read or write moves ahead of its predecessor; then
// griddepcontrol.launch_dependents, which lets the following grid launch
// once every CTA of this one has started.  GBS_PDL=0 launches without the
// attribute (measurement).
#define GBS_GRID_DEP()                                           \
  do {                                                           \
    asm volatile("griddepcontrol.wait;" ::: "memory");           \
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); \
  } while (0)

inline bool pdl_enabled() {
  static const bool on = [] {
    const char* e = std::getenv("GBS_PDL");
    return !(e && e[0] == '0');
  }();
  return on;
}

// fn<<<grid, block, smem, s>>>(a...) with programmatic stream
// serialization, except while s is being captured into a CUDA graph: in a
// replayed graph the attribute measured slower (C2 BiCGStab iteration, FP64
// 23.5 -> 24.3 ms a solve, BF16 12.5 -> 14.0 ms), while stream launches gain
// (C3 GMRES, FP64 103 -> 98.5 ms, BF16 68.4 -> 63.7 ms).  Errors surface
// through cudaPeekAtLastError at the caller.
template <class... KA, class... A>
inline void launch_k(void (*fn)(KA...), dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                     A&&... a) {
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  if (pdl_enabled() && cudaStreamIsCapturing(s, &cs) != cudaSuccess) {
    (void)cudaGetLastError();
    cs = cudaStreamCaptureStatusActive;   // unknown: launch without the attribute
  }
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = pdl_enabled() && cs == cudaStreamCaptureStatusNone ? 1 : 0;
  (void)cudaLaunchKernelEx(&cfg, fn, std::forward<A>(a)...);
}

template <class VT>
struct DevBsr {
  int nbr = 0, nbc = 0;
  const int* rp = nullptr;
  const int* col = nullptr;
  const VT* val = nullptr;
  const int* tmap = nullptr;  // transpose map (may be null)
  int G = 0;                  // lanes per block row (0: one lane per scalar row)
  int S = 1;                  // G == 0: lanes sharing each scalar row (1, 2, 4, 8)
};


// Scalar CSR of a level whose blocks are mostly zeros (per-level format
// choice): n scalar rows, S lanes per scalar row.
template <class VT>
struct DevCsr {
  int n = 0;
  const int* rp = nullptr;
  const int* col = nullptr;
  const VT* val = nullptr;
  int S = 1;
  int G = 0;   // FP32/BF16 products: G lanes a row stream 16-byte chunks (0: S lanes a row)
};

// Sliced scalar CSR (see HSell and sell.cuh): slice q holds component
// q % B of the 32 nodes of group q / B, column-major, padded with column -1.
template <class VT>
struct DevSell {
  int n = 0, B = 1, nslices = 0;
  const int* off = nullptr;   // nslices + 1, in columns of 32 entries
  const int* col = nullptr;
  const VT* val = nullptr;
  double* err = nullptr;      // set to 1.0 by a kernel whose pipeline wait timed out
  long long wait = 1LL << 31; // bound of a pipeline wait, in SM clocks
  // uniform slices (HSell): cinfo[q] < 0, and entry k of lane i sits at
  // column row_i + uinfo[-1 - cinfo[q] + k].x when bit i of .y is set
  const int* cinfo = nullptr;
  const int2* uinfo = nullptr;
  bool uniform = false;       // every slice is uniform (a stencil operator)
  const int* node = nullptr;  // sorted form: node of each slot (-1: none); null: natural
};

// Node of lane `lane` of 32-node group g of a sliced operator, -1 if none.
template <class VT>
__device__ __forceinline__ int64_t sell_node(const DevSell<VT>& A, int64_t g, int lane) {
  const int64_t p = g * 32 + lane;
  if (A.node) return __ldg(A.node + p);
  return p < A.n / A.B ? p : -1;
}

// Block-row slices of a block level (HBSell): slice q holds R = 32 / B
// block rows, slot i of the slice is block row perm[q * R + i] (-1: none),
// and entry k of slot i is block (off[q] + k) * R + i.
template <class VT>
struct DevBSell {
  int nbr = 0, nslices = 0;
  const int* perm = nullptr;
  const int* off = nullptr;
  const int* col = nullptr;
  const VT* val = nullptr;
};

// Lanes per scalar CSR row.  Short rows keep one lane per row: that lane
// reuses its row's sectors from L1 on the next iterations, and wider splits
// measured slower on GB300 (C2: 28 ms with one lane, 37 ms with four).
inline int csr_split(int64_t n, int64_t nnz) {
  const double avg = n ? (double)nnz / n : 0.0;
  if (avg < 12.0) return 1;
  if (avg < 24.0) return 2;
  if (avg < 48.0) return 4;
  return 8;
}

// ---------------------------------------------------------------- conversions
__device__ __forceinline__ float to_f(float v) { return v; }
__device__ __forceinline__ float to_f(double v) { return (float)v; }
__device__ __forceinline__ float to_f(__nv_bfloat16 v) { return __bfloat162float(v); }
template <class AT, class T>
__device__ __forceinline__ AT cvt(T v);
template <> __device__ __forceinline__ int cvt<int, int>(int v) { return v; }
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

// Row split: S lanes share each scalar row (lane s of the row takes blocks
// k0+s, k0+s+S, ...), B*S lanes per block row, 32/(B*S) block rows per
// warp.  Their partial sums meet in a shuffle-down tree that costs one add
// per step, so long rows get S-fold parallelism for log2(S) extra adds.
template <int B, int S>
struct RowMapS {
  static constexpr int GL = B * S;
  static constexpr int RPW = 32 / GL;
  int brow, r, s, lane, base;
  bool lane_ok;
  __device__ __forceinline__ explicit RowMapS(int64_t gtid) {
    const int64_t warp = gtid >> 5;
    lane = (int)(gtid & 31);
    const int sub = lane / GL;
    const int q = lane - sub * GL;
    s = q / B;
    r = q - s * B;
    base = sub * GL;
    lane_ok = sub < RPW;
    brow = (int)(warp * RPW + sub);
  }
};

template <int B, int S>
inline int64_t row_threads_s(int nbr) {
  constexpr int RPW = 32 / (B * S);
  return (int64_t)((nbr + RPW - 1) / RPW) * 32;
}

// Sum over the S lanes of a row; the total lands in the s == 0 lane.  All
// 32 lanes must call it.
template <int B, int S, class AT>
__device__ __forceinline__ AT split_reduce(AT v) {
#pragma unroll
  for (int off = S / 2; off > 0; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off * B);
  return v;
}

// Row r of (A x) for block row `brow` (A x or A^T x through tmap), over
// the blocks k0 + s, k0 + s + S, ... of the row.
template <int B, bool TR, class VT, class XT, class AT, int S = 1>
__device__ __forceinline__ AT row_dot(const DevBsr<VT>& A, const XT* __restrict__ x, int brow,
                                      int r, int s = 0) {
  AT acc = AT(0);
  const int k0 = A.rp[brow], k1 = A.rp[brow + 1];
#pragma unroll 4
  for (int k = k0 + s; k < k1; k += S) {
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

// Geometry of the coalesced "chunk streaming" read of one block row.  The
// values of a block row are contiguous (nblk blocks of B*B values), so G
// lanes read them as consecutive CB-byte chunks: a warp instruction covers
// 32*CB contiguous bytes.  When a block is a power-of-two number LPB of
// chunks and G is a multiple of LPB, lane g always sees the same position
// p = g % LPB inside a block: a fixed run of E values belonging to row(s)
// p*E/B, so it needs only E (or B) entries of x and one or two partial sums.
// Otherwise (B = 3) lanes stream single values ("element" mode).
template <int B, class VT>
struct Geom {
  static constexpr int BB = B * B * (int)sizeof(VT);
  static constexpr int CB = BB % 16 == 0 ? 16 : (BB % 8 == 0 ? 8 : (BB % 4 == 0 ? 4 : (int)sizeof(VT)));
  static constexpr int E = CB / (int)sizeof(VT);   // values per chunk
  static constexpr int LPB = BB / CB;              // chunks per block
  static constexpr bool FIXED = CB == 16 && (LPB & (LPB - 1)) == 0 && LPB <= 8 &&
                                (E <= B ? B % E == 0 : E % B == 0);
  static constexpr int E16 = 16 / (int)sizeof(VT);  // values per aligned 16-byte chunk
  static constexpr int NR = E > B ? E / B : 1;     // rows touched by one chunk
  static constexpr int NX = E > B ? B : E;         // x entries one chunk needs
};

// Lanes per block row (0 = one lane per scalar row, no cross-lane sums).
// FP64 accumulation is bound by GB300's FP64 pipe (about 2 DFMA per clock
// per SM), where every cross-lane reduction adds log2(G)*B FP64 adds per
// lane: FP64 keeps one lane per scalar row whenever that gives enough
// threads, and uses lane groups only on short coarse levels.  FP32
// accumulation is not ALU-bound and uses coalesced lane groups sized by
// row length; a whole 256-thread CTA per row when there are few, very
// long rows.
// Row split S for one-lane-per-scalar-row levels: long rows are shared by
// S lanes (one FP add per reduction step).
// Small levels are latency-bound: a level with fewer than LANES_TARGET
// lanes (a quarter of the threads the 152 SMs hold) splits its rows
// further, as long as each lane keeps at least one block.  (Measured on
// C2: the level-2 prolongator, 8k lanes at S = 1, drops from 14 to 6 us at
// S = 8; the level-1 prolongator, 127k lanes, is slower at S = 2.)
constexpr int64_t LANES_TARGET = 152 * 512;
template <int B>
inline int choose_split(int64_t nbr, int64_t nnzb) {
  const double avg = nbr ? (double)nnzb / nbr : 0.0;
  int S = 1;
  if (avg >= 12.0) S = 2;
  if (avg >= 24.0) S = 4;
  if (avg >= 48.0) S = 8;
  while (S < 8 && B * S * 2 <= 32 && 2.0 * S <= avg && nbr * B * S < LANES_TARGET) S *= 2;
  while (S > 1 && B * S > 32) S >>= 1;
  return S;
}

template <int B, class VT, class AT>
inline int choose_group(int64_t nbr, int64_t nnzb) {
  using Gm = Geom<B, VT>;
  const double avg = nbr ? (double)nnzb / nbr : 0.0;
  const double chunks = avg * (Gm::FIXED ? Gm::LPB : B * B);
  if (sizeof(AT) == 8 || !Gm::FIXED) {
    // FP64 (pipe-bound) and 3x3 / scalar FP32-BF16 rows: one lane per
    // scalar row with a row split (choose_split); a CTA per row only for a
    // few very long rows (a CTA per row measured 3x slower than a warp per
    // row on the 2017-row level 2 of C2)
    if (nbr <= 1024 && avg >= 128.0) return 256;
    // a warp per scalar row for a small level of long rows, where eight
    // lanes a row (the widest split) leave the GPU mostly idle (C3's
    // 1579-row level-3 pressure operator, 325 entries a row)
    if (B == 1 && nbr * 8 < LANES_TARGET / 4 && avg >= 64.0) return 32;
    return 0;
  }
  // a CTA per row when a warp per row leaves the GPU mostly idle and each
  // row still has two chunks for every lane (C2's 86-row level-2
  // restriction: 11 CTAs at a warp per row)
  if (nbr * 32 < LANES_TARGET && chunks >= 512) return 256;
  if (chunks <= 48) return 8;
  if (chunks <= 96) return 16;
  if (chunks <= 768 || nbr > 4096) return 32;
  return 256;
}

// Forward (A x)_brow with G lanes per block row (G in {8, 16, 32}, or 256 =
// one CTA, in which case this returns per-warp partials: the caller
// finishes the reduction across warps).  All 32 lanes of the warp must
// call it; inactive groups pass ok = false.  On return every lane of the
// group (warp) holds the complete B-vector.
template <int B, int G, class VT, class XT, class AT>
__device__ __forceinline__ void group_row_fwd(const DevBsr<VT>& A, const XT* __restrict__ x,
                                              int brow, int g, bool ok, AT (&acc)[B]) {
  using Gm = Geom<B, VT>;
#pragma unroll
  for (int r = 0; r < B; ++r) acc[r] = AT(0);
  if (ok) {
    const int k0 = A.rp[brow], k1 = A.rp[brow + 1];
    const VT* __restrict__ vrow = A.val + (size_t)k0 * (B * B);
    if constexpr (Gm::FIXED) {
      const int p = g % Gm::LPB;
      const int e0 = p * Gm::E;               // first value of the chunk in the block
      const int r0 = e0 / B;
      const int c0 = Gm::E <= B ? e0 % B : 0;
      AT part[Gm::NR];
#pragma unroll
      for (int q = 0; q < Gm::NR; ++q) part[q] = AT(0);
      const int nch = (k1 - k0) * Gm::LPB;
      // U chunks per batch: all index and value loads of a batch are issued
      // before the dependent x gathers, so each lane keeps 2U loads in flight.
      constexpr int U = 4;
      for (int cb = g; cb < nch; cb += U * G) {
        // out-of-range slots re-read the row's last chunk (always valid:
        // nch > 0 here) and are masked at the FMA, so no load is predicated
        int cc[U], j[U];
        AT v[U][Gm::E];
#pragma unroll
        for (int u = 0; u < U; ++u) cc[u] = min(cb + u * G, nch - 1);
#pragma unroll
        for (int u = 0; u < U; ++u) j[u] = __ldg(A.col + k0 + cc[u] / Gm::LPB);
#pragma unroll
        for (int u = 0; u < U; ++u) load_run<Gm::E, VT, AT, true>(vrow + (size_t)cc[u] * Gm::E, v[u]);
#pragma unroll
        for (int u = 0; u < U; ++u) {
          AT xv[Gm::NX];
          load_run<Gm::NX, XT, AT, false>(x + (size_t)j[u] * B + c0, xv);
          if (cb + u * G < nch) {
#pragma unroll
            for (int q = 0; q < Gm::NR; ++q)
#pragma unroll
              for (int e = 0; e < Gm::NX; ++e) part[q] += v[u][q * Gm::NX + e] * xv[e];
          }
        }
      }
#pragma unroll
      for (int r = 0; r < B; ++r)
#pragma unroll
        for (int q = 0; q < Gm::NR; ++q)
          if (r == r0 + q) acc[r] += part[q];
    } else {
      // Aligned-chunk streaming (B = 3, or blocks smaller than 16 bytes):
      // lanes take the 16-byte-aligned chunks of the global value array that
      // overlap this row's values [e0, e1) and skip the values outside it.
      // Element indices fit in int32 (checked at upload: nnzb*B*B < 2^31).
      constexpr int BB = B * B;
      constexpr int EC = Gm::E16;
      const int e0 = k0 * BB, e1 = k1 * BB;
      const int cfirst = e0 / EC, clast = (e1 - 1) / EC;
      constexpr int U = 2;
      for (int cb = cfirst + g; cb <= clast; cb += U * G) {
        AT v[U][EC];
        int cc[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
          cc[u] = min(cb + u * G, clast);
          load_run<EC, VT, AT, true>(A.val + (size_t)cc[u] * EC, v[u]);
        }
        if constexpr (B == 1) {
          // scalar CSR: the chunk's EC column indices are contiguous too
          int j[U][EC];
#pragma unroll
          for (int u = 0; u < U; ++u) load_run<EC, int, int, false>(A.col + (size_t)cc[u] * EC, j[u]);
#pragma unroll
          for (int u = 0; u < U; ++u) {
            if (cb + u * G > clast) continue;
#pragma unroll
            for (int q = 0; q < EC; ++q) {
              const int e = cc[u] * EC + q;
              const AT xv = cvt<AT>(__ldg(x + j[u][q]));
              if (e >= e0 && e < e1) acc[0] += v[u][q] * xv;
            }
          }
        } else if constexpr (EC <= BB) {
          // a chunk spans at most two blocks: fetch both blocks' x once
#pragma unroll
          for (int u = 0; u < U; ++u) {
            if (cb + u * G > clast) continue;
            const int ef = cc[u] * EC;
            const int kba = ef / BB;
            const int kbb = min((ef + EC - 1) / BB, k1 - 1);
            AT xa[B], xb[B];
            load_run<B, XT, AT, false>(x + (size_t)__ldg(A.col + max(kba, k0)) * B, xa);
            load_run<B, XT, AT, false>(x + (size_t)__ldg(A.col + kbb) * B, xb);
#pragma unroll
            for (int q = 0; q < EC; ++q) {
              const int e = ef + q;
              const int kb = e / BB;
              const int w = e - kb * BB;
              const int r = w / B, c = w - r * B;
              AT xv = AT(0);
#pragma unroll
              for (int t = 0; t < B; ++t)
                if (t == c) xv = (kb == kba) ? xa[t] : xb[t];
              const AT pv = (e >= e0 && e < e1) ? v[u][q] * xv : AT(0);
#pragma unroll
              for (int t = 0; t < B; ++t)
                if (t == r) acc[t] += pv;
            }
          }
        } else {
#pragma unroll
          for (int u = 0; u < U; ++u) {
            if (cb + u * G > clast) continue;
#pragma unroll
            for (int q = 0; q < EC; ++q) {
              const int e = cc[u] * EC + q;
              if (e < e0 || e >= e1) continue;
              const int kb = e / BB;
              const int w = e - kb * BB;
              const int r = w / B, c = w - r * B;
              const int j = __ldg(A.col + kb);
              const AT pv = v[u][q] * cvt<AT>(__ldg(x + (size_t)j * B + c));
#pragma unroll
              for (int t = 0; t < B; ++t)
                if (t == r) acc[t] += pv;
            }
          }
        }
      }
    }
  }
  constexpr int W = G < 32 ? G : 32;
#pragma unroll
  for (int o = W / 2; o > 0; o >>= 1)
#pragma unroll
    for (int r = 0; r < B; ++r) acc[r] += __shfl_xor_sync(0xffffffffu, acc[r], o);
}

// Transposed (A^T x)_brow through the transpose map: lane g takes whole
// blocks k0+g, k0+g+G, ... and reads block tmap[k] transposed.  Used by
// the adjoint only.  Same calling rules as group_row_fwd.
template <int B, int G, class VT, class XT, class AT>
__device__ __forceinline__ void group_row_tr(const DevBsr<VT>& A, const XT* __restrict__ x,
                                             int brow, int g, bool ok, AT (&acc)[B]) {
#pragma unroll
  for (int r = 0; r < B; ++r) acc[r] = AT(0);
  if (ok) {
    const int k0 = A.rp[brow], k1 = A.rp[brow + 1];
    for (int k = k0 + g; k < k1; k += G) {
      const int j = __ldg(A.col + k);
      const int kb = __ldg(A.tmap + k);
      AT a[B * B], xv[B];
      load_run<B * B, VT, AT, true>(A.val + (size_t)kb * (B * B), a);
      load_run<B, XT, AT, false>(x + (size_t)j * B, xv);
#pragma unroll
      for (int r = 0; r < B; ++r)
#pragma unroll
        for (int c = 0; c < B; ++c) acc[r] += a[c * B + r] * xv[c];
    }
  }
  constexpr int W = G < 32 ? G : 32;
#pragma unroll
  for (int o = W / 2; o > 0; o >>= 1)
#pragma unroll
    for (int r = 0; r < B; ++r) acc[r] += __shfl_xor_sync(0xffffffffu, acc[r], o);
}

template <int B, int G, bool TR, class VT, class XT, class AT>
__device__ __forceinline__ void group_row(const DevBsr<VT>& A, const XT* __restrict__ x, int brow,
                                          int g, bool ok, AT (&acc)[B]) {
  if constexpr (TR) group_row_tr<B, G, VT, XT, AT>(A, x, brow, g, ok, acc);
  else group_row_fwd<B, G, VT, XT, AT>(A, x, brow, g, ok, acc);
  if constexpr (G > 32) {
    // one CTA per block row: combine the per-warp sums
    __shared__ AT red[G / 32][B];
    const int w = threadIdx.x >> 5;
    if ((threadIdx.x & 31) == 0) {
#pragma unroll
      for (int r = 0; r < B; ++r) red[w][r] = acc[r];
    }
    __syncthreads();
#pragma unroll
    for (int r = 0; r < B; ++r) {
      AT t = AT(0);
#pragma unroll
      for (int q = 0; q < G / 32; ++q) t += red[q][r];
      acc[r] = t;
    }
  }
}

template <int B, class AT>
__device__ __forceinline__ AT pick(const AT (&v)[B], int r) {
  AT out = v[0];
#pragma unroll
  for (int q = 1; q < B; ++q)
    if (q == r) out = v[q];
  return out;
}

// ------------------------------------------------------------------ kernels
enum { SPMV_SET = 0, SPMV_RESID = 1, SPMV_ADD = 2 };

// MODE SET: y = A x;  RESID: y = f - A x;  ADD: y += A x.  One lane per
// scalar row, or S lanes per scalar row (row split).
template <int B, int S, bool TR, int MODE, class VT, class XT, class YT, class AT>
__global__ void __launch_bounds__(256, 4) k_spmv(DevBsr<VT> A, const XT* __restrict__ x,
                                              const YT* __restrict__ f, YT* __restrict__ y) {
  GBS_GRID_DEP();
  RowMapS<B, S> m(blockIdx.x * (int64_t)blockDim.x + threadIdx.x);
  const bool ok = m.lane_ok && m.brow < A.nbr;
  AT acc = ok ? row_dot<B, TR, VT, XT, AT, S>(A, x, m.brow, m.r, m.s) : AT(0);
  if constexpr (S > 1) acc = split_reduce<B, S, AT>(acc);
  if (!ok || m.s != 0) return;
  const size_t o = (size_t)m.brow * B + m.r;
  if constexpr (MODE == SPMV_SET) y[o] = (YT)acc;
  else if constexpr (MODE == SPMV_RESID) y[o] = (YT)(cvt<AT>(f[o]) - acc);
  else y[o] = (YT)(cvt<AT>(y[o]) + acc);
}

// Wide variant of k_spmv (G lanes per block row).
template <int B, int G, bool TR, int MODE, class VT, class XT, class YT, class AT>
__global__ void __launch_bounds__(256, 4) k_spmv_w(DevBsr<VT> A, const XT* __restrict__ x,
                                                const YT* __restrict__ f, YT* __restrict__ y) {
  GBS_GRID_DEP();
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int brow = (int)(t / G);
  const int g = (int)(t % G);
  const bool ok = brow < A.nbr;
  AT acc[B];
  group_row<B, G, TR, VT, XT, AT>(A, x, brow, g, ok, acc);
  if (!ok || g >= B) return;
  const size_t o = (size_t)brow * B + g;
  const AT v = pick<B, AT>(acc, g);
  if constexpr (MODE == SPMV_SET) y[o] = (YT)v;
  else if constexpr (MODE == SPMV_RESID) y[o] = (YT)(cvt<AT>(f[o]) - v);
  else y[o] = (YT)(cvt<AT>(y[o]) + v);
}

// Wide variant of k_relax.
template <int B, int G, bool TR, class VT, class XT, class AT>
__global__ void __launch_bounds__(256, 4) k_relax_w(DevBsr<VT> A, const VT* __restrict__ M,
                                                 const XT* __restrict__ f,
                                                 const XT* __restrict__ x, XT* __restrict__ xo) {
  GBS_GRID_DEP();
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int brow = (int)(t / G);
  const int g = (int)(t % G);
  const bool ok = brow < A.nbr;
  AT acc[B];
  group_row<B, G, TR, VT, XT, AT>(A, x, brow, g, ok, acc);
  if (!ok || g >= B) return;
  AT fv[B];
  load_run<B, XT, AT, false>(f + (size_t)brow * B, fv);
  AT mr[B];
  if constexpr (!TR) load_run<B, VT, AT, false>(M + (size_t)brow * (B * B) + g * B, mr);
  else load_col<B, VT, AT>(M + (size_t)brow * (B * B), g, mr);
  const size_t o = (size_t)brow * B + g;
  AT out = cvt<AT>(x[o]);
#pragma unroll
  for (int c = 0; c < B; ++c) out += mr[c] * (fv[c] - acc[c]);
  xo[o] = (XT)out;
}

// xo = x + M (f - A x)   (one relaxation sweep; M^T, A^T when TR).  One
// lane per scalar row or S lanes per scalar row.
template <int B, int S, bool TR, class VT, class XT, class AT>
__global__ void __launch_bounds__(256, 4) k_relax(DevBsr<VT> A, const VT* __restrict__ M,
                                               const XT* __restrict__ f,
                                               const XT* __restrict__ x, XT* __restrict__ xo) {
  GBS_GRID_DEP();
  RowMapS<B, S> m(blockIdx.x * (int64_t)blockDim.x + threadIdx.x);
  const bool ok = m.lane_ok && m.brow < A.nbr;
  const size_t o = (size_t)m.brow * B + m.r;
  AT acc = ok ? row_dot<B, TR, VT, XT, AT, S>(A, x, m.brow, m.r, m.s) : AT(0);
  if constexpr (S > 1) acc = split_reduce<B, S, AT>(acc);
  const AT res = (ok && m.s == 0) ? cvt<AT>(f[o]) - acc : AT(0);
  AT rb[B];
#pragma unroll
  for (int c = 0; c < B; ++c) rb[c] = __shfl_sync(0xffffffffu, res, (m.base + c) & 31);
  if (!ok || m.s != 0) return;
  AT mr[B];
  if constexpr (!TR) load_run<B, VT, AT, false>(M + (size_t)m.brow * (B * B) + m.r * B, mr);
  else load_col<B, VT, AT>(M + (size_t)m.brow * (B * B), m.r, mr);
  AT out = cvt<AT>(x[o]);
#pragma unroll
  for (int c = 0; c < B; ++c) out += mr[c] * rb[c];
  xo[o] = (XT)out;
}

// ------------------------------------------------------- block-row slices
// One warp per slice, one lane per scalar row: lane (slot, r) sums row r of
// its slot's blocks.  The rows of a slice have nearly equal lengths (sorted
// at setup), so few lanes idle, and no lane shares a row, so there are no
// cross-lane sums: every FP64 instruction is an FMA of the product.  Entry
// k of the slice's R slots is R consecutive blocks, so a warp's value load
// reads R * B * B contiguous values.
// Loads in issue order (volatile PTX keeps them in program order, so a
// batch of entries puts all its loads in flight before the first use; the
// compiler otherwise sinks each load to its use -- measured on the FP64
// block slices: 38 long-scoreboard stalls per issue, FP64 pipe 78% busy).
__device__ __forceinline__ int ld_nc_s32(const int* p) {
  int v;
  asm volatile("ld.global.nc.s32 %0, [%1];" : "=r"(v) : "l"(p));
  return v;
}
__device__ __forceinline__ double ld_nc_f64(const double* p) {
  double v;
  asm volatile("ld.global.nc.f64 %0, [%1];" : "=d"(v) : "l"(p));
  return v;
}
__device__ __forceinline__ double ld_cs_f64(const double* p) {
  double v;
  asm volatile("ld.global.cs.f64 %0, [%1];" : "=d"(v) : "l"(p));
  return v;
}
__device__ __forceinline__ void ld_nc_v2f64(const double* p, double& a, double& b) {
  asm volatile("ld.global.nc.v2.f64 {%0, %1}, [%2];" : "=d"(a), "=d"(b) : "l"(p));
}
__device__ __forceinline__ void ld_cs_v2f64(const double* p, double& a, double& b) {
  asm volatile("ld.global.cs.v2.f64 {%0, %1}, [%2];" : "=d"(a), "=d"(b) : "l"(p));
}
// B consecutive doubles at p (16-byte aligned when B is even).
template <int B, bool CS>
__device__ __forceinline__ void ld_run_f64(const double* p, double (&o)[B]) {
  if constexpr (B % 2 == 0) {
#pragma unroll
    for (int e = 0; e < B; e += 2) {
      if constexpr (CS) ld_cs_v2f64(p + e, o[e], o[e + 1]);
      else ld_nc_v2f64(p + e, o[e], o[e + 1]);
    }
  } else {
#pragma unroll
    for (int e = 0; e < B; ++e) o[e] = CS ? ld_cs_f64(p + e) : ld_nc_f64(p + e);
  }
}

// FP64 block slices: row r of slot `slot` of slice q times x, in batches of
// U entries whose column, value and x loads all issue before the FMAs.  U
// keeps the kernels within 64 registers, so that every slice's warp is
// resident at once on the levels that take slices (4 CTAs of 256 threads
// per SM; without a minimum the compiler caps them at 32 registers and
// serialises the loads).
template <int B>
__device__ __forceinline__ double bsell_row_dot_f64(const int* __restrict__ off,
                                                    const int* __restrict__ col,
                                                    const double* __restrict__ val,
                                                    const double* __restrict__ x, int q, int slot,
                                                    int r) {
  constexpr int R = 32 / B;
  constexpr int U = B >= 3 ? 2 : 8 / B;
  const int k0 = __ldg(off + q), w = __ldg(off + q + 1) - k0;
  const int* __restrict__ c = col + (size_t)k0 * R + slot;
  const double* __restrict__ v = val + ((size_t)k0 * R + slot) * (B * B) + r * B;
  double acc = 0.0;
  // the next batch's columns load one batch ahead, so a batch's x gathers
  // wait on one memory round trip instead of two (column, then x)
  int jn[U];
#pragma unroll
  for (int u = 0; u < U; ++u) jn[u] = ld_nc_s32(c + (size_t)min(u, w - 1) * R);
  for (int k = 0; k < w; k += U) {
    int j[U];
    double a[U][B], xv[U][B];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      j[u] = jn[u];
      jn[u] = ld_nc_s32(c + (size_t)min(k + U + u, w - 1) * R);
    }
#pragma unroll
    for (int u = 0; u < U; ++u) ld_run_f64<B, true>(v + (size_t)min(k + u, w - 1) * (R * B * B), a[u]);
#pragma unroll
    for (int u = 0; u < U; ++u) ld_run_f64<B, false>(x + (size_t)j[u] * B, xv[u]);
#pragma unroll
    for (int u = 0; u < U; ++u)
      if (k + u < w) {
#pragma unroll
        for (int cc = 0; cc < B; ++cc) acc += a[u][cc] * xv[u][cc];
      }
  }
  return acc;
}

template <int B, class VT, class XT, class AT>
__device__ __forceinline__ AT bsell_row_dot(const DevBSell<VT>& A, const XT* __restrict__ x, int q,
                                            int slot, int r) {
  constexpr int R = 32 / B;
  const int k0 = __ldg(A.off + q), w = __ldg(A.off + q + 1) - k0;
  const int* __restrict__ c = A.col + (size_t)k0 * R + slot;
  const VT* __restrict__ v = A.val + ((size_t)k0 * R + slot) * (B * B) + r * B;
  AT acc = AT(0);
  if constexpr (std::is_same<VT, double>::value && std::is_same<XT, double>::value) {
    return bsell_row_dot_f64<B>(A.off, A.col, A.val, x, q, slot, r);
  }
  // U entries per batch: all column and value loads of a batch issue before
  // the dependent x gathers.  Entries past the slice's width re-read its
  // last entry and are dropped at the FMA (w is warp-uniform: no divergence).
  constexpr int U = 4;
  for (int k = 0; k < w; k += U) {
    int j[U];
    AT a[U][B];
#pragma unroll
    for (int u = 0; u < U; ++u) j[u] = __ldg(c + (size_t)min(k + u, w - 1) * R);
#pragma unroll
    for (int u = 0; u < U; ++u)
      load_run<B, VT, AT, true>(v + (size_t)min(k + u, w - 1) * (R * B * B), a[u]);
#pragma unroll
    for (int u = 0; u < U; ++u) {
      AT xv[B];
      load_run<B, XT, AT, false>(x + (size_t)j[u] * B, xv);
      if (k + u < w) {
#pragma unroll
        for (int cc = 0; cc < B; ++cc) acc += a[u][cc] * xv[cc];
      }
    }
  }
  return acc;
}

// MODE SET / RESID / ADD on a level in block-row slices.
template <int B, int MODE, class VT, class XT, class YT, class AT>
__global__ void __launch_bounds__(256, 4) k_bsell_spmv(DevBSell<VT> A, const XT* __restrict__ x,
                                                     const YT* __restrict__ f, YT* __restrict__ y) {
  GBS_GRID_DEP();
  constexpr int R = 32 / B;
  const int64_t q = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  if (q >= A.nslices) return;
  const int lane = threadIdx.x & 31;
  const int slot = lane / B, r = lane - slot * B;
  if (slot >= R) return;   // B = 3: lanes 30 and 31 hold no row
  const int row = __ldg(A.perm + q * R + slot);
  const AT acc = bsell_row_dot<B, VT, XT, AT>(A, x, (int)q, slot, r);
  if (row < 0) return;
  const size_t o = (size_t)row * B + r;
  if constexpr (MODE == SPMV_SET) y[o] = (YT)acc;
  else if constexpr (MODE == SPMV_RESID) y[o] = (YT)(cvt<AT>(f[o]) - acc);
  else y[o] = (YT)(cvt<AT>(y[o]) + acc);
}

// xo = x + M (f - A x) on a level in block-row slices: the B lanes of a
// slot exchange their residuals by shuffles for the B x B block of M.
template <int B, class VT, class XT, class AT>
__global__ void __launch_bounds__(256, 4) k_bsell_relax(DevBSell<VT> A, const VT* __restrict__ M,
                                                      const XT* __restrict__ f,
                                                      const XT* __restrict__ x,
                                                      XT* __restrict__ xo) {
  GBS_GRID_DEP();
  constexpr int R = 32 / B;
  const int64_t q = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  if (q >= A.nslices) return;   // warp-uniform
  const int lane = threadIdx.x & 31;
  const int slot0 = lane / B;
  const bool lane_ok = slot0 < R;
  const int slot = lane_ok ? slot0 : R - 1;   // B = 3: lanes 30, 31 shadow slot R - 1
  const int r = lane_ok ? lane - slot * B : 0;
  const int row = __ldg(A.perm + q * R + slot);
  const AT acc = bsell_row_dot<B, VT, XT, AT>(A, x, (int)q, slot, r);
  const size_t o = (size_t)(row < 0 ? 0 : row) * B + r;
  const AT res = row >= 0 ? cvt<AT>(f[o]) - acc : AT(0);
  AT rb[B];
#pragma unroll
  for (int c = 0; c < B; ++c) rb[c] = __shfl_sync(0xffffffffu, res, slot * B + c);
  if (!lane_ok || row < 0) return;
  AT mr[B];
  load_run<B, VT, AT, false>(M + (size_t)row * (B * B) + r * B, mr);
  AT out = cvt<AT>(x[o]);
#pragma unroll
  for (int c = 0; c < B; ++c) out += mr[c] * rb[c];
  xo[o] = (XT)out;
}

// Zero-guess pre-smoothing step fused with the residual on a level in
// block-row slices: x = M f and r = f - (A M) f (AM = A M precomputed on
// the slices).  Each lane forms its own row of both outputs; no shuffles.
template <int B, class VT, class XT, class AT>
__global__ void __launch_bounds__(256, 4) k_bsell_presmooth(DevBSell<VT> AM, const VT* __restrict__ M,
                                                          const XT* __restrict__ f,
                                                          XT* __restrict__ x, XT* __restrict__ r) {
  GBS_GRID_DEP();
  constexpr int R = 32 / B;
  const int64_t q = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  if (q >= AM.nslices) return;
  const int lane = threadIdx.x & 31;
  const int slot = lane / B, rr = lane - slot * B;
  if (slot >= R) return;
  const int row = __ldg(AM.perm + q * R + slot);
  const AT acc = bsell_row_dot<B, VT, XT, AT>(AM, f, (int)q, slot, rr);
  if (row < 0) return;
  AT fv[B], mr[B];
  load_run<B, XT, AT, false>(f + (size_t)row * B, fv);
  load_run<B, VT, AT, false>(M + (size_t)row * (B * B) + rr * B, mr);
  AT xo = AT(0);
#pragma unroll
  for (int c = 0; c < B; ++c) xo += mr[c] * fv[c];
  const size_t o = (size_t)row * B + rr;
  x[o] = (XT)xo;
  r[o] = (XT)(cvt<AT>(f[o]) - acc);
}

// ------------------------------------------------------- scalar CSR levels
template <int S, class VT, class XT, class AT>
__device__ __forceinline__ AT csr_row_dot(const DevCsr<VT>& A, const XT* __restrict__ x, int row,
                                          int s) {
  AT acc = AT(0);
  const int k0 = A.rp[row], k1 = A.rp[row + 1];
#pragma unroll 4
  for (int k = k0 + s; k < k1; k += S)
    acc += cvt<AT>(__ldcs(A.val + k)) * cvt<AT>(__ldg(x + __ldg(A.col + k)));
  return acc;
}

// MODE SET / RESID / ADD on a scalar CSR level; S lanes per scalar row.
template <int S, int MODE, class VT, class XT, class YT, class AT>
__global__ void __launch_bounds__(256, 4) k_csr_spmv(DevCsr<VT> A, const XT* __restrict__ x,
                                                  const YT* __restrict__ f, YT* __restrict__ y) {
  GBS_GRID_DEP();
  RowMapS<1, S> m(blockIdx.x * (int64_t)blockDim.x + threadIdx.x);
  const bool ok = m.lane_ok && m.brow < A.n;
  AT acc = ok ? csr_row_dot<S, VT, XT, AT>(A, x, m.brow, m.s) : AT(0);
  if constexpr (S > 1) acc = split_reduce<1, S, AT>(acc);
  if (!ok || m.s != 0) return;
  const size_t o = (size_t)m.brow;
  if constexpr (MODE == SPMV_SET) y[o] = (YT)acc;
  else if constexpr (MODE == SPMV_RESID) y[o] = (YT)(cvt<AT>(f[o]) - acc);
  else y[o] = (YT)(cvt<AT>(y[o]) + acc);
}

// xo = x + M (f - A x) with A in scalar CSR and M in B x B blocks: the B
// scalar rows of a node (each over S lanes) meet by shuffles for M.
template <int B, int S, class VT, class XT, class AT>
__global__ void __launch_bounds__(256, 4) k_csr_relax(DevCsr<VT> A, const VT* __restrict__ M,
                                                   const XT* __restrict__ f,
                                                   const XT* __restrict__ x,
                                                   XT* __restrict__ xo) {
  GBS_GRID_DEP();
  RowMapS<B, S> m(blockIdx.x * (int64_t)blockDim.x + threadIdx.x);
  const int nnodes = A.n / B;
  const bool ok = m.lane_ok && m.brow < nnodes;
  const int row = m.brow * B + m.r;
  AT acc = ok ? csr_row_dot<S, VT, XT, AT>(A, x, row, m.s) : AT(0);
  if constexpr (S > 1) acc = split_reduce<B, S, AT>(acc);
  const AT res = (ok && m.s == 0) ? cvt<AT>(f[row]) - acc : AT(0);
  AT rb[B];
#pragma unroll
  for (int c = 0; c < B; ++c) rb[c] = __shfl_sync(0xffffffffu, res, (m.base + c) & 31);
  if (!ok || m.s != 0) return;
  AT mr[B];
  load_run<B, VT, AT, false>(M + (size_t)m.brow * (B * B) + m.r * B, mr);
  AT out = cvt<AT>(x[row]);
#pragma unroll
  for (int c = 0; c < B; ++c) out += mr[c] * rb[c];
  xo[row] = (XT)out;
}

// x = M f   (zero-guess smoothing step).
template <int B, bool TR, class VT, class XT, class AT>
__global__ void __launch_bounds__(256, 4) k_mapply(int nbr, const VT* __restrict__ M,
                                                const XT* __restrict__ f, XT* __restrict__ x) {
  GBS_GRID_DEP();
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

// The zero-guess smoothing step of a mixed form's finest level with the
// FP64 -> FP32 precision boundary folded in: fin = (XT) r, rounded to
// nearest even as the separate cast would, and x = M fin (M^T when TR),
// in one pass over r.
template <int B, bool TR, class VT, class XT, class AT>
__global__ void __launch_bounds__(256, 4) k_cast_mapply(int nbr, const VT* __restrict__ M,
                                                     const double* __restrict__ r,
                                                     XT* __restrict__ fin, XT* __restrict__ x) {
  GBS_GRID_DEP();
  RowMap<B> m(blockIdx.x * (int64_t)blockDim.x + threadIdx.x);
  if ((int64_t)(blockIdx.x * (int64_t)blockDim.x + threadIdx.x - (threadIdx.x & 31)) / 32 *
          RowMap<B>::RPW >= nbr)
    return;   // the whole warp is past the last row
  const bool ok = m.lane_ok && m.brow < nbr;
  const size_t o = (size_t)m.brow * B + m.r;
  // each lane reads its own entry; the node's B entries meet by shuffles
  const XT ri = ok ? (XT)r[o] : XT(0);
  AT fv[B], mr[B];
#pragma unroll
  for (int c = 0; c < B; ++c) fv[c] = cvt<AT>(__shfl_sync(0xffffffffu, ri, (m.base + c) & 31));
  if (!ok) return;
  if constexpr (!TR) load_run<B, VT, AT, false>(M + (size_t)m.brow * (B * B) + m.r * B, mr);
  else load_col<B, VT, AT>(M + (size_t)m.brow * (B * B), m.r, mr);
  AT out = AT(0);
#pragma unroll
  for (int c = 0; c < B; ++c) out += mr[c] * fv[c];
  fin[o] = ri;
  x[o] = (XT)out;
}

// x = Ainv f, dense n x n row-major, one warp per row.
template <class VT, class XT, class AT>
__global__ void __launch_bounds__(256, 4) k_gemv(int n, const VT* __restrict__ Ainv,
                                              const XT* __restrict__ f, XT* __restrict__ x) {
  GBS_GRID_DEP();
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
  GBS_GRID_DEP();
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    out[i] = (TO)cvt<float>(in[i]);
}
template <>
__global__ void k_cast<double, double>(int64_t n, const double* __restrict__ in,
                                       double* __restrict__ out) {
  GBS_GRID_DEP();
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    out[i] = in[i];
}
template <>
__global__ void k_cast<float, double>(int64_t n, const float* __restrict__ in,
                                      double* __restrict__ out) {
  GBS_GRID_DEP();
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    out[i] = (double)in[i];
}

// out = s .* in (ILUT: scaling by D^-1).
template <class VT, class ST>
__global__ void k_vscale(int64_t n, const VT* __restrict__ sc, const ST* __restrict__ in,
                         ST* __restrict__ out) {
  GBS_GRID_DEP();
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    out[i] = cvt<ST>(sc[i]) * in[i];
}

// out = x + w z (x null: out = w z).
template <class ST>
__global__ void k_vaxpy(int64_t n, const ST* __restrict__ x, ST w, const ST* __restrict__ z,
                        ST* __restrict__ out) {
  GBS_GRID_DEP();
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    out[i] = x ? x[i] + w * z[i] : w * z[i];
}

inline unsigned grid_for(int64_t threads, int tpb = 256) {
  int64_t g = (threads + tpb - 1) / tpb;
  return (unsigned)(g < 1 ? 1 : g);
}

}  // namespace gbs
