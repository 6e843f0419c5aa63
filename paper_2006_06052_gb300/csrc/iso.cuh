// Levels whose blocks are scalar multiples of the identity.
//
// When every stored block of a level operator is a_ij * I_B -- the
// velocity block of a Stokes system with a scalar viscosity, whose B
// components share every stencil coefficient, and therefore every
// smoothed-aggregation level built from it (P_tent is identity blocks,
// and products and inverses of a_ij * I_B blocks stay of that form) --
// the operator is S (x) I_B for a scalar matrix S.  Such a level is
// stored as S: one value and one column per block, where the scalar CSR
// of the nonzeros stores B of each and the block form B*B values.  The
// smoother is diag(m) (x) I_B, one value per node.
//
// This is a storage form of the statically sized 3x3 velocity blocks of
// the paper's Section 4 (Listing V3) without their zeros and repeats; the
// primitives are those of Section 2.3 (residual, relaxation, restriction,
// prolongation).  A scalar level (B = 1) is S (x) I_1 and takes the same
// kernels with NV = 1.
//
// One lane owns one node (row of S) and applies the row to the node's B
// interleaved components at once: each value is loaded once for B FMAs,
// the B gathered x entries of a column are adjacent, and the node's B
// outputs are formed and stored by the same lane.  The arithmetic per
// output is the block form's with the zero terms left out, so results
// agree with it to rounding order.  Rows of S run one lane each in 32-node
// slices, or with S lanes (up to a warp) or a 256-thread CTA per row in
// plain CSR, sized to the level (set_iso_lanes).
#pragma once

#include "kernels.cuh"

namespace gbs {

// x[j*NV .. j*NV + NV - 1] as AT.
template <int NV, class XT, class AT>
__device__ __forceinline__ void iso_gather(const XT* __restrict__ x, int64_t j, AT (&o)[NV]) {
  load_run<NV, XT, AT, false>(x + j * NV, o);
}

// Row `row` of S over the entries k0 + s, k0 + s + S, ... times the NV
// components of x.
// BATCH: entries go in batches of U per lane -- their column and value
// loads, then their x gathers, all issue before the FMAs (entries past the
// row's end re-read its last entry and are dropped at the FMA); for FP32
// accumulation and for small, latency-bound levels.  Large FP64 levels,
// bound by the FP64 pipe, keep the plain loop, which measured faster
// there (C3 FP64 97.4 ms against 100.5 with batches; C1 14.3 ms against
// 15.7 with the plain loop).
template <int NV, int S, class VT, class XT, class AT, bool BATCH = true>
__device__ __forceinline__ void iso_csr_row(const DevCsr<VT>& A, const XT* __restrict__ x,
                                            int row, int s, AT (&acc)[NV]) {
  constexpr int U = 4;
#pragma unroll
  for (int v = 0; v < NV; ++v) acc[v] = AT(0);
  const int k0 = A.rp[row], k1 = A.rp[row + 1];
  if constexpr (!BATCH) {
#pragma unroll 4
    for (int k = k0 + s; k < k1; k += S) {
      const AT a = cvt<AT>(__ldcs(A.val + k));
      AT xv[NV];
      iso_gather<NV, XT, AT>(x, __ldg(A.col + k), xv);
#pragma unroll
      for (int v = 0; v < NV; ++v) acc[v] += a * xv[v];
    }
  } else {
    for (int k = k0 + s; k < k1; k += U * S) {
      int j[U];
      VT a[U];
      AT xv[U][NV];
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int kk = min(k + u * S, k1 - 1);
        j[u] = __ldg(A.col + kk);
        a[u] = __ldcs(A.val + kk);
      }
#pragma unroll
      for (int u = 0; u < U; ++u) iso_gather<NV, XT, AT>(x, j[u], xv[u]);
#pragma unroll
      for (int u = 0; u < U; ++u)
        if (k + u * S < k1) {
          const AT au = cvt<AT>(a[u]);
#pragma unroll
          for (int v = 0; v < NV; ++v) acc[v] += au * xv[u][v];
        }
    }
  }
}

template <int NV, int MODE, class XT, class YT, class AT>
__device__ __forceinline__ void iso_store(int64_t node, const AT (&acc)[NV],
                                          const YT* __restrict__ f, YT* __restrict__ y) {
  const size_t o = (size_t)node * NV;
#pragma unroll
  for (int v = 0; v < NV; ++v) {
    if constexpr (MODE == SPMV_SET) y[o + v] = (YT)acc[v];
    else if constexpr (MODE == SPMV_RESID) y[o + v] = (YT)(cvt<AT>(f[o + v]) - acc[v]);
    else y[o + v] = (YT)(cvt<AT>(y[o + v]) + acc[v]);
  }
}

// MODE SET / RESID / ADD: y = (S (x) I) x, f - (S (x) I) x, y + (S (x) I) x
// with S in scalar CSR and S lanes per row.
template <int NV, int S, int MODE, class VT, class XT, class YT, class AT, bool BATCH>
__global__ void __launch_bounds__(256, 4) k_iso_csr_spmv(DevCsr<VT> A, const XT* __restrict__ x,
                                                      const YT* __restrict__ f,
                                                      YT* __restrict__ y) {
  GBS_GRID_DEP();
  RowMapS<1, S> m(blockIdx.x * (int64_t)blockDim.x + threadIdx.x);
  const bool ok = m.lane_ok && m.brow < A.n;
  AT acc[NV];
  if (ok) iso_csr_row<NV, S, VT, XT, AT, BATCH>(A, x, m.brow, m.s, acc);
  else
#pragma unroll
    for (int v = 0; v < NV; ++v) acc[v] = AT(0);
  if constexpr (S > 1) {
#pragma unroll
    for (int v = 0; v < NV; ++v) acc[v] = split_reduce<1, S, AT>(acc[v]);
  }
  if (!ok || m.s != 0) return;
  iso_store<NV, MODE, XT, YT, AT>(m.brow, acc, f, y);
}

// One CTA (G threads) per row of S: for small levels with long rows (the
// coarse levels and their transfer operators, hundreds of entries a row),
// where lane groups within a warp leave the GPU mostly idle and each lane
// walks a long dependent chain.  Every thread of the CTA must call it; on
// return every thread holds the row's NV sums.
template <int NV, int G, class VT, class XT, class AT>
__device__ __forceinline__ void iso_cta_row(const DevCsr<VT>& A, const XT* __restrict__ x, int row,
                                            AT (&acc)[NV]) {
  static_assert(G % 32 == 0 && G <= 1024, "G: whole warps");
  iso_csr_row<NV, G, VT, XT, AT>(A, x, row, threadIdx.x, acc);
#pragma unroll
  for (int v = 0; v < NV; ++v)
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc[v] += __shfl_xor_sync(0xffffffffu, acc[v], o);
  __shared__ AT red[G / 32][NV];
  const int w = threadIdx.x >> 5;
  if ((threadIdx.x & 31) == 0)
#pragma unroll
    for (int v = 0; v < NV; ++v) red[w][v] = acc[v];
  __syncthreads();
#pragma unroll
  for (int v = 0; v < NV; ++v) {
    AT t = AT(0);
#pragma unroll
    for (int q = 0; q < G / 32; ++q) t += red[q][v];
    acc[v] = t;
  }
}
template <int NV, int G, int MODE, class VT, class XT, class YT, class AT>
__global__ void __launch_bounds__(G) k_iso_csr_spmv_cta(DevCsr<VT> A, const XT* __restrict__ x,
                                                        const YT* __restrict__ f,
                                                        YT* __restrict__ y) {
  GBS_GRID_DEP();
  const int row = blockIdx.x;   // the grid has one CTA per row
  AT acc[NV];
  iso_cta_row<NV, G, VT, XT, AT>(A, x, row, acc);
  if (threadIdx.x == 0) iso_store<NV, MODE, XT, YT, AT>(row, acc, f, y);
}
template <int NV, int G, class VT, class XT, class AT, class OT = XT>
__global__ void __launch_bounds__(G) k_iso_csr_relax_cta(DevCsr<VT> A, const VT* __restrict__ M,
                                                         const XT* __restrict__ f,
                                                         const XT* __restrict__ x,
                                                         OT* __restrict__ xo) {
  GBS_GRID_DEP();
  const int row = blockIdx.x;
  AT acc[NV];
  iso_cta_row<NV, G, VT, XT, AT>(A, x, row, acc);
  if (threadIdx.x != 0) return;
  const AT mi = cvt<AT>(M[row]);
  const size_t o = (size_t)row * NV;
#pragma unroll
  for (int v = 0; v < NV; ++v)
    xo[o + v] = (OT)(XT)(cvt<AT>(x[o + v]) + mi * (cvt<AT>(f[o + v]) - acc[v]));
}

// xo = x + m .* (f - (S (x) I) x), m one smoother value per node.
template <int NV, int S, class VT, class XT, class AT, class OT, bool BATCH>
__global__ void __launch_bounds__(256, 4) k_iso_csr_relax(DevCsr<VT> A, const VT* __restrict__ M,
                                                       const XT* __restrict__ f,
                                                       const XT* __restrict__ x,
                                                       OT* __restrict__ xo) {
  GBS_GRID_DEP();
  RowMapS<1, S> m(blockIdx.x * (int64_t)blockDim.x + threadIdx.x);
  const bool ok = m.lane_ok && m.brow < A.n;
  AT acc[NV];
  if (ok) iso_csr_row<NV, S, VT, XT, AT, BATCH>(A, x, m.brow, m.s, acc);
  else
#pragma unroll
    for (int v = 0; v < NV; ++v) acc[v] = AT(0);
  if constexpr (S > 1) {
#pragma unroll
    for (int v = 0; v < NV; ++v) acc[v] = split_reduce<1, S, AT>(acc[v]);
  }
  if (!ok || m.s != 0) return;
  const AT mi = cvt<AT>(M[m.brow]);
  const size_t o = (size_t)m.brow * NV;
#pragma unroll
  for (int v = 0; v < NV; ++v)
    xo[o + v] = (OT)(XT)(cvt<AT>(x[o + v]) + mi * (cvt<AT>(f[o + v]) - acc[v]));
}

// Row of lane `lane` of slice q of S (32 consecutive nodes a slice) times
// the NV components of x; a uniform slice gathers at node + offset with no
// column loads.  Entries go in batches of U whose value (and column) loads
// and x gathers all issue before the FMAs; entries past the slice's width
// re-read its last one and lanes without the entry gather their own node,
// both dropped at the FMA (w is warp-uniform: no divergence).
//
// SCALE: the operand is diag(m) x with m gathered beside x (one value per
// node): the zero-guess smoothing step's x = m .* f formed on the fly, each
// product rounded as the stored x would be.
template <int NV, class VT, class XT, class AT, bool SCALE = false>
__device__ __forceinline__ void iso_sell_row(const DevSell<VT>& A, const XT* __restrict__ x, int q,
                                             int lane, int64_t node, AT (&acc)[NV],
                                             const VT* __restrict__ m = nullptr) {
  constexpr int U = 4;
#pragma unroll
  for (int v = 0; v < NV; ++v) acc[v] = AT(0);
  const int k0 = __ldg(A.off + q), w = __ldg(A.off + q + 1) - k0;
  const VT* v0 = A.val + (size_t)k0 * 32 + lane;
  const int ci = __ldg(A.cinfo + q);
  if (ci < 0) {
    const int2* u0 = A.uinfo + (-1 - ci);
    for (int k = 0; k < w; k += U) {
      int2 om[U];
      VT a[U];
      AT xv[U][NV];
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int kk = min(k + u, w - 1);
        om[u] = __ldg(u0 + kk);   // warp-uniform: one broadcast load
        a[u] = __ldcs(v0 + (size_t)kk * 32);
      }
      bool on[U];
#pragma unroll
      for (int u = 0; u < U; ++u) {
        on[u] = k + u < w && (((unsigned)om[u].y >> lane) & 1u);
        const int64_t jj = on[u] ? node + om[u].x : node;
        iso_gather<NV, XT, AT>(x, jj, xv[u]);
        if constexpr (SCALE) {
          const AT mj = cvt<AT>(__ldg(m + jj));
#pragma unroll
          for (int v = 0; v < NV; ++v) xv[u][v] = cvt<AT>((XT)(mj * xv[u][v]));
        }
      }
#pragma unroll
      for (int u = 0; u < U; ++u)
        if (on[u]) {
          const AT au = cvt<AT>(a[u]);
#pragma unroll
          for (int v = 0; v < NV; ++v) acc[v] += au * xv[u][v];
        }
    }
    return;
  }
  const int* c0 = A.col + (size_t)k0 * 32 + lane;
  for (int k = 0; k < w; k += U) {
    int j[U];
    VT a[U];
    AT xv[U][NV];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int kk = min(k + u, w - 1);
      j[u] = __ldcs(c0 + (size_t)kk * 32);
      a[u] = __ldcs(v0 + (size_t)kk * 32);
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      if (k + u >= w) j[u] = -1;
      const int64_t jj = j[u] >= 0 ? (int64_t)j[u] : node;
      iso_gather<NV, XT, AT>(x, jj, xv[u]);
      if constexpr (SCALE) {
        const AT mj = cvt<AT>(__ldg(m + jj));
#pragma unroll
        for (int v = 0; v < NV; ++v) xv[u][v] = cvt<AT>((XT)(mj * xv[u][v]));
      }
    }
#pragma unroll
    for (int u = 0; u < U; ++u)
      if (j[u] >= 0) {
        const AT au = cvt<AT>(a[u]);
#pragma unroll
        for (int v = 0; v < NV; ++v) acc[v] += au * xv[u][v];
      }
  }
}

// MODE SET / RESID / ADD on S in slices, one warp per slice.
template <int NV, int MODE, class VT, class XT, class YT, class AT>
__global__ void __launch_bounds__(256, 4) k_iso_sell_spmv(DevSell<VT> A, const XT* __restrict__ x,
                                                       const YT* __restrict__ f,
                                                       YT* __restrict__ y) {
  GBS_GRID_DEP();
  const int64_t q = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  if (q >= A.nslices) return;   // warp-uniform
  const int lane = threadIdx.x & 31;
  const int64_t node = sell_node(A, q, lane);
  AT acc[NV];
  iso_sell_row<NV, VT, XT, AT>(A, x, (int)q, lane, node < 0 ? 0 : node, acc);
  if (node < 0) return;
  iso_store<NV, MODE, XT, YT, AT>(node, acc, f, y);
}

// xo = x + m .* (f - (S (x) I) x) on S in slices; OT: the output's type
// (the last level-0 sweep of a mixed form writes the FP64 output).
template <int NV, class VT, class XT, class AT, class OT = XT>
__global__ void __launch_bounds__(256, 4) k_iso_sell_relax(DevSell<VT> A, const VT* __restrict__ M,
                                                        const XT* __restrict__ f,
                                                        const XT* __restrict__ x,
                                                        OT* __restrict__ xo) {
  GBS_GRID_DEP();
  const int64_t q = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  if (q >= A.nslices) return;
  const int lane = threadIdx.x & 31;
  const int64_t node = sell_node(A, q, lane);
  AT acc[NV];
  iso_sell_row<NV, VT, XT, AT>(A, x, (int)q, lane, node < 0 ? 0 : node, acc);
  if (node < 0) return;
  const AT mi = cvt<AT>(M[node]);
  const size_t o = (size_t)node * NV;
  AT fv[NV], xv[NV];
  load_run<NV, XT, AT, false>(f + o, fv);
  load_run<NV, XT, AT, false>(x + o, xv);
#pragma unroll
  for (int v = 0; v < NV; ++v) xo[o + v] = (OT)(XT)(xv[v] + mi * (fv[v] - acc[v]));
}

// Zero-guess pre-smoothing step fused with the residual (FP64 forms):
// x = m .* f and r = f - ((S diag(m)) (x) I) f, with S diag(m) stored in
// the level's slices.
template <int NV, class VT, class XT, class AT>
__global__ void __launch_bounds__(256, 4) k_iso_sell_presmooth(DevSell<VT> AM,
                                                            const VT* __restrict__ M,
                                                            const XT* __restrict__ f,
                                                            XT* __restrict__ x,
                                                            XT* __restrict__ r) {
  GBS_GRID_DEP();
  const int64_t q = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  if (q >= AM.nslices) return;
  const int lane = threadIdx.x & 31;
  const int64_t node = sell_node(AM, q, lane);
  AT acc[NV];
  iso_sell_row<NV, VT, XT, AT>(AM, f, (int)q, lane, node < 0 ? 0 : node, acc);
  if (node < 0) return;
  const AT mi = cvt<AT>(M[node]);
  const size_t o = (size_t)node * NV;
  AT fv[NV];
  load_run<NV, XT, AT, false>(f + o, fv);
#pragma unroll
  for (int v = 0; v < NV; ++v) {
    x[o + v] = (XT)(mi * fv[v]);
    r[o + v] = (XT)(fv[v] - acc[v]);
  }
}

// The same step for the mixed forms without a stored S diag(m) (which
// rounded to FP32/BF16 would not be S and m rounded): x = m .* f, and
// r = f - (S (x) I) x with each x_j = m_j f_j formed in the gather as the
// separate step would store it, so r equals the two-pass residual.
template <int NV, class VT, class XT, class AT>
__global__ void __launch_bounds__(256, 4) k_iso_sell_presmooth_otf(DevSell<VT> A,
                                                                const VT* __restrict__ M,
                                                                const XT* __restrict__ f,
                                                                XT* __restrict__ x,
                                                                XT* __restrict__ r) {
  GBS_GRID_DEP();
  const int64_t q = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  if (q >= A.nslices) return;
  const int lane = threadIdx.x & 31;
  const int64_t node = sell_node(A, q, lane);
  AT acc[NV];
  iso_sell_row<NV, VT, XT, AT, true>(A, f, (int)q, lane, node < 0 ? 0 : node, acc, M);
  if (node < 0) return;
  const AT mi = cvt<AT>(M[node]);
  const size_t o = (size_t)node * NV;
  AT fv[NV];
  load_run<NV, XT, AT, false>(f + o, fv);
#pragma unroll
  for (int v = 0; v < NV; ++v) {
    x[o + v] = (XT)(mi * fv[v]);
    r[o + v] = (XT)(fv[v] - acc[v]);
  }
}

// x = m .* f per node (the zero-guess smoothing step; diag(m) (x) I is
// symmetric, so the transposed cycle uses it as well).
// One thread a node (nn nodes).
template <int NV, class VT, class XT, class AT>
__global__ void k_iso_mapply(int64_t nn, const VT* __restrict__ M, const XT* __restrict__ f,
                             XT* __restrict__ x) {
  GBS_GRID_DEP();
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nn;
       i += (int64_t)gridDim.x * blockDim.x) {
    const AT mi = cvt<AT>(M[i]);
    AT fv[NV];
    load_run<NV, XT, AT, false>(f + i * NV, fv);
#pragma unroll
    for (int v = 0; v < NV; ++v) x[i * NV + v] = (XT)(mi * fv[v]);
  }
}

// The mixed forms' finest level with the FP64 -> FP32 boundary folded in:
// fin = (XT) r (round to nearest even) and x = m .* fin.
template <int NV, class VT, class XT, class AT>
__global__ void k_iso_cast_mapply(int64_t nn, const VT* __restrict__ M, const double* __restrict__ r,
                                  XT* __restrict__ fin, XT* __restrict__ x) {
  GBS_GRID_DEP();
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nn;
       i += (int64_t)gridDim.x * blockDim.x) {
    const AT mi = cvt<AT>(M[i]);
    double rv[NV];
    load_run<NV, double, double, true>(r + i * NV, rv);
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      const XT ri = (XT)rv[v];
      fin[i * NV + v] = ri;
      x[i * NV + v] = (XT)(mi * cvt<AT>(ri));
    }
  }
}

}  // namespace gbs
