// FP64 outer-Krylov kernels: SpMV of K with fused dot products,
// BiCGStab vector updates, GMRES orthogonalisation, sampled outer
// product.  Dots use a deterministic two-level reduction: a fixed grid of
// at most Red::cap blocks (all resident at once), warp-shuffle +
// shared-memory tree per block, then
// the last block to finish sums the per-block partials in block order
// and runs a scalar epilogue ("finalize") on thread 0.  No result depends
// on block scheduling.
//
// Scalars of the iteration live in device memory (sc[]), so kernels read
// alpha, beta, omega there and only the convergence check crosses to the
// host (Section 2.3's residual and inner-product primitives, kept in FP64
// as in the mixed-precision scheme of Section 4, Listing V4).
#pragma once

#include "kernels.cuh"
#include "sell.cuh"

namespace gbs {

constexpr int RED_THREADS = 256;
// The allocation-free entry point's fixed grid: 4 CTAs per SM of GB300's
// 152 (one-lane-per-row FP64 SpMV: FP64-pipe bound, half occupancy is
// faster).  A handle sizes its own grids from the device (Red::cap).
constexpr int OUTER_N_BLOCKS = 152 * 4;
constexpr int MAX_DOTS = 72;   // GMRES multi-dot: up to 64 basis vectors + spares

enum ScalarSlot {
  S_RHO = 0, S_RHO_OLD, S_ALPHA, S_OMEGA, S_RV, S_TS, S_TT, S_RR, S_BB, S_FIRST, S_BREAK,
  S_WW0, S_WW, S_REORTH, S_D0, S_D1,
  S_ERR,           // nonzero: a pipelined kernel's bounded wait timed out
  S_COUNT = 32
};

enum FinOp {
  FIN_STORE = 0,   // sc[S_D0] = d0, sc[S_D1] = d1
  FIN_ALPHA,       // rv = d0; alpha = rho / rv
  FIN_OMEGA,       // ts = d0, tt = d1, omega = ts / tt
  FIN_RHO,         // rho_old = rho; rho = d0; rr = d1; first = 0
  FIN_REPLACE,     // rho = d0; rr = d1
  FIN_INIT,        // rhat = r: rho = rr = d1; rho_old = alpha = omega = 1; first = 1
  FIN_BB,          // bb = d0
  FIN_RR,          // rr = d1
  FIN_OUT          // sc[0] = d0, sc[1] = d1 (sc points at a caller's 2-double output)
};

// Launch a grid-stride kernel of RED_THREADS threads with resident_grid blocks.
template <class... KA, class... A>
inline void launch_resident(void (*fn)(KA...), int cap, cudaStream_t s, A&&... a) {
  ::gbs::launch_k(fn, resident_grid((const void*)fn, cap, RED_THREADS, 0), RED_THREADS, 0, s, 
      std::forward<A>(a)...);
}

struct Red {
  int cap = 1;        // CTAs of a reduction grid: 8 per SM of this device (one wave)
  double* partials;   // cap * MAX_DOTS
  unsigned* counter;  // one per reduction slot; reset by the last block
  double* sc;
};

__device__ __forceinline__ void finalize(int op, const double* d, double* sc) {
  switch (op) {
    case FIN_STORE: sc[S_D0] = d[0]; sc[S_D1] = d[1]; break;
    case FIN_ALPHA:
      sc[S_RV] = d[0];
      if (d[0] == 0.0 || !isfinite(d[0])) { sc[S_BREAK] = 1.0; sc[S_ALPHA] = 0.0; }
      else sc[S_ALPHA] = sc[S_RHO] / d[0];
      break;
    case FIN_OMEGA:
      sc[S_TS] = d[0];
      sc[S_TT] = d[1];
      sc[S_OMEGA] = d[1] > 0.0 ? d[0] / d[1] : 0.0;
      break;
    case FIN_RHO:
      sc[S_RHO_OLD] = sc[S_RHO];
      sc[S_RHO] = d[0];
      sc[S_RR] = d[1];
      sc[S_FIRST] = 0.0;
      break;
    case FIN_REPLACE: sc[S_RHO] = d[0]; sc[S_RR] = d[1]; break;
    case FIN_INIT:
      sc[S_RHO] = d[1];
      sc[S_RR] = d[1];
      sc[S_RHO_OLD] = 1.0;
      sc[S_ALPHA] = 1.0;
      sc[S_OMEGA] = 1.0;
      sc[S_FIRST] = 1.0;
      sc[S_BREAK] = 0.0;
      break;
    case FIN_BB: sc[S_BB] = d[0]; break;
    case FIN_RR: sc[S_RR] = d[1]; break;
    case FIN_OUT: sc[0] = d[0]; sc[1] = d[1]; break;
  }
}

// Block-level deterministic reduction of ND values held per thread; the
// result is valid in thread 0.
template <int ND>
__device__ __forceinline__ void block_sum(double (&v)[ND], double (*sh)[ND]) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
  for (int q = 0; q < ND; ++q) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v[q] += __shfl_xor_sync(0xffffffffu, v[q], o);
  }
  __syncthreads();
  if (lane == 0) {
#pragma unroll
    for (int q = 0; q < ND; ++q) sh[w][q] = v[q];
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    const int nw = blockDim.x >> 5;
#pragma unroll
    for (int q = 0; q < ND; ++q) {
      double s = 0.0;
      for (int i = 0; i < nw; ++i) s += sh[i][q];
      v[q] = s;
    }
  }
}

// Store the block partials, and in the last block reduce them and run
// the epilogue.  Returns true in the thread that ran the epilogue.
template <int ND>
__device__ __forceinline__ void grid_reduce(double (&v)[ND], const Red& R, int slot, int op) {
  __shared__ double sh[RED_THREADS / 32][ND];
  __shared__ bool last;
  block_sum<ND>(v, sh);
  if (threadIdx.x == 0) {
#pragma unroll
    for (int q = 0; q < ND; ++q) R.partials[(size_t)blockIdx.x * ND + q] = v[q];
    __threadfence();
    unsigned t = atomicAdd(R.counter + slot, 1u);
    last = (t == gridDim.x - 1);
  }
  __syncthreads();
  if (!last) return;
  __threadfence();
  double s[ND];
#pragma unroll
  for (int q = 0; q < ND; ++q) s[q] = 0.0;
  for (int b = threadIdx.x; b < (int)gridDim.x; b += blockDim.x) {
#pragma unroll
    for (int q = 0; q < ND; ++q) s[q] += __ldcg(R.partials + (size_t)b * ND + q);
  }
  block_sum<ND>(s, sh);
  if (threadIdx.x == 0) {
    double d[2] = {s[0], ND > 1 ? s[ND > 1 ? 1 : 0] : 0.0};
    finalize(op, d, R.sc);
    R.counter[slot] = 0u;
  }
}

// y = K x (RESID: y = f - K x); d0 = sum y*w0 (w0 null: 0), d1 = sum y*y
// when self_dot (w0 must not alias y).  G lanes per block row (chunk
// streaming, see group_row_fwd), grid-stride over block rows with a
// warp-uniform exit so that every lane takes part in the shuffles.
template <int B, int G, bool TR, int MODE>
__global__ void __launch_bounds__(RED_THREADS, 4)
    k_outer(DevBsr<double> K, const double* __restrict__ x, const double* __restrict__ f,
            double* __restrict__ y, const double* __restrict__ w0, int self_dot, Red R, int slot,
            int op, int reduce) {
  GBS_GRID_DEP();
  static_assert(G <= 32, "outer SpMV groups stay inside a warp");
  double d[2] = {0.0, 0.0};
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int64_t gid = t / G;
  const int g = (int)(t % G);
  const int64_t ngroups = ((int64_t)gridDim.x * blockDim.x) / G;
  for (int64_t brow = gid;; brow += ngroups) {
    const bool ok = brow < K.nbr;
    if (!__any_sync(0xffffffffu, ok)) break;
    double acc[B];
    group_row<B, G, TR, double, double, double>(K, x, (int)brow, g, ok, acc);
    if (ok && g < B) {
      const size_t o = (size_t)brow * B + g;
      const double a = pick<B, double>(acc, g);
      const double val = MODE == SPMV_RESID ? f[o] - a : a;
      y[o] = val;
      if (w0) d[0] += val * w0[o];
      if (self_dot) d[1] += val * val;
    }
  }
  if (reduce) grid_reduce<2>(d, R, slot, op);
}

// Same operation with one lane per scalar row (B lanes per block row, no
// cross-lane sums): the fewest FP64 operations, used whenever K has
// enough rows to fill the GPU.
template <int B, bool TR, int MODE>
__global__ void __launch_bounds__(RED_THREADS, 4)
    k_outer_n(DevBsr<double> K, const double* __restrict__ x, const double* __restrict__ f,
              double* __restrict__ y, const double* __restrict__ w0, int self_dot, Red R,
              int slot, int op, int reduce) {
  GBS_GRID_DEP();
  constexpr int RPW = 32 / B;
  double d[2] = {0.0, 0.0};
  const int64_t nwarps = ((int64_t)K.nbr + RPW - 1) / RPW;
  const int lane = threadIdx.x & 31;
  const int sub = lane / B, r = lane - sub * B;
  const bool lane_ok = sub < RPW;
  for (int64_t w = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; w < nwarps;
       w += ((int64_t)gridDim.x * blockDim.x) >> 5) {
    const int brow = (int)(w * RPW + sub);
    if (!lane_ok || brow >= K.nbr) continue;
    const double acc = row_dot<B, TR, double, double, double>(K, x, brow, r);
    const size_t o = (size_t)brow * B + r;
    const double val = MODE == SPMV_RESID ? f[o] - acc : acc;
    y[o] = val;
    if (w0) d[0] += val * w0[o];
    if (self_dot) d[1] += val * val;
  }
  if (reduce) grid_reduce<2>(d, R, slot, op);
}

// Outer SpMV of K held as scalar CSR (S lanes per scalar row), same
// outputs and dots as k_outer_n; grid-stride with a warp-uniform bound.
template <int S, int MODE>
__global__ void __launch_bounds__(RED_THREADS, 4)
    k_outer_csr(DevCsr<double> K, const double* __restrict__ x, const double* __restrict__ f,
                double* __restrict__ y, const double* __restrict__ w0, int self_dot, Red R,
                int slot, int op, int reduce) {
  GBS_GRID_DEP();
  constexpr int RPW = 32 / S;
  double d[2] = {0.0, 0.0};
  const int64_t nwarps = ((int64_t)K.n + RPW - 1) / RPW;
  const int lane = threadIdx.x & 31;
  const int sub = lane / S, s = lane - sub * S;
  for (int64_t w = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; w < nwarps;
       w += ((int64_t)gridDim.x * blockDim.x) >> 5) {
    const int row = (int)(w * RPW + sub);
    const bool ok = row < K.n;
    double acc = ok ? csr_row_dot<S, double, double, double>(K, x, row, s) : 0.0;
    if constexpr (S > 1) acc = split_reduce<1, S, double>(acc);
    if (ok && s == 0) {
      const double val = MODE == SPMV_RESID ? f[row] - acc : acc;
      y[row] = val;
      if (w0) d[0] += val * w0[row];
      if (self_dot) d[1] += val * val;
    }
  }
  if (reduce) grid_reduce<2>(d, R, slot, op);
}

// y = K x (RESID: y = f - K x) with K in 32-node component slices, one
// warp per 32-node group (grid-stride), direct loads (sell.cuh); dots as
// k_outer.  The warp walks the group's B slices and each lane then stores
// its node's B rows contiguously.  On a stencil operator every slice is
// uniform: no column loads, and the gather address comes from the row
// index.
template <int MODE, int B>
__global__ void __launch_bounds__(RED_THREADS, 4)
    k_outer_sell(DevSell<double> K, const double* __restrict__ x, const double* __restrict__ f,
                 double* __restrict__ y, const double* __restrict__ w0, int self_dot, Red R,
                 int slot, int op, int reduce) {
  GBS_GRID_DEP();
  double d[2] = {0.0, 0.0};
  const int lane = threadIdx.x & 31;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const int64_t ng = K.nslices / B;
  for (int64_t g = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; g < ng; g += nw) {
    const int64_t node = sell_node(K, g, lane);
    const int64_t nd = node < 0 ? 0 : node;   // no entries in an empty lane
    double res[B];
#pragma unroll
    for (int c = 0; c < B; ++c)
      res[c] = sell_row_dot_direct<double, double, double>(K, x, (int)(g * B + c), lane, nd * B + c);
    if (node >= 0) {
      double fv[B];
      if (MODE == SPMV_RESID) load_run<B, double, double, false>(f + node * B, fv);
#pragma unroll
      for (int c = 0; c < B; ++c) {
        const double val = MODE == SPMV_RESID ? fv[c] - res[c] : res[c];
        y[node * B + c] = val;
        if (w0) d[0] += val * w0[node * B + c];
        if (self_dot) d[1] += val * val;
      }
    }
  }
  if (reduce) grid_reduce<2>(d, R, slot, op);
}

// Sliced values of K from its block values (map -1: padding).
static __global__ void k_gather_sell(int64_t n, const int* __restrict__ map,
                                     const double* __restrict__ bval, double* __restrict__ sval) {
  GBS_GRID_DEP();
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int m = map[i];
    sval[i] = m >= 0 ? bval[m] : 0.0;
  }
}

// CSR values of K from its block values (after gbs_update_values).
static __global__ void k_gather_vals(int64_t nnz, const int* __restrict__ map,
                                     const double* __restrict__ bval, double* __restrict__ cval) {
  GBS_GRID_DEP();
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nnz;
       i += (int64_t)gridDim.x * blockDim.x)
    cval[i] = bval[map[i]];
}

// flag = 1 if any block value outside the CSR pattern (mask bit set) is nonzero.
static __global__ void k_check_outside(int64_t nvals, const unsigned* __restrict__ zero_mask,
                                       const double* __restrict__ bval, int* __restrict__ flag) {
  GBS_GRID_DEP();
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nvals;
       i += (int64_t)gridDim.x * blockDim.x)
    if (((zero_mask[i >> 5] >> (i & 31)) & 1u) && bval[i] != 0.0) *flag = 1;
}

// p = r + beta (p - omega v), beta = (rho / rho_old) (alpha / omega); p = r on the first step.
static __global__ void k_bicg_p(int64_t n, const double* __restrict__ r, const double* __restrict__ v,
                         double* __restrict__ p, const double* __restrict__ sc) {
  GBS_GRID_DEP();
  // the two FP64 divisions once per CTA, not once per thread
  __shared__ double sbeta;
  const bool first = sc[S_FIRST] != 0.0;
  const double omega = sc[S_OMEGA];
  if (threadIdx.x == 0) sbeta = first ? 0.0 : (sc[S_RHO] / sc[S_RHO_OLD]) * (sc[S_ALPHA] / omega);
  __syncthreads();
  const double beta = sbeta;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    p[i] = first ? r[i] : r[i] + beta * (p[i] - omega * v[i]);
}

// s = r - alpha v
static __global__ void k_bicg_s(int64_t n, const double* __restrict__ r, const double* __restrict__ v,
                         double* __restrict__ s, const double* __restrict__ sc) {
  GBS_GRID_DEP();
  const double alpha = sc[S_ALPHA];
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    s[i] = r[i] - alpha * v[i];
}

// x += alpha phat + omega shat; r = s - omega t; d0 = rhat.r, d1 = r.r
static __global__ void __launch_bounds__(RED_THREADS, 4)
    k_bicg_xr(int64_t n, double* __restrict__ x, const double* __restrict__ ph,
              const double* __restrict__ sh, const double* __restrict__ s,
              const double* __restrict__ t, double* __restrict__ r,
              const double* __restrict__ rhat, Red R, int slot) {
  GBS_GRID_DEP();
  const double alpha = R.sc[S_ALPHA], omega = R.sc[S_OMEGA];
  double d[2] = {0.0, 0.0};
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    x[i] += alpha * ph[i] + omega * sh[i];
    const double ri = s[i] - omega * t[i];
    r[i] = ri;
    d[0] += rhat[i] * ri;
    d[1] += ri * ri;
  }
  grid_reduce<2>(d, R, slot, FIN_RHO);
}

// d0 = a.b, d1 = c.c (c may be null)
static __global__ void __launch_bounds__(RED_THREADS, 4)
    k_dot2(int64_t n, const double* __restrict__ a, const double* __restrict__ b,
           const double* __restrict__ c, Red R, int slot, int op) {
  GBS_GRID_DEP();
  double d[2] = {0.0, 0.0};
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    if (a) d[0] += a[i] * b[i];
    if (c) d[1] += c[i] * c[i];
  }
  grid_reduce<2>(d, R, slot, op);
}

static __global__ void k_set_restart(double* sc) {
  GBS_GRID_DEP();
  sc[S_RHO] = sc[S_RR];
  sc[S_RHO_OLD] = 1.0;
  sc[S_ALPHA] = 1.0;
  sc[S_OMEGA] = 1.0;
  sc[S_FIRST] = 1.0;
}

// ------------------------------------------------------------------ IDR(s)
struct Coefs {
  double c[8];
};

// out = alpha * a + sum_{i<m} c_i V_i  (V_i = V + i*n).  out may alias a
// or V_0: every element reads its inputs before writing.
static __global__ void k_idr_comb(int64_t n, double* out, double alpha, const double* a,
                                  const double* V, int m, Coefs c) {
  GBS_GRID_DEP();
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n;
       e += (int64_t)gridDim.x * blockDim.x) {
    double acc = a ? alpha * a[e] : 0.0;
#pragma unroll
    for (int i = 0; i < 8; ++i)
      if (i < m) acc += c.c[i] * V[(size_t)i * n + e];
    out[e] = acc;
  }
}

// r -= beta g; x += beta u; sc[S_RR] = r . r
static __global__ void __launch_bounds__(RED_THREADS, 4)
    k_idr_update(int64_t n, double* __restrict__ r, double* __restrict__ x,
                 const double* __restrict__ g, const double* __restrict__ u, double beta, Red R,
                 int slot) {
  GBS_GRID_DEP();
  double d[2] = {0.0, 0.0};
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const double ri = r[i] - beta * g[i];
    r[i] = ri;
    x[i] += beta * u[i];
    d[1] += ri * ri;
  }
  grid_reduce<2>(d, R, slot, FIN_RR);
}

// ------------------------------------------------------------------ GMRES
// Partial dots of one pass over the CHN vectors V0 + q n (q < CHN) against
// w, plus w . w when WW: no branch in the element loop, so each element's
// loads issue together (a per-vector bounds test there serialised the
// loads and ran the kernel at a third of the bandwidth).  Block sums go to
// out[0..CHN) and, with WW, to ww_out.
template <int CHN, bool WW>
__device__ __forceinline__ void multidot_pass(int64_t n, const double* __restrict__ V0,
                                              const double* __restrict__ w, double* out,
                                              double* ww_out, double (*sh)[8]) {
  double v[CHN + 1];
#pragma unroll
  for (int q = 0; q <= CHN; ++q) v[q] = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const double wi = w[i];
    double a[CHN > 0 ? CHN : 1];
#pragma unroll
    for (int q = 0; q < CHN; ++q) a[q] = V0[(size_t)q * n + i];
#pragma unroll
    for (int q = 0; q < CHN; ++q) v[q] += a[q] * wi;
    if constexpr (WW) v[CHN] += wi * wi;
  }
  double t[8];
#pragma unroll
  for (int q = 0; q < 8; ++q) t[q] = q <= CHN ? v[q <= CHN ? q : 0] : 0.0;
  block_sum<8>(t, sh);
  if (threadIdx.x == 0) {
#pragma unroll
    for (int q = 0; q < CHN; ++q) out[q] = t[q];
    if constexpr (WW) *ww_out = t[CHN];
  }
  __syncthreads();
}

// h[i] = V_i . w for i < J, and sc[S_WW0] = w . w: passes of 7 (the first
// also forms w . w), 8, 4, 2, 1 vectors, so no FP64 work goes to padding.
static __global__ void __launch_bounds__(RED_THREADS, 4)
    k_multidot(int64_t n, const double* __restrict__ V, int J, const double* __restrict__ w,
               double* __restrict__ h, Red R, int slot, const double* __restrict__ gate) {
  GBS_GRID_DEP();
  if (gate && *gate == 0.0) return;
  __shared__ double sh[RED_THREADS / 32][8];
  __shared__ bool last;
  const int nv = J + 1;   // partial slot J holds w . w
  double* part = R.partials + (size_t)blockIdx.x * MAX_DOTS;
  // first pass: up to 7 vectors and w . w
  int v0 = J < 7 ? J : 7;
  switch (v0) {
    case 0: multidot_pass<0, true>(n, V, w, part, part + J, sh); break;
    case 1: multidot_pass<1, true>(n, V, w, part, part + J, sh); break;
    case 2: multidot_pass<2, true>(n, V, w, part, part + J, sh); break;
    case 3: multidot_pass<3, true>(n, V, w, part, part + J, sh); break;
    case 4: multidot_pass<4, true>(n, V, w, part, part + J, sh); break;
    case 5: multidot_pass<5, true>(n, V, w, part, part + J, sh); break;
    case 6: multidot_pass<6, true>(n, V, w, part, part + J, sh); break;
    default: multidot_pass<7, true>(n, V, w, part, part + J, sh); break;
  }
  while (v0 < J) {
    const int left = J - v0;
    const double* V0 = V + (size_t)v0 * n;
    if (left >= 8) {
      multidot_pass<8, false>(n, V0, w, part + v0, nullptr, sh);
      v0 += 8;
    } else if (left >= 4) {
      multidot_pass<4, false>(n, V0, w, part + v0, nullptr, sh);
      v0 += 4;
    } else if (left >= 2) {
      multidot_pass<2, false>(n, V0, w, part + v0, nullptr, sh);
      v0 += 2;
    } else {
      multidot_pass<1, false>(n, V0, w, part + v0, nullptr, sh);
      v0 += 1;
    }
  }
  if (threadIdx.x == 0) {
    __threadfence();
    unsigned t = atomicAdd(R.counter + slot, 1u);
    last = (t == gridDim.x - 1);
  }
  __syncthreads();
  if (!last) return;
  __threadfence();
  for (int c0 = 0; c0 < nv; c0 += 8) {
    double s[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) s[q] = 0.0;
    for (int b = threadIdx.x; b < (int)gridDim.x; b += blockDim.x) {
#pragma unroll
      for (int q = 0; q < 8; ++q)
        if (c0 + q < nv) s[q] += __ldcg(R.partials + (size_t)b * MAX_DOTS + c0 + q);
    }
    block_sum<8>(s, sh);
    if (threadIdx.x == 0) {
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        const int vi = c0 + q;
        if (vi < J) h[vi] = s[q];
        else if (vi == J) R.sc[S_WW0] = s[q];
      }
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) R.counter[slot] = 0u;
}

// w -= sum_i h[i] V_i; sc[S_WW] = w.w; sc[S_REORTH] = (ww < 0.5 ww0).
// accumulate (non-null): hacc[i] += h[i] as well (second pass).
static __global__ void __launch_bounds__(RED_THREADS, 4)
    k_orth(int64_t n, const double* __restrict__ V, int J, double* __restrict__ w,
           const double* __restrict__ h, double* __restrict__ hacc, Red R, int slot,
           const double* __restrict__ gate) {
  GBS_GRID_DEP();
  if (gate && *gate == 0.0) return;
  __shared__ double hs[MAX_DOTS];
  for (int i = threadIdx.x; i < J; i += blockDim.x) hs[i] = h[i];
  __syncthreads();
  double d[1] = {0.0};
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    double wi = w[i];
    for (int q = 0; q < J; ++q) wi -= hs[q] * V[(size_t)q * n + i];
    w[i] = wi;
    d[0] += wi * wi;
  }
  __shared__ double sh[RED_THREADS / 32][1];
  __shared__ bool last;
  block_sum<1>(d, sh);
  if (threadIdx.x == 0) {
    R.partials[blockIdx.x] = d[0];
    __threadfence();
    unsigned t = atomicAdd(R.counter + slot, 1u);
    last = (t == gridDim.x - 1);
  }
  __syncthreads();
  if (!last) return;
  __threadfence();
  double s[1] = {0.0};
  for (int b = threadIdx.x; b < (int)gridDim.x; b += blockDim.x) s[0] += __ldcg(R.partials + b);
  block_sum<1>(s, sh);
  if (threadIdx.x == 0) {
    R.sc[S_WW] = s[0];
    if (hacc) {
      for (int q = 0; q < J; ++q) hacc[q] += hs[q];
      R.sc[S_REORTH] = 0.0;
    } else {
      R.sc[S_REORTH] = (s[0] < 0.5 * R.sc[S_WW0]) ? 1.0 : 0.0;
    }
    R.counter[slot] = 0u;
  }
}

// w /= sqrt(sc[S_WW]) (if nonzero); hnext = sqrt(sc[S_WW])
static __global__ void k_normalize(int64_t n, double* __restrict__ w, const double* __restrict__ sc,
                            double* __restrict__ hnext) {
  GBS_GRID_DEP();
  const double nrm = sqrt(sc[S_WW]);
  if (blockIdx.x == 0 && threadIdx.x == 0) *hnext = nrm;
  if (nrm == 0.0) return;
  const double inv = 1.0 / nrm;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    w[i] *= inv;
}

// v = r / sqrt(sc[S_RR])
static __global__ void k_scale_rr(int64_t n, const double* __restrict__ r, double* __restrict__ v,
                           const double* __restrict__ sc) {
  GBS_GRID_DEP();
  const double inv = 1.0 / sqrt(sc[S_RR]);
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    v[i] = r[i] * inv;
}

// u = sum_{i<J} y[i] V_i
static __global__ void k_combine(int64_t n, const double* __restrict__ V, int J,
                          const double* __restrict__ y, double* __restrict__ u) {
  GBS_GRID_DEP();
  __shared__ double ys[MAX_DOTS];
  for (int i = threadIdx.x; i < J; i += blockDim.x) ys[i] = y[i];
  __syncthreads();
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    double acc = 0.0;
    for (int q = 0; q < J; ++q) acc += ys[q] * V[(size_t)q * n + i];
    u[i] = acc;
  }
}

static __global__ void k_axpy(int64_t n, double a, const double* __restrict__ x, double* __restrict__ y) {
  GBS_GRID_DEP();
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    y[i] += a * x[i];
}

// grad[k, a, c] = alpha * lam[B i + a] * x[B j + c] on the stored pattern.
template <int B>
__global__ void __launch_bounds__(256)
    k_sampled_outer(DevBsr<double> K, const double* __restrict__ lam,
                    const double* __restrict__ x, double alpha, double* __restrict__ grad) {
  GBS_GRID_DEP();
  RowMap<B> m(blockIdx.x * (int64_t)blockDim.x + threadIdx.x);
  if (!m.lane_ok || m.brow >= K.nbr) return;
  const double la = alpha * lam[(size_t)m.brow * B + m.r];
  for (int k = K.rp[m.brow]; k < K.rp[m.brow + 1]; ++k) {
    const int j = K.col[k];
    double xv[B];
    load_run<B, double, double, false>(x + (size_t)j * B, xv);
    double* g = grad + (size_t)k * (B * B) + m.r * B;
#pragma unroll
    for (int c = 0; c < B; ++c) __stcs(g + c, la * xv[c]);
  }
}

}  // namespace gbs
