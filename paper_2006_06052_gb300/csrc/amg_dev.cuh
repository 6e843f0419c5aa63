// Device AMG hierarchy, V-cycle and Schur pressure correction, templated
// on the storage form (FP64 / FP32 / BF16 values).  Included once per
// form by amg_fp64.cu, amg_fp32.cu, amg_bf16.cu.
//
// V-cycle (Section 2.1: AMG with SPAI0 relaxation on every level): one
// zero-guess pre-sweep x = M f, residual r = f - A x, restriction
// f_c = R r, recursive coarse correction, prolongation x += P e_c, one
// post-sweep x += M (f - A x); dense inverse on the coarsest level.  The
// transposed cycle uses A^T (transpose map), M^T, the same P and R
// (R = P^T) and the transposed coarse inverse, with the sweep counts
// swapped, which makes it the exact adjoint of the forward cycle.
//
// Schur pressure correction (Section 4, Eq. SchurPC, one V-cycle per
// inner solve): u* = V_A(r_u); p = V_S(r_p - D u*); u = V_A(r_u - G p).
// The transposed application runs the same steps on K^T = [A^T D^T; G^T
// C^T] with transposed V-cycles.
#pragma once

#include <cuda_bf16.h>

#include <algorithm>
#include <cstdlib>

#include "device.hpp"
#include "iso.cuh"
#include "kernels.cuh"
#include "sell.cuh"

namespace gbs {

template <int P>
struct FormT;
template <>
struct FormT<0> {
  using VT = double;  // stored values
  using ST = double;  // V-cycle vectors and accumulation
};
template <>
struct FormT<1> {
  using VT = float;
  using ST = float;
};
template <>
struct FormT<2> {
  using VT = __nv_bfloat16;
  using ST = float;
};

template <class VT>
inline VT cast_host(double v);
template <>
inline double cast_host<double>(double v) { return v; }
template <>
inline float cast_host<float>(double v) { return (float)v; }
template <>
inline __nv_bfloat16 cast_host<__nv_bfloat16>(double v) { return __double2bfloat16(v); }

template <class VT>
std::vector<VT> cast_vec(const std::vector<double>& v) {
  std::vector<VT> o(v.size());
  for (size_t i = 0; i < v.size(); ++i) o[i] = cast_host<VT>(v[i]);
  return o;
}

// The chunk-streaming products (group_row_fwd) read whole 16-byte-aligned
// chunks of a level's value array and, for scalar rows, of its column
// array, and gather x at every column of a chunk: the last chunk reaches up
// to 16 bytes past the last entry.  Uploads therefore pad both arrays to a
// multiple of CHUNK_PAD entries (at least one chunk) with value 0 and
// column 0, so every chunk lies inside its allocation and every gathered
// column is a valid index.
constexpr size_t CHUNK_PAD = 8;   // entries in 16 bytes of 2-byte values
inline size_t chunk_padded(size_t n) {
  return std::max<size_t>(CHUNK_PAD, (n + CHUNK_PAD - 1) / CHUNK_PAD * CHUNK_PAD);
}
inline std::vector<int32_t> padded_cols(const std::vector<int32_t>& c) {
  std::vector<int32_t> o(chunk_padded(c.size()), 0);
  std::copy(c.begin(), c.end(), o.begin());
  return o;
}
template <class VT>
std::vector<VT> padded_vals(const std::vector<double>& v) {
  std::vector<VT> o = cast_vec<VT>(v);
  o.resize(chunk_padded(v.size()), cast_host<VT>(0.0));
  return o;
}

template <class VT, class AT>
DevBsr<VT> upload_bsr(Arena& ar, const HBsr& H, bool with_tmap, cudaStream_t s,
                      std::vector<std::vector<VT>>& keep) {
  DevBsr<VT> d;
  d.nbr = H.nbr;
  d.nbc = H.nbc;
  d.rp = ar.upload(H.ptr.data(), H.ptr.size(), s);
  const std::vector<int32_t> cp = padded_cols(H.col);
  d.col = ar.upload(cp.data(), cp.size(), s);
  keep.push_back(padded_vals<VT>(H.val));
  d.val = ar.upload(keep.back().data(), keep.back().size(), s);
  if (H.nnzb() * H.br * H.bc >= (int64_t)INT32_MAX)
    throw SetupError{"a level holds 2^31 or more block values (int32 element indices)"};
  switch (H.br) {
    case 1: d.S = choose_split<1>(H.nbr, H.nnzb()); break;
    case 2: d.S = choose_split<2>(H.nbr, H.nnzb()); break;
    case 3: d.S = choose_split<3>(H.nbr, H.nnzb()); break;
    default: d.S = choose_split<4>(H.nbr, H.nnzb()); break;
  }
  if (const char* e = std::getenv("GBS_SPMV_SPLIT")) {  // tuning override: 1, 2, 4, 8
    int sp = std::atoi(e);
    if (sp == 1 || sp == 2 || sp == 4 || sp == 8) d.S = sp;
  }
  while (d.S > 1 && H.br * d.S > 32) d.S >>= 1;
  switch (H.br) {
    case 1: d.G = choose_group<1, VT, AT>(H.nbr, H.nnzb()); break;
    case 2: d.G = choose_group<2, VT, AT>(H.nbr, H.nnzb()); break;
    case 3: d.G = choose_group<3, VT, AT>(H.nbr, H.nnzb()); break;
    default: d.G = choose_group<4, VT, AT>(H.nbr, H.nnzb()); break;
  }
  if (const char* e = std::getenv("GBS_SPMV_GROUP")) {  // tuning override: 0, 8, 16, 32, 256
    int g = std::atoi(e);
    if (g == 0 || g == 8 || g == 16 || g == 32 || g == 256) d.G = g;
  }
  if (with_tmap) {
    std::vector<int32_t> tm;
    if (!transpose_map(H, tm))
      throw SetupError{"block pattern is not structurally symmetric (needed for the adjoint)"};
    d.tmap = ar.upload(tm.data(), tm.size(), s);
  }
  return d;
}

template <class VT>
DevCsr<VT> upload_csr(Arena& ar, const HCsr& C, cudaStream_t s, std::vector<std::vector<VT>>& keep) {
  DevCsr<VT> d;
  d.n = C.n;
  d.rp = ar.upload(C.ptr.data(), C.ptr.size(), s);
  const std::vector<int32_t> cp = padded_cols(C.col);   // see CHUNK_PAD
  d.col = ar.upload(cp.data(), cp.size(), s);
  keep.push_back(padded_vals<VT>(C.val));
  d.val = ar.upload(keep.back().data(), keep.back().size(), s);
  d.S = csr_split(C.n, (int64_t)C.col.size());
  if (const char* e = std::getenv("GBS_SPMV_SPLIT")) {
    int sp = std::atoi(e);
    if (sp == 1 || sp == 2 || sp == 4 || sp == 8) d.S = sp;
  }
  // FP32/BF16 values (not FP64-pipe bound): long rows stream as aligned
  // 16-byte chunks over G lanes (group_row_fwd with B = 1), so a warp's
  // loads cover contiguous runs instead of S lanes striding one entry at a
  // time.  GBS_CSR_CHUNK=0 keeps the strided lanes (measurement, tests).
  if (sizeof(VT) < 8 && C.n > 0) {
    const double chunks = (double)C.col.size() / C.n * sizeof(VT) / 16.0;
    d.G = chunks >= 48 ? 32 : chunks >= 16 ? 16 : chunks >= 4 ? 8 : 0;
    if (const char* e = std::getenv("GBS_CSR_CHUNK"))
      if (e[0] == '0') d.G = 0;
  }
  return d;
}

template <class VT>
DevBSell<VT> upload_bsell(Arena& ar, const HBSell& S, cudaStream_t s,
                          std::vector<std::vector<VT>>& keep) {
  DevBSell<VT> d;
  d.nbr = S.nbr;
  d.nslices = S.nslices;
  d.perm = ar.upload(S.perm.data(), S.perm.size(), s);
  d.off = ar.upload(S.off.data(), S.off.size(), s);
  d.col = ar.upload(S.col.data(), S.col.size(), s);
  keep.push_back(cast_vec<VT>(S.val));
  d.val = ar.upload(keep.back().data(), keep.back().size(), s);
  return d;
}

// Block-row slices (HBSell) for a block level of an FP64 form: the FP64
// pipe bounds those kernels, and the sorted slices give every lane a whole
// row of nearly the common length, with no cross-lane sums.  Taken when
// the level has at least 32k scalar rows (a warp per slice then still
// fills the GPU), runs one lane per scalar row (G = 0), and padding adds
// at most 15%.  GBS_BSELL=0 / 1 switches the choice off / forces it on
// every square block level (tests).
constexpr int BSELL_WINDOW = 32;   // slices per sorting window
template <class AT>
inline bool use_bsell(const HBsr& H, int G) {
  if (H.br != H.bc) return false;
  if (const char* e = std::getenv("GBS_BSELL")) {
    if (e[0] == '0') return false;
    if (e[0] == '1') return true;
  }
  if (sizeof(AT) != 8 || G != 0 || (int64_t)H.nbr * H.br < 32768) return false;
  return bsell_padding(H, BSELL_WINDOW) <= 0.15;
}

// Zero-guess pre-smoothing fused with the residual (x = M f, r = f - (A M) f)
// on FP64 levels that run in slices, with one pre-sweep of SPAI0 or Jacobi:
// one pass instead of two, and no wait for x between them.  The mixed forms
// keep the two passes (A M rounded to FP32/BF16 is not A and M rounded).
// GBS_FUSE=0 switches it off (measurement and tests).
template <class AT>
inline bool use_fused(const HLevel& h, const PrecondOptions& o) {
  if (sizeof(AT) != 8 || o.npre != 1 || !h.ilu.d.empty() || h.M.empty()) return false;
  if (const char* e = std::getenv("GBS_FUSE")) return e[0] != '0';
  return true;
}
inline bool fuse_enabled() {
  const char* e = std::getenv("GBS_FUSE");
  return !(e && e[0] == '0');
}

// Per-level format choice: a level whose stored blocks are at most half
// nonzero is kept as scalar CSR of its nonzeros (fewer bytes and, on the
// FP64 pipe, fewer FMAs); dense-block levels stay block CSR.
inline int level_format_of(int level_format) {
  if (const char* e = std::getenv("GBS_LEVEL_FORMAT")) return std::atoi(e);
  return level_format;
}
inline bool use_scalar_csr(const HBsr& H, int level_format) {
  const int f = level_format_of(level_format);
  if (f == 1 || H.br * H.bc == 1) return false;
  if (f == 2 || f == 3) return true;   // scalar CSR wherever possible
  return block_fill(H) <= 0.5;
}

// Sliced layout of a scalar CSR operator (sell.cuh): automatic when
// padding each slice to its longest row adds at most 10% entries; format 3
// forces it wherever B divides the rows, format 2 keeps plain CSR.
// 0 plain CSR, 1 slices in natural node order, 2 slices in sorted node
// order (HSell::node).  An irregular operator pads little once its nodes
// are sorted by row length, and its lanes then need no cross-lane sums,
// but the 32 rows of a slice come from 32 places in a window of 1024 nodes
// and their x gathers no longer share cache lines: measured slower in every
// form (C3 FP64 129 -> 181 ms, BF16 94 -> 146 ms with the velocity levels
// and transfer operators sorted).  So sorted slices are used only when
// GBS_SELL_SORT=1 forces them (tests).
inline int use_sell(const HCsr& C, int B, int level_format) {
  const int f = level_format_of(level_format);
  if (B < 1 || C.n == 0 || C.n % B != 0 || f == 2) return 0;
  const double pad = sell_padding(C, B);
  if (const char* e = std::getenv("GBS_SELL_SORT"))
    if (e[0] == '1' && pad > 0.01) return 2;
  if (f == 3) return 1;
  return pad <= 0.10 ? 1 : 0;   // 0.4 measured slower in every form
}

// Stored entries of the slices that carry explicit columns (a uniform
// slice's entries need no column load in the direct kernels).
inline int64_t explicit_entries(const HSell& S) {
  int64_t e = 0;
  for (int q = 0; q < S.nslices; ++q)
    if (S.cinfo[q] >= 0) e += (int64_t)(S.off[q + 1] - S.off[q]) * 32;
  return e;
}

template <class VT>
DevSell<VT> upload_sell(Arena& ar, const HSell& S, double* err, long long wait, cudaStream_t s,
                        std::vector<std::vector<VT>>& keep) {
  DevSell<VT> d;
  d.n = S.n;
  d.B = S.B;
  d.nslices = S.nslices;
  d.off = ar.upload(S.off.data(), S.off.size(), s);
  d.col = ar.upload(S.col.data(), S.col.size(), s);
  keep.push_back(cast_vec<VT>(S.val));
  d.val = ar.upload(keep.back().data(), keep.back().size(), s);
  d.err = err;
  d.wait = wait;
  d.cinfo = ar.upload(S.cinfo.data(), S.cinfo.size(), s);
  if (!S.node.empty()) d.node = ar.upload(S.node.data(), S.node.size(), s);
  d.uniform = S.nslices > 0 && std::all_of(S.cinfo.begin(), S.cinfo.end(),
                                           [](int32_t c) { return c < 0; });
  if (!S.uoff.empty()) {
    std::vector<int2> ui(S.uoff.size());
    for (size_t k = 0; k < ui.size(); ++k) ui[k] = make_int2(S.uoff[k], (int)S.umask[k]);
    d.uinfo = ar.upload(ui.data(), ui.size(), s);
    GBS_CUDA(cudaStreamSynchronize(s));   // ui dies here
  }
  return d;
}

// Staged (bulk-copy pipeline) kernels for FP32/BF16 forms, direct loads for
// FP64 (sell.cuh).  The direct kernels would stream only the values of a
// uniform (stencil) operator in the mixed forms, 2 or 4 bytes an entry
// against 6 or 8 with staged column indices, but measured slower there
// (C2 BF16 solve 13.5 ms direct, 13.1 staged; with the value loads and
// gathers batched four entries deep as in the identity-block kernels,
// 13.5 ms against 12.4 staged, and FP32 15.9 against 14.7):
// GBS_SELL_DIRECT=1 sends the mixed forms' uniform operators to them, =0
// keeps every one staged.
template <class VT, class AT>
inline bool sell_direct(const DevSell<VT>& A) {
  if (sizeof(AT) == 8) return true;
  if (const char* e = std::getenv("GBS_SELL_DIRECT")) return e[0] == '1';
  return false;
}
// One warp per 32-node group (B slices, contiguous stores) unless
// GBS_SELL_GROUP=0 asks for one warp per slice (measurement and tests).
inline bool sell_grouped() {
  const char* e = std::getenv("GBS_SELL_GROUP");
  return !(e && e[0] == '0');
}
template <int B, int MODE, class VT, class XT, class YT, class AT>
void sell_spmv_g(const DevSell<VT>& A, const XT* x, const YT* f, YT* y, cudaStream_t s) {
  const int64_t groups = (int64_t)A.nslices / B;
  if (sell_direct<VT, AT>(A))
    ::gbs::launch_k(k_sell_spmv_direct_g<B, MODE, VT, XT, YT, AT>, grid_for(groups * 32), 256, 0, s, A, x, f, y);
  else
    launch_sell(k_sell_spmv_g<B, MODE, VT, XT, YT, AT>, sell_smem_bytes<VT>(),
                (groups + SELL_WARPS - 1) / SELL_WARPS, s, A, x, f, y);
}
template <int MODE, class VT, class XT, class YT, class AT>
void sell_spmv(const DevSell<VT>& A, const XT* x, const YT* f, YT* y, cudaStream_t s) {
  if (A.n == 0) return;
  if (A.B > 1 && sell_grouped()) {
    switch (A.B) {
      case 2: sell_spmv_g<2, MODE, VT, XT, YT, AT>(A, x, f, y, s); break;
      case 3: sell_spmv_g<3, MODE, VT, XT, YT, AT>(A, x, f, y, s); break;
      default: sell_spmv_g<4, MODE, VT, XT, YT, AT>(A, x, f, y, s); break;
    }
  } else if (sell_direct<VT, AT>(A)) {
    ::gbs::launch_k(k_sell_spmv_direct<MODE, VT, XT, YT, AT>
        , grid_for((int64_t)A.nslices * 32), 256, 0, s, A, x, f, y);
  } else {
    launch_sell(k_sell_spmv<MODE, VT, XT, YT, AT>, sell_smem_bytes<VT>(),
                ((int64_t)A.nslices + SELL_WARPS - 1) / SELL_WARPS, s, A, x, f, y);
  }
  GBS_LAUNCH_CHECK();
}
template <int B, class VT, class XT, class AT, class OT>
void sell_relax_B(const DevSell<VT>& A, const VT* M, const XT* f, const XT* x, OT* xo,
                  cudaStream_t s) {
  const int64_t groups = (int64_t)A.nslices / B;
  if (sell_direct<VT, AT>(A)) {
    ::gbs::launch_k(k_sell_relax_direct<B, VT, XT, AT, OT>, grid_for(groups * 32), 256, 0, s, A, M, f, x, xo);
  } else {
    launch_sell(k_sell_relax<B, VT, XT, AT, OT>, sell_smem_bytes<VT>(),
                (groups + SELL_WARPS - 1) / SELL_WARPS, s, A, M, f, x, xo);
  }
}
// xo = x + M (f - A x) on a sliced level; OT: the output's type (the last
// level-0 sweep of a mixed form writes the FP64 preconditioner output).
template <class VT, class XT, class AT, class OT = XT>
void sell_relax(int B, const DevSell<VT>& A, const VT* M, const XT* f, const XT* x, OT* xo,
                cudaStream_t s) {
  if (A.n == 0) return;
  switch (B) {
    case 1: sell_relax_B<1, VT, XT, AT, OT>(A, M, f, x, xo, s); break;
    case 2: sell_relax_B<2, VT, XT, AT, OT>(A, M, f, x, xo, s); break;
    case 3: sell_relax_B<3, VT, XT, AT, OT>(A, M, f, x, xo, s); break;
    case 4: sell_relax_B<4, VT, XT, AT, OT>(A, M, f, x, xo, s); break;
  }
  GBS_LAUNCH_CHECK();
}

template <int B, bool TR, int MODE, class VT, class XT, class YT, class AT>
void spmv_B(const DevBsr<VT>& A, const XT* x, const YT* f, YT* y, cudaStream_t s);

template <int MODE, class VT, class XT, class YT, class AT>
void csr_spmv(const DevCsr<VT>& A, const XT* x, const YT* f, YT* y, cudaStream_t s) {
  if (A.n == 0) return;
  if (A.G) {   // a scalar CSR matrix is a block CSR matrix with 1 x 1 blocks
    DevBsr<VT> v;
    v.nbr = v.nbc = A.n;
    v.rp = A.rp;
    v.col = A.col;
    v.val = A.val;
    v.G = A.G;
    spmv_B<1, false, MODE, VT, XT, YT, AT>(v, x, f, y, s);
    GBS_LAUNCH_CHECK();
    return;
  }
  switch (A.S) {
    case 2: ::gbs::launch_k(k_csr_spmv<2, MODE, VT, XT, YT, AT>, grid_for(row_threads_s<1, 2>(A.n)), 256, 0, s, A, x, f, y); break;
    case 4: ::gbs::launch_k(k_csr_spmv<4, MODE, VT, XT, YT, AT>, grid_for(row_threads_s<1, 4>(A.n)), 256, 0, s, A, x, f, y); break;
    case 8: ::gbs::launch_k(k_csr_spmv<8, MODE, VT, XT, YT, AT>, grid_for(row_threads_s<1, 8>(A.n)), 256, 0, s, A, x, f, y); break;
    default: ::gbs::launch_k(k_csr_spmv<1, MODE, VT, XT, YT, AT>, grid_for(row_threads_s<1, 1>(A.n)), 256, 0, s, A, x, f, y);
  }
  GBS_LAUNCH_CHECK();
}
template <int B, class VT, class XT, class AT>
void csr_relax_B(const DevCsr<VT>& A, const VT* M, const XT* f, const XT* x, XT* xo, cudaStream_t s) {
  const int nn = A.n / B;
  switch (A.S) {
    case 2: ::gbs::launch_k(k_csr_relax<B, 2, VT, XT, AT>, grid_for(row_threads_s<B, 2>(nn)), 256, 0, s, A, M, f, x, xo); break;
    case 4:
      if constexpr (B * 4 <= 32) ::gbs::launch_k(k_csr_relax<B, 4, VT, XT, AT>, grid_for(row_threads_s<B, 4>(nn)), 256, 0, s, A, M, f, x, xo);
      break;
    case 8:
      if constexpr (B * 8 <= 32) ::gbs::launch_k(k_csr_relax<B, 8, VT, XT, AT>, grid_for(row_threads_s<B, 8>(nn)), 256, 0, s, A, M, f, x, xo);
      break;
    default: ::gbs::launch_k(k_csr_relax<B, 1, VT, XT, AT>, grid_for(row_threads_s<B, 1>(nn)), 256, 0, s, A, M, f, x, xo);
  }
}
template <class VT, class XT, class AT>
void csr_relax(int B, DevCsr<VT> A, const VT* M, const XT* f, const XT* x, XT* xo, cudaStream_t s) {
  if (A.n == 0) return;
  while (A.S > 1 && B * A.S > 32) A.S >>= 1;
  switch (B) {
    case 1: csr_relax_B<1, VT, XT, AT>(A, M, f, x, xo, s); break;
    case 2: csr_relax_B<2, VT, XT, AT>(A, M, f, x, xo, s); break;
    case 3: csr_relax_B<3, VT, XT, AT>(A, M, f, x, xo, s); break;
    case 4: csr_relax_B<4, VT, XT, AT>(A, M, f, x, xo, s); break;
  }
  GBS_LAUNCH_CHECK();
}

template <int MODE, class VT, class XT, class YT, class AT>
void bsell_spmv(int B, const DevBSell<VT>& A, const XT* x, const YT* f, YT* y, cudaStream_t s) {
  if (A.nslices == 0) return;
  const unsigned g = grid_for((int64_t)A.nslices * 32);
  switch (B) {
    case 1: ::gbs::launch_k(k_bsell_spmv<1, MODE, VT, XT, YT, AT>, g, 256, 0, s, A, x, f, y); break;
    case 2: ::gbs::launch_k(k_bsell_spmv<2, MODE, VT, XT, YT, AT>, g, 256, 0, s, A, x, f, y); break;
    case 3: ::gbs::launch_k(k_bsell_spmv<3, MODE, VT, XT, YT, AT>, g, 256, 0, s, A, x, f, y); break;
    case 4: ::gbs::launch_k(k_bsell_spmv<4, MODE, VT, XT, YT, AT>, g, 256, 0, s, A, x, f, y); break;
  }
  GBS_LAUNCH_CHECK();
}
template <class VT, class XT, class AT>
void bsell_relax(int B, const DevBSell<VT>& A, const VT* M, const XT* f, const XT* x, XT* xo,
                 cudaStream_t s) {
  if (A.nslices == 0) return;
  const unsigned g = grid_for((int64_t)A.nslices * 32);
  switch (B) {
    case 1: ::gbs::launch_k(k_bsell_relax<1, VT, XT, AT>, g, 256, 0, s, A, M, f, x, xo); break;
    case 2: ::gbs::launch_k(k_bsell_relax<2, VT, XT, AT>, g, 256, 0, s, A, M, f, x, xo); break;
    case 3: ::gbs::launch_k(k_bsell_relax<3, VT, XT, AT>, g, 256, 0, s, A, M, f, x, xo); break;
    case 4: ::gbs::launch_k(k_bsell_relax<4, VT, XT, AT>, g, 256, 0, s, A, M, f, x, xo); break;
  }
  GBS_LAUNCH_CHECK();
}

// ------------------------------------------------------------ launch helpers
template <int B, bool TR, int MODE, class VT, class XT, class YT, class AT>
void spmv_B(const DevBsr<VT>& A, const XT* x, const YT* f, YT* y, cudaStream_t s) {
  if (A.nbr == 0) return;
  const int64_t nt = (int64_t)A.nbr * A.G;
  switch (A.G) {
    case 8: ::gbs::launch_k(k_spmv_w<B, 8, TR, MODE, VT, XT, YT, AT>, grid_for(nt), 256, 0, s, A, x, f, y); break;
    case 16: ::gbs::launch_k(k_spmv_w<B, 16, TR, MODE, VT, XT, YT, AT>, grid_for(nt), 256, 0, s, A, x, f, y); break;
    case 32: ::gbs::launch_k(k_spmv_w<B, 32, TR, MODE, VT, XT, YT, AT>, grid_for(nt), 256, 0, s, A, x, f, y); break;
    case 256: ::gbs::launch_k(k_spmv_w<B, 256, TR, MODE, VT, XT, YT, AT>, grid_for(nt), 256, 0, s, A, x, f, y); break;
    default:
      switch (A.S) {
        case 2: ::gbs::launch_k(k_spmv<B, 2, TR, MODE, VT, XT, YT, AT>, grid_for(row_threads_s<B, 2>(A.nbr)), 256, 0, s, A, x, f, y); break;
        case 4:
          if constexpr (B * 4 <= 32) ::gbs::launch_k(k_spmv<B, 4, TR, MODE, VT, XT, YT, AT>, grid_for(row_threads_s<B, 4>(A.nbr)), 256, 0, s, A, x, f, y);
          break;
        case 8:
          if constexpr (B * 8 <= 32) ::gbs::launch_k(k_spmv<B, 8, TR, MODE, VT, XT, YT, AT>, grid_for(row_threads_s<B, 8>(A.nbr)), 256, 0, s, A, x, f, y);
          break;
        default: ::gbs::launch_k(k_spmv<B, 1, TR, MODE, VT, XT, YT, AT>, grid_for(row_threads_s<B, 1>(A.nbr)), 256, 0, s, A, x, f, y);
      }
  }
}
template <bool TR, int MODE, class VT, class XT, class YT, class AT>
void spmv(int B, const DevBsr<VT>& A, const XT* x, const YT* f, YT* y, cudaStream_t s) {
  switch (B) {
    case 1: spmv_B<1, TR, MODE, VT, XT, YT, AT>(A, x, f, y, s); break;
    case 2: spmv_B<2, TR, MODE, VT, XT, YT, AT>(A, x, f, y, s); break;
    case 3: spmv_B<3, TR, MODE, VT, XT, YT, AT>(A, x, f, y, s); break;
    case 4: spmv_B<4, TR, MODE, VT, XT, YT, AT>(A, x, f, y, s); break;
  }
  GBS_LAUNCH_CHECK();
}
template <bool TR, class VT, class XT, class AT>
void relax(int B, const DevBsr<VT>& A, const VT* M, const XT* f, const XT* x, XT* xo,
           cudaStream_t s) {
  if (A.nbr == 0) return;
#define GBS_RELAX(BB)                                                                            \
  switch (A.G) {                                                                                 \
    case 8: ::gbs::launch_k(k_relax_w<BB, 8, TR, VT, XT, AT>, grid_for((int64_t)A.nbr * 8), 256, 0, s, A, M, f, x, xo); break;   \
    case 16: ::gbs::launch_k(k_relax_w<BB, 16, TR, VT, XT, AT>, grid_for((int64_t)A.nbr * 16), 256, 0, s, A, M, f, x, xo); break; \
    case 32: ::gbs::launch_k(k_relax_w<BB, 32, TR, VT, XT, AT>, grid_for((int64_t)A.nbr * 32), 256, 0, s, A, M, f, x, xo); break; \
    case 256: ::gbs::launch_k(k_relax_w<BB, 256, TR, VT, XT, AT>, grid_for((int64_t)A.nbr * 256), 256, 0, s, A, M, f, x, xo); break; \
    default:                                                                                     \
      switch (A.S) {                                                                             \
        case 2: ::gbs::launch_k(k_relax<BB, 2, TR, VT, XT, AT>, grid_for(row_threads_s<BB, 2>(A.nbr)), 256, 0, s, A, M, f, x, xo); break; \
        case 4:                                                                                  \
          if constexpr (BB * 4 <= 32) ::gbs::launch_k(k_relax<BB, 4, TR, VT, XT, AT>, grid_for(row_threads_s<BB, 4>(A.nbr)), 256, 0, s, A, M, f, x, xo); \
          break;                                                                                 \
        case 8:                                                                                  \
          if constexpr (BB * 8 <= 32) ::gbs::launch_k(k_relax<BB, 8, TR, VT, XT, AT>, grid_for(row_threads_s<BB, 8>(A.nbr)), 256, 0, s, A, M, f, x, xo); \
          break;                                                                                 \
        default: ::gbs::launch_k(k_relax<BB, 1, TR, VT, XT, AT>, grid_for(row_threads_s<BB, 1>(A.nbr)), 256, 0, s, A, M, f, x, xo); \
      }                                                                                          \
  }
  switch (B) {
    case 1: GBS_RELAX(1); break;
    case 2: GBS_RELAX(2); break;
    case 3: GBS_RELAX(3); break;
    case 4: GBS_RELAX(4); break;
  }
#undef GBS_RELAX
  GBS_LAUNCH_CHECK();
}
template <bool TR, class VT, class XT, class AT>
void mapply(int B, int nbr, const VT* M, const XT* f, XT* x, cudaStream_t s) {
  if (nbr == 0) return;
#define GBS_MAP(BB) \
  ::gbs::launch_k(k_mapply<BB, TR, VT, XT, AT>, grid_for(row_threads<BB>(nbr)), 256, 0, s, nbr, M, f, x)
  switch (B) {
    case 1: GBS_MAP(1); break;
    case 2: GBS_MAP(2); break;
    case 3: GBS_MAP(3); break;
    case 4: GBS_MAP(4); break;
  }
#undef GBS_MAP
  GBS_LAUNCH_CHECK();
}

// ---- levels stored as S (x) I_B (iso.cuh): NV = B interleaved components
// Lanes per row of S in the iso products: the scalar split by row length
// (csr_split), widened on small levels until they have LANES_TARGET lanes
// while every lane keeps at least four entries, up to a warp a row; a CTA
// of 256 threads a row (G = 256) when even a warp a row leaves a level of
// long rows with a quarter of that.  Measured (C3 velocity, 8 lanes a row):
// the 42-row level-3 restriction, 481 entries a row, took 24 us in BF16
// and 49 us in FP64; its 1108-row level-2 counterpart 29 and 48 us.
template <class VT>
void set_iso_lanes(DevCsr<VT>& d, int64_t rows, int64_t nnz) {
  const double avg = rows ? (double)nnz / rows : 0.0;
  int S = csr_split(rows, nnz);
  while (S < 32 && rows * S < LANES_TARGET && avg >= 4.0 * S) S *= 2;
  d.S = S;
  d.G = S == 32 && rows * 32 < LANES_TARGET / 4 && avg >= 128.0 ? 256 : 0;
  if (const char* e = std::getenv("GBS_ISO_SPLIT")) {   // tuning override: 1 .. 32, 256
    const int v = std::atoi(e);
    if (v == 256) { d.S = 32; d.G = 256; }
    else if (v == 1 || v == 2 || v == 4 || v == 8 || v == 16 || v == 32) { d.S = v; d.G = 0; }
  }
}
// Batched loads in the iso CSR rows (iso_csr_row): FP32 accumulation, or a
// level small enough to be latency-bound (fewer lanes than LANES_TARGET).
template <class AT, class VT>
inline bool iso_batched(const DevCsr<VT>& A) {
  return sizeof(AT) == 4 || (int64_t)A.n * A.S < LANES_TARGET;
}
template <int NV, int MODE, class VT, class XT, class YT, class AT>
void iso_csr_spmv_nv(const DevCsr<VT>& A, const XT* x, const YT* f, YT* y, cudaStream_t s) {
  if (A.G == 256) {
    ::gbs::launch_k(k_iso_csr_spmv_cta<NV, 256, MODE, VT, XT, YT, AT>, A.n, 256, 0, s, A, x, f, y);
    return;
  }
#define GBS_ISO(SS)                                                                              \
  if (iso_batched<AT>(A)) ::gbs::launch_k(k_iso_csr_spmv<NV, SS, MODE, VT, XT, YT, AT, true>,    \
                                          grid_for(row_threads_s<1, SS>(A.n)), 256, 0, s, A, x, f, y); \
  else ::gbs::launch_k(k_iso_csr_spmv<NV, SS, MODE, VT, XT, YT, AT, false>,                    \
                       grid_for(row_threads_s<1, SS>(A.n)), 256, 0, s, A, x, f, y)
  switch (A.S) {
    case 2: GBS_ISO(2); break;
    case 4: GBS_ISO(4); break;
    case 8: GBS_ISO(8); break;
    case 16: GBS_ISO(16); break;
    case 32: GBS_ISO(32); break;
    default: GBS_ISO(1);
  }
#undef GBS_ISO
}
// MODE SET / RESID / ADD with S in slices (sl) or plain CSR.
template <int MODE, class VT, class XT, class YT, class AT>
void iso_spmv(int NV, const DevCsr<VT>& Ac, const DevSell<VT>& As, bool sl, const XT* x,
              const YT* f, YT* y, cudaStream_t s) {
  if (sl) {
    if (As.n == 0) return;
    const unsigned g = grid_for((int64_t)As.nslices * 32);
    switch (NV) {
      case 1: ::gbs::launch_k(k_iso_sell_spmv<1, MODE, VT, XT, YT, AT>, g, 256, 0, s, As, x, f, y); break;
      case 2: ::gbs::launch_k(k_iso_sell_spmv<2, MODE, VT, XT, YT, AT>, g, 256, 0, s, As, x, f, y); break;
      case 3: ::gbs::launch_k(k_iso_sell_spmv<3, MODE, VT, XT, YT, AT>, g, 256, 0, s, As, x, f, y); break;
      case 4: ::gbs::launch_k(k_iso_sell_spmv<4, MODE, VT, XT, YT, AT>, g, 256, 0, s, As, x, f, y); break;
    }
  } else {
    if (Ac.n == 0) return;
    switch (NV) {
      case 1: iso_csr_spmv_nv<1, MODE, VT, XT, YT, AT>(Ac, x, f, y, s); break;
      case 2: iso_csr_spmv_nv<2, MODE, VT, XT, YT, AT>(Ac, x, f, y, s); break;
      case 3: iso_csr_spmv_nv<3, MODE, VT, XT, YT, AT>(Ac, x, f, y, s); break;
      case 4: iso_csr_spmv_nv<4, MODE, VT, XT, YT, AT>(Ac, x, f, y, s); break;
    }
  }
  GBS_LAUNCH_CHECK();
}
template <int NV, class VT, class XT, class AT, class OT>
void iso_relax_nv(const DevCsr<VT>& Ac, const DevSell<VT>& As, bool sl, const VT* M, const XT* f,
                  const XT* x, OT* xo, cudaStream_t s) {
  if (sl) {
    ::gbs::launch_k(k_iso_sell_relax<NV, VT, XT, AT, OT>
        , grid_for((int64_t)As.nslices * 32), 256, 0, s, As, M, f, x, xo);
    return;
  }
  if (Ac.G == 256) {
    ::gbs::launch_k(k_iso_csr_relax_cta<NV, 256, VT, XT, AT, OT>, Ac.n, 256, 0, s, Ac, M, f, x, xo);
    return;
  }
#define GBS_ISO(SS)                                                                          \
  if (iso_batched<AT>(Ac)) ::gbs::launch_k(k_iso_csr_relax<NV, SS, VT, XT, AT, OT, true>,    \
                                           grid_for(row_threads_s<1, SS>(Ac.n)), 256, 0, s, Ac, M, f, x, xo); \
  else ::gbs::launch_k(k_iso_csr_relax<NV, SS, VT, XT, AT, OT, false>,                     \
                       grid_for(row_threads_s<1, SS>(Ac.n)), 256, 0, s, Ac, M, f, x, xo)
  switch (Ac.S) {
    case 2: GBS_ISO(2); break;
    case 4: GBS_ISO(4); break;
    case 8: GBS_ISO(8); break;
    case 16: GBS_ISO(16); break;
    case 32: GBS_ISO(32); break;
    default: GBS_ISO(1);
  }
#undef GBS_ISO
}
// xo = x + (diag(m) (x) I) (f - (S (x) I) x); OT as in sell_relax.
template <class VT, class XT, class AT, class OT = XT>
void iso_relax(int NV, const DevCsr<VT>& Ac, const DevSell<VT>& As, bool sl, const VT* M,
               const XT* f, const XT* x, OT* xo, cudaStream_t s) {
  if (sl ? As.n == 0 : Ac.n == 0) return;
  switch (NV) {
    case 1: iso_relax_nv<1, VT, XT, AT, OT>(Ac, As, sl, M, f, x, xo, s); break;
    case 2: iso_relax_nv<2, VT, XT, AT, OT>(Ac, As, sl, M, f, x, xo, s); break;
    case 3: iso_relax_nv<3, VT, XT, AT, OT>(Ac, As, sl, M, f, x, xo, s); break;
    case 4: iso_relax_nv<4, VT, XT, AT, OT>(Ac, As, sl, M, f, x, xo, s); break;
  }
  GBS_LAUNCH_CHECK();
}
// Mixed forms: the same step with x = m .* f formed in the gather
// (k_iso_sell_presmooth_otf; A holds S itself).
template <class VT, class XT, class AT>
void iso_presmooth_otf(int NV, const DevSell<VT>& A, const VT* M, const XT* f, XT* x, XT* r,
                       cudaStream_t s) {
  if (A.n == 0) return;
  const unsigned g = grid_for((int64_t)A.nslices * 32);
  switch (NV) {
    case 1: ::gbs::launch_k(k_iso_sell_presmooth_otf<1, VT, XT, AT>, g, 256, 0, s, A, M, f, x, r); break;
    case 2: ::gbs::launch_k(k_iso_sell_presmooth_otf<2, VT, XT, AT>, g, 256, 0, s, A, M, f, x, r); break;
    case 3: ::gbs::launch_k(k_iso_sell_presmooth_otf<3, VT, XT, AT>, g, 256, 0, s, A, M, f, x, r); break;
    case 4: ::gbs::launch_k(k_iso_sell_presmooth_otf<4, VT, XT, AT>, g, 256, 0, s, A, M, f, x, r); break;
  }
  GBS_LAUNCH_CHECK();
}
template <class VT, class XT, class AT>
void iso_presmooth(int NV, const DevSell<VT>& AM, const VT* M, const XT* f, XT* x, XT* r,
                   cudaStream_t s) {
  if (AM.n == 0) return;
  const unsigned g = grid_for((int64_t)AM.nslices * 32);
  switch (NV) {
    case 1: ::gbs::launch_k(k_iso_sell_presmooth<1, VT, XT, AT>, g, 256, 0, s, AM, M, f, x, r); break;
    case 2: ::gbs::launch_k(k_iso_sell_presmooth<2, VT, XT, AT>, g, 256, 0, s, AM, M, f, x, r); break;
    case 3: ::gbs::launch_k(k_iso_sell_presmooth<3, VT, XT, AT>, g, 256, 0, s, AM, M, f, x, r); break;
    case 4: ::gbs::launch_k(k_iso_sell_presmooth<4, VT, XT, AT>, g, 256, 0, s, AM, M, f, x, r); break;
  }
  GBS_LAUNCH_CHECK();
}
template <class VT, class XT, class AT>
void iso_mapply(int NV, int64_t n, const VT* M, const XT* f, XT* x, cudaStream_t s) {
  if (n == 0) return;
  n /= NV;   // nodes
  const unsigned g = grid_for(n);
  switch (NV) {
    case 1: ::gbs::launch_k(k_iso_mapply<1, VT, XT, AT>, g, 256, 0, s, n, M, f, x); break;
    case 2: ::gbs::launch_k(k_iso_mapply<2, VT, XT, AT>, g, 256, 0, s, n, M, f, x); break;
    case 3: ::gbs::launch_k(k_iso_mapply<3, VT, XT, AT>, g, 256, 0, s, n, M, f, x); break;
    case 4: ::gbs::launch_k(k_iso_mapply<4, VT, XT, AT>, g, 256, 0, s, n, M, f, x); break;
  }
  GBS_LAUNCH_CHECK();
}
template <class VT, class XT, class AT>
void iso_cast_mapply(int NV, int64_t n, const VT* M, const double* r64, XT* fin, XT* x,
                     cudaStream_t s) {
  if (n == 0) return;
  n /= NV;   // nodes
  const unsigned g = grid_for(n);
  switch (NV) {
    case 1: ::gbs::launch_k(k_iso_cast_mapply<1, VT, XT, AT>, g, 256, 0, s, n, M, r64, fin, x); break;
    case 2: ::gbs::launch_k(k_iso_cast_mapply<2, VT, XT, AT>, g, 256, 0, s, n, M, r64, fin, x); break;
    case 3: ::gbs::launch_k(k_iso_cast_mapply<3, VT, XT, AT>, g, 256, 0, s, n, M, r64, fin, x); break;
    case 4: ::gbs::launch_k(k_iso_cast_mapply<4, VT, XT, AT>, g, 256, 0, s, n, M, r64, fin, x); break;
  }
  GBS_LAUNCH_CHECK();
}

template <class TI, class TO>
void cast(int64_t n, const TI* in, TO* out, cudaStream_t s) {
  if (n == 0) return;
  unsigned g = (unsigned)std::min<int64_t>((n + 255) / 256, 152 * 16);
  ::gbs::launch_k(k_cast<TI, TO>, g, 256, 0, s, n, in, out);
  GBS_LAUNCH_CHECK();
}

// ------------------------------------------------------------------ AMG
template <int P>
struct DevAmg {
  using VT = typename FormT<P>::VT;
  using ST = typename FormT<P>::ST;
  using AT = ST;

  struct Lev {
    DevBsr<VT> A, Pm, R;
    DevCsr<VT> Ac, Pc, Rc;              // scalar CSR forms (per-level format choice)
    DevSell<VT> As, Ps, Rs;             // sliced forms of the scalar CSR operators
    // ILUT relaxation: L strictly lower, Us = D^-1 U strictly upper, their
    // transposes (adjoint), D^-1, and three work vectors
    bool ilu = false;
    DevCsr<VT> Li, Ui, LiT, UiT;
    const VT* dinv = nullptr;
    ST *wa = nullptr, *wb = nullptr, *wc = nullptr;
    int64_t nnz_Li = 0, nnz_Ui = 0;
    bool a_csr = false, p_csr = false, r_csr = false;
    bool a_sell = false, p_sell = false, r_sell = false;
    // A = S (x) I_B (every block of A, P, R and M a multiple of I_B): Ac/As,
    // Pc/Ps, Rc/Rs hold S and the scalar P and R (one row per node), M one
    // value per node, AcT = S^T for the transposed cycle (iso.cuh)
    bool iso = false;
    DevCsr<VT> AcT;
    int64_t xsl_A = 0, xsl_P = 0, xsl_R = 0, xsl_AM = 0;  // slices: entries with column loads
    bool dir_A = false, dir_P = false, dir_R = false;       // slices read by direct kernels
    DevBSell<VT> Ab;                    // block-row slices of A (FP64 block levels)
    bool a_bsell = false;
    int64_t slots_Ab = 0;
    // fused zero-guess pre-smoothing + residual (FP64 forms): A M in the
    // level's slices (fused 1: scalar slices AMs; 2: block-row slices AMb)
    int fused = 0;
    DevSell<VT> AMs;
    DevBSell<VT> AMb;
    int64_t slots_AM = 0, sl_AM = 0;
    const VT* M = nullptr;
    ST *f = nullptr, *r = nullptr, *x = nullptr, *xt = nullptr, *e = nullptr;
    int64_t n = 0;
    int64_t nnzb_A = 0, nnzb_P = 0, nnzb_R = 0;
    int64_t nnz_A = 0, nnz_P = 0, nnz_R = 0;  // scalar nonzeros when in CSR
    int64_t slots_A = 0, slots_P = 0, slots_R = 0;  // sliced: stored entries
    int64_t sl_A = 0, sl_P = 0, sl_R = 0;           // sliced: slices
  };
  int B = 1;
  int npre = 1, npost = 1;
  int ilu_sweeps = 2;
  double ilu_omega = 1.0;
  std::vector<Lev> lev;        // lev.back() is the coarsest (no A/P/R/M used)
  const ST* Ainv = nullptr;    // coarse inverse (ST precision)
  const ST* AinvT = nullptr;
  int nc = 0;                  // scalar size of the coarsest level
  Arena ar;

  void build(const HAmg& H, const PrecondOptions& o, cudaStream_t s) {
    B = H.B;
    npre = o.npre;
    npost = o.npost;
    ilu_sweeps = o.ilut_sweeps;
    ilu_omega = o.ilut_omega;
    std::vector<std::vector<VT>> keep;
    for (size_t l = 0; l < H.levels.size(); ++l) {
      const HLevel& h = H.levels[l];
      Lev L;
      L.n = (int64_t)h.A.nbr * B;
      if (iso_level(h, o)) {
        build_iso(h, o, L, s, keep);
      } else {
        L.a_csr = use_scalar_csr(h.A, o.level_format);
        L.p_csr = use_scalar_csr(h.P, o.level_format);
        L.r_csr = use_scalar_csr(h.R, o.level_format);
        // the block form of A stays resident when the adjoint may need A^T
        if (!L.a_csr || o.tmaps) L.A = upload_bsr<VT, AT>(ar, h.A, o.tmaps, s, keep);
        else { L.A.nbr = h.A.nbr; L.A.nbc = h.A.nbc; }
        if (!L.a_csr && use_bsell<AT>(h.A, L.A.G)) {
          const HBSell Sb = to_bsell(h.A, BSELL_WINDOW);
          L.Ab = upload_bsell<VT>(ar, Sb, s, keep);
          L.a_bsell = true;
          L.slots_Ab = (int64_t)Sb.col.size();
          GBS_CUDA(cudaStreamSynchronize(s));  // Sb's host arrays die here
        }
        // scalar CSR, as plain rows or in slices
        auto scalar = [&](const HBsr& Hm, DevCsr<VT>& dc, DevSell<VT>& ds, bool& sl, int64_t& nnz,
                          int64_t& slots, int64_t& nsl, int64_t& xsl, bool& dir) {
          HCsr c = to_scalar_csr(Hm);
          nnz = (int64_t)c.col.size();
          const int how = use_sell(c, B, o.level_format);
          sl = how != 0;
          if (sl) {
            const HSell S = to_sell(c, B, how == 2);
            slots = (int64_t)S.col.size();
            nsl = S.nslices;
            xsl = explicit_entries(S);
            ds = upload_sell<VT>(ar, S, o.err, o.wait_cycles, s, keep);
            dir = sell_direct<VT, AT>(ds);
            GBS_CUDA(cudaStreamSynchronize(s));  // S's host arrays die here
          } else {
            dc = upload_csr<VT>(ar, c, s, keep);
          }
        };
        if (L.a_csr) scalar(h.A, L.Ac, L.As, L.a_sell, L.nnz_A, L.slots_A, L.sl_A, L.xsl_A, L.dir_A);
        if (L.p_csr) scalar(h.P, L.Pc, L.Ps, L.p_sell, L.nnz_P, L.slots_P, L.sl_P, L.xsl_P, L.dir_P);
        else L.Pm = upload_bsr<VT, AT>(ar, h.P, false, s, keep);
        if (L.r_csr) scalar(h.R, L.Rc, L.Rs, L.r_sell, L.nnz_R, L.slots_R, L.sl_R, L.xsl_R, L.dir_R);
        else L.R = upload_bsr<VT, AT>(ar, h.R, false, s, keep);
        keep.push_back(cast_vec<VT>(h.M));
        L.M = ar.upload(keep.back().data(), keep.back().size(), s);
        if (!h.ilu.d.empty()) {
          L.ilu = true;
          HCsr Us = h.ilu.U;
          for (int i = 0; i < Us.n; ++i)
            for (int k = Us.ptr[i]; k < Us.ptr[i + 1]; ++k) Us.val[k] /= h.ilu.d[i];
          std::vector<double> di(h.ilu.d.size());
          for (size_t i = 0; i < di.size(); ++i) di[i] = 1.0 / h.ilu.d[i];
          L.Li = upload_csr<VT>(ar, h.ilu.L, s, keep);
          L.Ui = upload_csr<VT>(ar, Us, s, keep);
          if (o.tmaps) {
            L.LiT = upload_csr<VT>(ar, transpose(h.ilu.L), s, keep);
            L.UiT = upload_csr<VT>(ar, transpose(Us), s, keep);
          }
          keep.push_back(cast_vec<VT>(di));
          L.dinv = ar.upload(keep.back().data(), keep.back().size(), s);
          L.wa = ar.alloc<ST>(L.n);
          L.wb = ar.alloc<ST>(L.n);
          L.wc = ar.alloc<ST>(L.n);
          L.nnz_Li = (int64_t)h.ilu.L.col.size();
          L.nnz_Ui = (int64_t)h.ilu.U.col.size();
          GBS_CUDA(cudaStreamSynchronize(s));  // host staging (Us, transposes) dies here
        }
        if (use_fused<AT>(h, o) && (L.a_sell || L.a_bsell)) {
          const HBsr AM = scale_columns(h.A, h.M);
          if (L.a_bsell) {
            const HBSell Sb = to_bsell(AM, BSELL_WINDOW);
            L.AMb = upload_bsell<VT>(ar, Sb, s, keep);
            L.slots_AM = (int64_t)Sb.col.size();
            L.fused = 2;
            GBS_CUDA(cudaStreamSynchronize(s));
          } else {
            const HCsr c = to_scalar_csr(AM);
            const int how = use_sell(c, B, o.level_format);
            if (how) {
              const HSell Sa = to_sell(c, B, how == 2);
              L.AMs = upload_sell<VT>(ar, Sa, o.err, o.wait_cycles, s, keep);
              L.slots_AM = (int64_t)Sa.col.size();
              L.sl_AM = Sa.nslices;
              L.xsl_AM = explicit_entries(Sa);
              L.fused = 1;
              GBS_CUDA(cudaStreamSynchronize(s));
            }
          }
        }
      }
      L.f = ar.alloc<ST>(L.n);
      L.r = ar.alloc<ST>(L.n);
      L.x = ar.alloc<ST>(L.n);
      L.xt = ar.alloc<ST>(L.n);
      L.e = ar.alloc<ST>(L.n);
      L.nnzb_A = h.A.nnzb();
      L.nnzb_P = h.P.nnzb();
      L.nnzb_R = h.R.nnzb();
      lev.push_back(L);
    }
    Lev C;
    C.n = (int64_t)H.Ac.nbr * B;
    C.nnzb_A = H.Ac.nnzb();
    C.f = ar.alloc<ST>(C.n);
    C.e = ar.alloc<ST>(C.n);
    C.x = ar.alloc<ST>(C.n);
    lev.push_back(C);
    nc = (int)C.n;
    std::vector<ST> inv(H.Ainv.size()), invT(H.Ainv.size());
    for (int i = 0; i < nc; ++i)
      for (int j = 0; j < nc; ++j) {
        inv[(size_t)i * nc + j] = (ST)H.Ainv[(size_t)i * nc + j];
        invT[(size_t)j * nc + i] = (ST)H.Ainv[(size_t)i * nc + j];
      }
    Ainv = ar.upload(inv.data(), inv.size(), s);
    AinvT = ar.upload(invT.data(), invT.size(), s);
    GBS_CUDA(cudaStreamSynchronize(s));  // host staging buffers die here
  }

  // A level stored as S (x) I_B: every block of A, P, R and of the smoother
  // is a multiple of the identity (checked bitwise; not for ILUT levels,
  // nor under level_format 1, which keeps every level in block form).
  // GBS_ISO=0 / 1 overrides iso_blocks (measurement and tests).
  bool iso_level(const HLevel& h, const PrecondOptions& o) const {
    bool on = o.iso;
    if (const char* e = std::getenv("GBS_ISO")) on = e[0] != '0';
    if (level_format_of(o.level_format) == 1) on = false;
    if (!on || !h.ilu.d.empty() || h.M.empty()) return false;
    // a scalar level is S (x) I_1: one lane a row, in slices or wide CSR
    return B == 1 || (is_iso(h.A) && is_iso(h.P) && is_iso(h.R) && is_iso_blocks(h.M, B));
  }
  void build_iso(const HLevel& h, const PrecondOptions& o, Lev& L, cudaStream_t s,
                 std::vector<std::vector<VT>>& keep) {
    L.iso = true;
    L.A.nbr = h.A.nbr;
    L.A.nbc = h.A.nbc;
    L.a_csr = L.p_csr = L.r_csr = true;
    L.dir_A = L.dir_P = L.dir_R = true;   // the iso kernels load every slice directly
    // S, P and R as scalar CSR with one row per node, in slices where
    // they pad little (use_sell with one component a node)
    auto scalar = [&](const HCsr& c, DevCsr<VT>& dc, DevSell<VT>& ds, bool& sl, int64_t& nnz,
                      int64_t& slots, int64_t& nsl, int64_t& xsl) {
      nnz = (int64_t)c.col.size();
      const int how = use_sell(c, 1, o.level_format);
      sl = how != 0;
      if (sl) {
        const HSell S = to_sell(c, 1, how == 2);
        slots = (int64_t)S.col.size();
        nsl = S.nslices;
        xsl = explicit_entries(S);
        ds = upload_sell<VT>(ar, S, o.err, o.wait_cycles, s, keep);
        GBS_CUDA(cudaStreamSynchronize(s));  // S's host arrays die here
      } else {
        dc = upload_csr<VT>(ar, c, s, keep);
        set_iso_lanes(dc, c.n, nnz);
      }
    };
    const HCsr Sa = iso_scalar(h.A);
    scalar(Sa, L.Ac, L.As, L.a_sell, L.nnz_A, L.slots_A, L.sl_A, L.xsl_A);
    scalar(iso_scalar(h.P), L.Pc, L.Ps, L.p_sell, L.nnz_P, L.slots_P, L.sl_P, L.xsl_P);
    scalar(iso_scalar(h.R), L.Rc, L.Rs, L.r_sell, L.nnz_R, L.slots_R, L.sl_R, L.xsl_R);
    if (o.tmaps) {
      const HCsr St = transpose(Sa);
      L.AcT = upload_csr<VT>(ar, St, s, keep);
      set_iso_lanes(L.AcT, St.n, (int64_t)St.col.size());
      GBS_CUDA(cudaStreamSynchronize(s));
    }
    keep.push_back(cast_vec<VT>(iso_diag(h.M, B)));
    L.M = ar.upload(keep.back().data(), keep.back().size(), s);
    if (sizeof(AT) < 8 && o.npre == 1 && L.a_sell && fuse_enabled()) {
      L.fused = 3;   // mixed forms: x = m .* f formed in the residual's gather
    } else if (use_fused<AT>(h, o) && L.a_sell) {
      const HCsr c = iso_scalar(scale_columns(h.A, h.M));
      const int how = use_sell(c, 1, o.level_format);
      if (how) {
        const HSell Sm = to_sell(c, 1, how == 2);
        L.AMs = upload_sell<VT>(ar, Sm, o.err, o.wait_cycles, s, keep);
        L.slots_AM = (int64_t)Sm.col.size();
        L.sl_AM = Sm.nslices;
        L.xsl_AM = explicit_entries(Sm);
        L.fused = 1;
        GBS_CUDA(cudaStreamSynchronize(s));
      }
    }
  }

  int64_t n0() const { return lev[0].n; }
  int layout(size_t l) const {
    const Lev& L = lev[l];
    const int base = L.a_bsell ? 3 : L.a_sell ? 2 : L.a_csr ? 1 : 0;
    return base + (L.fused ? 4 : 0) + (L.iso ? 8 : 0);
  }

  // z = S r with S the approximate (LU)^-1 of an ILUT level (S^T when TR):
  // ilu_sweeps Jacobi sweeps per triangular solve.  Returns the buffer
  // holding z (one of the level's work vectors; r may be any other vector).
  template <bool TR>
  const ST* ilu_apply(Lev& L, const ST* r, cudaStream_t s) {
    const unsigned g = grid_for(L.n);
    ST* pp[2] = {L.wa, L.wb};
    int q = 0;
    const ST* y = r;
    const DevCsr<VT>& first = TR ? L.UiT : L.Li;
    const DevCsr<VT>& second = TR ? L.LiT : L.Ui;
    for (int k = 0; k < ilu_sweeps; ++k) {   // forward: y = r - L y; transposed: v = r - Us^T v
      csr_spmv<SPMV_RESID, VT, ST, ST, AT>(first, y, r, pp[q], s);
      y = pp[q];
      q ^= 1;
    }
    ::gbs::launch_k(k_vscale<VT, ST>, g, 256, 0, s, L.n, L.dinv, y, L.wc);   // D^-1 y
    GBS_LAUNCH_CHECK();
    const ST* z = L.wc;
    for (int k = 0; k < ilu_sweeps; ++k) {   // forward: z = D^-1 y - Us z; transposed: t = t0 - L^T t
      csr_spmv<SPMV_RESID, VT, ST, ST, AT>(second, z, L.wc, pp[q], s);
      z = pp[q];
      q ^= 1;
    }
    return z;
  }

  // out = V(f) at level l; f and out are ST vectors of that level's size.
  // r = f - A_l x (A^T when TR)
  template <bool TR>
  void resid(Lev& L, const ST* x, const ST* f, ST* r, cudaStream_t s) {
    if (L.iso) {   // (S (x) I)^T = S^T (x) I
      if (TR) iso_spmv<SPMV_RESID, VT, ST, ST, AT>(B, L.AcT, L.As, false, x, f, r, s);
      else iso_spmv<SPMV_RESID, VT, ST, ST, AT>(B, L.Ac, L.As, L.a_sell, x, f, r, s);
      return;
    }
    const bool acsr = L.a_csr && !TR;   // A^T goes through the block form's transpose map
    if (L.a_bsell && !TR) bsell_spmv<SPMV_RESID, VT, ST, ST, AT>(B, L.Ab, x, f, r, s);
    else if (acsr && L.a_sell) sell_spmv<SPMV_RESID, VT, ST, ST, AT>(L.As, x, f, r, s);
    else if (acsr) csr_spmv<SPMV_RESID, VT, ST, ST, AT>(L.Ac, x, f, r, s);
    else spmv<TR, SPMV_RESID, VT, ST, ST, AT>(B, L.A, x, f, r, s);
  }

  // One relaxation sweep xout = xin + S (f - A_l xin) (S^T, A^T when TR).
  template <bool TR>
  void sweep(Lev& L, const ST* f, const ST* xin, ST* xout, cudaStream_t s) {
    const bool acsr = L.a_csr && !TR;
    if (L.ilu) {   // xout = xin + omega S (f - A xin)
      resid<TR>(L, xin, f, L.r, s);
      const ST* z = ilu_apply<TR>(L, L.r, s);
      ::gbs::launch_k(k_vaxpy<ST>, grid_for(L.n), 256, 0, s, L.n, xin, (ST)ilu_omega, z, xout);
      GBS_LAUNCH_CHECK();
    } else if (L.iso) {   // diag(m) (x) I is symmetric: the transposed sweep uses S^T only
      if (TR) iso_relax<VT, ST, AT>(B, L.AcT, L.As, false, L.M, f, xin, xout, s);
      else iso_relax<VT, ST, AT>(B, L.Ac, L.As, L.a_sell, L.M, f, xin, xout, s);
    } else if (L.a_bsell && !TR) {
      bsell_relax<VT, ST, AT>(B, L.Ab, L.M, f, xin, xout, s);
    } else if (acsr && L.a_sell) {
      sell_relax<VT, ST, AT>(B, L.As, L.M, f, xin, xout, s);
    } else if (acsr) {
      csr_relax<VT, ST, AT>(B, L.Ac, L.M, f, xin, xout, s);
    } else {
      relax<TR, VT, ST, AT>(B, L.A, L.M, f, xin, xout, s);
    }
  }

  // x = M f and r = f - A x (zero-guess pre-smoothing + residual, fused).
  void presmooth_resid(Lev& L, const ST* f, ST* x, ST* r, cudaStream_t s) {
    if (L.iso) {
      if (L.fused == 3) iso_presmooth_otf<VT, ST, AT>(B, L.As, L.M, f, x, r, s);
      else iso_presmooth<VT, ST, AT>(B, L.AMs, L.M, f, x, r, s);
      return;
    }
    if (L.fused == 2) {
      const unsigned g = grid_for((int64_t)L.AMb.nslices * 32);
      switch (B) {
        case 1: ::gbs::launch_k(k_bsell_presmooth<1, VT, ST, AT>, g, 256, 0, s, L.AMb, L.M, f, x, r); break;
        case 2: ::gbs::launch_k(k_bsell_presmooth<2, VT, ST, AT>, g, 256, 0, s, L.AMb, L.M, f, x, r); break;
        case 3: ::gbs::launch_k(k_bsell_presmooth<3, VT, ST, AT>, g, 256, 0, s, L.AMb, L.M, f, x, r); break;
        case 4: ::gbs::launch_k(k_bsell_presmooth<4, VT, ST, AT>, g, 256, 0, s, L.AMb, L.M, f, x, r); break;
      }
    } else {
      const unsigned g = grid_for((int64_t)(L.AMs.nslices / B) * 32);
      switch (B) {
        case 1: ::gbs::launch_k(k_sell_presmooth_direct<1, VT, ST, AT>, g, 256, 0, s, L.AMs, L.M, f, x, r); break;
        case 2: ::gbs::launch_k(k_sell_presmooth_direct<2, VT, ST, AT>, g, 256, 0, s, L.AMs, L.M, f, x, r); break;
        case 3: ::gbs::launch_k(k_sell_presmooth_direct<3, VT, ST, AT>, g, 256, 0, s, L.AMs, L.M, f, x, r); break;
        case 4: ::gbs::launch_k(k_sell_presmooth_direct<4, VT, ST, AT>, g, 256, 0, s, L.AMs, L.M, f, x, r); break;
      }
    }
    GBS_LAUNCH_CHECK();
  }

  // out = V(f) at level l; f and out are ST vectors of that level's size.
  // r64 / z64 (mixed forms, level 0 only): the V-cycle's FP64 input and
  // output.  The input is rounded into f (the caller's FP32 buffer) by the
  // first level-0 kernel, and the last level-0 sweep writes z64 in FP64,
  // where the level's kernels allow it; otherwise separate cast passes.
  template <bool TR>
  void cycle(size_t l, const ST* f, ST* out, cudaStream_t s, const double* r64 = nullptr,
             double* z64 = nullptr) {
    static const char* const kLevel[] = {"V-cycle level 0", "V-cycle level 1", "V-cycle level 2",
                                         "V-cycle level 3", "V-cycle level 4", "V-cycle level 5",
                                         "V-cycle level 6", "V-cycle level 7", "V-cycle level 8",
                                         "V-cycle level 9+"};
    NvtxRange range(kLevel[l < 9 ? l : 9]);
    if (r64 && (l + 1 == lev.size() || lev[l].ilu || (TR ? npost : npre) < 1)) {
      cast<double, ST>(lev[l].n, r64, const_cast<ST*>(f), s);   // no folding here
      r64 = nullptr;
    }
    if (l + 1 == lev.size()) {
      const ST* Ai = TR ? AinvT : Ainv;
      ::gbs::launch_k(k_gemv<ST, ST, AT>, grid_for((int64_t)nc * 32), 256, 0, s, nc, Ai, f, out);
      GBS_LAUNCH_CHECK();
      if (z64) cast<ST, double>(nc, out, z64, s);
      return;
    }
    Lev& L = lev[l];
    const int nb = L.A.nbr;
    const int pre = TR ? npost : npre;
    const int post = TR ? npre : npost;
    ST* x = L.x;
    ST* xt = L.xt;
    bool have_r = false;
    if (pre >= 1) {
      if (L.ilu) {
        const ST* z = ilu_apply<TR>(L, f, s);
        ::gbs::launch_k(k_vaxpy<ST>, grid_for(L.n), 256, 0, s, L.n, (const ST*)nullptr, (ST)ilu_omega, z, x);
        GBS_LAUNCH_CHECK();
      } else if (L.fused && !TR && pre == 1 && !(L.fused == 3 && r64)) {
        presmooth_resid(L, f, x, L.r, s);   // x = M f and r = f - A x in one pass
        have_r = true;
      } else if (r64) {
        cast_mapply<TR>(L, r64, const_cast<ST*>(f), x, s);   // f = (ST) r64 and x = M f
      } else if (L.iso) {
        iso_mapply<VT, ST, AT>(B, L.n, L.M, f, x, s);
      } else {
        mapply<TR, VT, ST, AT>(B, nb, L.M, f, x, s);
      }
      for (int it = 1; it < pre; ++it) {
        sweep<TR>(L, f, x, xt, s);
        std::swap(x, xt);
      }
    } else {
      GBS_CUDA(cudaMemsetAsync(x, 0, sizeof(ST) * L.n, s));
    }
    if (!have_r) resid<TR>(L, x, f, L.r, s);
    Lev& Cn = lev[l + 1];
    const ST* none = nullptr;
    if (L.iso) iso_spmv<SPMV_SET, VT, ST, ST, AT>(B, L.Rc, L.Rs, L.r_sell, L.r, none, Cn.f, s);
    else if (L.r_sell) sell_spmv<SPMV_SET, VT, ST, ST, AT>(L.Rs, L.r, none, Cn.f, s);
    else if (L.r_csr) csr_spmv<SPMV_SET, VT, ST, ST, AT>(L.Rc, L.r, none, Cn.f, s);
    else spmv<false, SPMV_SET, VT, ST, ST, AT>(B, L.R, L.r, none, Cn.f, s);
    cycle<TR>(l + 1, Cn.f, Cn.e, s);
    if (L.iso) iso_spmv<SPMV_ADD, VT, ST, ST, AT>(B, L.Pc, L.Ps, L.p_sell, Cn.e, none, x, s);
    else if (L.p_sell) sell_spmv<SPMV_ADD, VT, ST, ST, AT>(L.Ps, Cn.e, none, x, s);
    else if (L.p_csr) csr_spmv<SPMV_ADD, VT, ST, ST, AT>(L.Pc, Cn.e, none, x, s);
    else spmv<false, SPMV_ADD, VT, ST, ST, AT>(B, L.Pm, Cn.e, none, x, s);
    for (int it = 0; it < post; ++it) {
      const bool last = it + 1 == post;
      if (last && z64 && !TR && L.iso) {   // the last sweep writes the FP64 output
        iso_relax<VT, ST, AT, double>(B, L.Ac, L.As, L.a_sell, L.M, f, x, z64, s);
        return;
      }
      if (last && z64 && !TR && L.a_csr && L.a_sell && !L.ilu) {
        // the last sweep writes the FP64 output (no cast pass)
        sell_relax<VT, ST, AT, double>(B, L.As, L.M, f, x, z64, s);
        return;
      }
      ST* dst = last ? out : xt;
      sweep<TR>(L, f, x, dst, s);
      std::swap(x, xt);
    }
    if (post == 0) GBS_CUDA(cudaMemcpyAsync(out, x, sizeof(ST) * L.n, cudaMemcpyDeviceToDevice, s));
    if (z64) cast<ST, double>(L.n, out, z64, s);
  }

  template <bool TR>
  void cast_mapply(Lev& L, const double* r64, ST* fin, ST* x, cudaStream_t s) {
    if (L.iso) {
      iso_cast_mapply<VT, ST, AT>(B, L.n, L.M, r64, fin, x, s);
      return;
    }
    const int nb = L.A.nbr;
    switch (B) {
      case 1: ::gbs::launch_k(k_cast_mapply<1, TR, VT, ST, AT>, grid_for(row_threads<1>(nb)), 256, 0, s, nb, L.M, r64, fin, x); break;
      case 2: ::gbs::launch_k(k_cast_mapply<2, TR, VT, ST, AT>, grid_for(row_threads<2>(nb)), 256, 0, s, nb, L.M, r64, fin, x); break;
      case 3: ::gbs::launch_k(k_cast_mapply<3, TR, VT, ST, AT>, grid_for(row_threads<3>(nb)), 256, 0, s, nb, L.M, r64, fin, x); break;
      case 4: ::gbs::launch_k(k_cast_mapply<4, TR, VT, ST, AT>, grid_for(row_threads<4>(nb)), 256, 0, s, nb, L.M, r64, fin, x); break;
    }
    GBS_LAUNCH_CHECK();
  }

  // One level operation as the V-cycle runs it (measurement and tests):
  // op 0: y = f - A_l x; op 1: one relaxation sweep y = x + S (f - A_l x).
  void level_op(size_t l, int op, const ST* x, const ST* f, ST* y, cudaStream_t s) {
    if (l + 1 >= lev.size()) throw SetupError{"level_op: the coarsest level has no smoother"};
    if (op == 0) resid<false>(lev[l], x, f, y, s);
    else if (op == 1) sweep<false>(lev[l], f, x, y, s);
    else throw SetupError{"level_op: op must be 0 (residual) or 1 (relaxation sweep)"};
  }

  void vcycle(const ST* f, ST* out, bool tr, cudaStream_t s) {
    if (tr) cycle<true>(0, f, out, s);
    else cycle<false>(0, f, out, s);
  }

  double bytes_per_cycle() const {
    double b = 0;
    const double sv = sizeof(VT), sx = sizeof(ST);
    for (size_t l = 0; l + 1 < lev.size(); ++l) {
      const Lev& L = lev[l];
      const double nb = (double)L.A.nbr;
      const double nc = (double)(lev[l + 1].n / B);
      // slices: values, columns where a kernel loads them (staged kernels
      // stage every column; direct ones skip uniform slices), offsets
      auto sliced = [&](int64_t slots, int64_t xsl, bool dir, int64_t nsl) {
        return slots * sv + 4.0 * (dir ? xsl : slots) + 4 * (nsl + 1.0);
      };
      // scalar CSR rows: one per scalar row, or one per node (iso levels)
      const double rows_f = L.iso ? nb : (double)L.n, rows_c = L.iso ? nc : nc * B;
      const double Abytes = L.a_bsell ? L.slots_Ab * (B * B * sv + 4) + 4.0 * L.Ab.nslices * (32 / B + 1)
                            : L.a_sell ? sliced(L.slots_A, L.xsl_A, L.dir_A, L.sl_A)
                            : L.a_csr ? L.nnz_A * (sv + 4) + 4 * (rows_f + 1.0)
                                      : L.nnzb_A * (B * B * sv + 4) + 4 * (nb + 1);
      const double Pbytes = L.p_sell ? sliced(L.slots_P, L.xsl_P, L.dir_P, L.sl_P)
                            : L.p_csr ? L.nnz_P * (sv + 4) + 4 * (rows_f + 1.0)
                                      : L.nnzb_P * (B * B * sv + 4) + 4 * (nb + 1);
      const double Rbytes = L.r_sell ? sliced(L.slots_R, L.xsl_R, L.dir_R, L.sl_R)
                            : L.r_csr ? L.nnz_R * (sv + 4) + 4 * (rows_c + 1)
                                      : L.nnzb_R * (B * B * sv + 4) + 4 * (nc + 1);
      const double Mbytes = L.iso ? nb * sv : nb * B * B * sv;
      b += Abytes + 3 * L.n * sx;                               // resid (A, x, f, r)
      b += Rbytes + L.n * sx + lev[l + 1].n * sx;               // restrict (R, r, fc)
      b += Pbytes + lev[l + 1].n * sx + 2 * L.n * sx;           // prolong (P, ec, x rw)
      if (L.ilu) {
        const double m = ilu_sweeps;
        const double ilu = m * (L.nnz_Li * (sv + 4) + 4 * (L.n + 1.0) + 3 * L.n * sx) +
                           (L.n * sv + 2 * L.n * sx) +
                           m * (L.nnz_Ui * (sv + 4) + 4 * (L.n + 1.0) + 3 * L.n * sx);
        b += ilu + 2 * L.n * sx;                                 // zero-guess step
        b += Abytes + 3 * L.n * sx + ilu + 3 * L.n * sx;          // resid + S + axpy
      } else {
        b += Mbytes + 2 * L.n * sx;                              // mapply (M, f, x)
        b += Abytes + Mbytes + 3 * L.n * sx;                     // relax (A, M, f, x, out)
      }
      if (L.fused) {
        // the fused pass (A M -- or A with M gathered beside f -- f
        // gathered, M, x and r written) replaces mapply and the residual
        const double AMbytes = L.fused == 2
            ? L.slots_AM * (B * B * sv + 4) + 4.0 * L.AMb.nslices * (32 / B + 1)
            : L.fused == 3 ? Abytes
            : sliced(L.slots_AM, L.xsl_AM, true, L.sl_AM);
        b -= (Mbytes + 2 * L.n * sx) + (Abytes + 3 * L.n * sx);
        b += AMbytes + Mbytes + 3 * L.n * sx;
      }
    }
    b += (double)nc * nc * sx + 2.0 * nc * sx;
    return b;
  }
};

template <int P>
struct AmgPrecond final : DevPrecond {
  using ST = typename FormT<P>::ST;
  DevAmg<P> amg;
  ST *fin = nullptr, *fout = nullptr;  // mixed forms: FP32 staging of r and z
  Arena ar;
  void init(const HAmg& H, const PrecondOptions& o, cudaStream_t s) {
    amg.build(H, o, s);
    if constexpr (!std::is_same<ST, double>::value) {
      fin = ar.alloc<ST>(amg.n0());
      fout = ar.alloc<ST>(amg.n0());
    }
  }
  void apply(const double* r, double* z, bool tr, cudaStream_t s) override {
    NvtxRange range("AMG preconditioner");
    if constexpr (std::is_same<ST, double>::value) {
      amg.vcycle(r, z, tr, s);
    } else {
      // the precision boundary is folded into the first and the last level-0
      // kernels where they allow it (DevAmg::cycle)
      if (tr) amg.template cycle<true>(0, fin, fout, s, r, z);
      else amg.template cycle<false>(0, fin, fout, s, r, z);
    }
  }
  int64_t bytes() const override { return amg.ar.bytes + ar.bytes; }
  void level_op(int which, int l, int op, const void* x, const void* f, void* y,
                cudaStream_t s) override {
    if (which != 0) throw SetupError{"level_op: the monolithic AMG is hierarchy 0"};
    amg.level_op((size_t)l, op, static_cast<const ST*>(x), static_cast<const ST*>(f),
                 static_cast<ST*>(y), s);
  }
  int vector_bytes() const override { return (int)sizeof(ST); }
  int level_layout(int, int l) const override { return amg.layout((size_t)l); }
  int nlevels(int which) const override { return which == 0 ? (int)amg.lev.size() : 0; }
  int64_t level_rows(int, int l) const override { return amg.lev[l].n / amg.B; }
  int64_t level_nnzb(int, int l) const override { return amg.lev[l].nnzb_A; }
  double bytes_per_apply() const override {
    double b = amg.bytes_per_cycle();
    if constexpr (!std::is_same<ST, double>::value) {
      // FP64 -> ST and back; a folded side moves 4 bytes an entry more than
      // the level-0 kernel it joins instead of a separate cast pass
      const double n = (double)amg.n0(), sx = sizeof(ST);
      const auto& L = amg.lev[0];
      const bool deep = amg.lev.size() > 1 && !L.ilu;
      b += deep && amg.npre >= 1 ? n * (8 - sx) : n * (8 + sx);
      b += deep && (L.iso || (L.a_csr && L.a_sell)) ? n * (8 - sx) : n * (8 + sx);
    }
    return b;
  }
};

// ------------------------------------------------------------- Schur kernels
// fu[i*NV + c] = r[i*(NV+1) + c]
// One thread a node: its NV + 1 interleaved FP64 entries load as one run.
template <int NV, class ST>
__global__ void k_gather_u(int nn, const double* __restrict__ r, ST* __restrict__ fu) {
  GBS_GRID_DEP();
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nn;
       i += (int64_t)gridDim.x * blockDim.x) {
    double v[NV + 1];
    load_run<NV + 1, double, double, true>(r + i * (NV + 1), v);
#pragma unroll
    for (int c = 0; c < NV; ++c) fu[i * NV + c] = (ST)v[c];
  }
}
// The couplings as scalar CSR of their nonzeros (on the FD stencil one
// velocity component per neighbour block: 6 entries a pressure row of D,
// 2 a velocity row of G, against 21 and 7 stored values on K's block
// pattern).  Entries keep the block order, so the sums equal the block
// kernels' above term for term.
// q_i = r_p,i - sum_k C_k u_{col k}   (C = D, or G^T for the transposed step)
template <int NV, class VT, class ST>
__global__ void k_schur_q_csr(DevCsr<VT> C, const double* __restrict__ r, const ST* __restrict__ u,
                              ST* __restrict__ q) {
  GBS_GRID_DEP();
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < C.n; i += gridDim.x * blockDim.x) {
    ST acc = ST(0);
    for (int k = C.rp[i]; k < C.rp[i + 1]; ++k) acc += cvt<ST>(C.val[k]) * u[C.col[k]];
    q[i] = (ST)r[(size_t)i * (NV + 1) + NV] - acc;
  }
}
// fu2_t = fu_t - sum_k C_k p_{col k}   (C = G, or D^T for the transposed step)
template <class VT, class ST>
__global__ void k_schur_u_csr(DevCsr<VT> C, const ST* __restrict__ fu, const ST* __restrict__ p,
                              ST* __restrict__ fu2) {
  GBS_GRID_DEP();
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < C.n; t += gridDim.x * blockDim.x) {
    ST acc = fu[t];
    for (int k = C.rp[t]; k < C.rp[t + 1]; ++k) acc -= cvt<ST>(C.val[k]) * p[C.col[k]];
    fu2[t] = acc;
  }
}
// q_i = r_p,i (pressure part of an interleaved vector)
template <int NV, class ST>
__global__ void k_gather_p(int nn, const double* __restrict__ r, ST* __restrict__ q) {
  GBS_GRID_DEP();
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nn;
       i += (int64_t)gridDim.x * blockDim.x)
    q[i] = (ST)r[i * (NV + 1) + NV];
}
// p_i = m_i q_i (one application of a scalar pressure smoother)
template <class VT, class ST>
__global__ void k_diag_apply(int nn, const VT* __restrict__ m, const ST* __restrict__ q,
                             ST* __restrict__ p) {
  GBS_GRID_DEP();
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nn;
       i += (int64_t)gridDim.x * blockDim.x)
    p[i] = cvt<ST>(m[i]) * q[i];
}
template <int NV, class ST>
__global__ void k_scatter_z(int nn, const ST* __restrict__ u, const ST* __restrict__ p,
                            double* __restrict__ z) {
  GBS_GRID_DEP();
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nn;
       i += (int64_t)gridDim.x * blockDim.x) {
    double v[NV + 1];
#pragma unroll
    for (int c = 0; c < NV; ++c) v[c] = (double)u[i * NV + c];
    v[NV] = (double)p[i];
    if constexpr ((NV + 1) % 2 == 0) {   // 16-byte stores of the node's run
#pragma unroll
      for (int c = 0; c < NV + 1; c += 2)
        *reinterpret_cast<double2*>(z + i * (NV + 1) + c) = make_double2(v[c], v[c + 1]);
    } else {
#pragma unroll
      for (int c = 0; c < NV + 1; ++c) z[i * (NV + 1) + c] = v[c];
    }
  }
}

template <int P>
struct SchurPrecond final : DevPrecond {
  using VT = typename FormT<P>::VT;
  using ST = typename FormT<P>::ST;
  using AT = ST;
  DevAmg<P> A, S;
  // couplings as scalar CSR of their nonzeros: D (pressure rows), G
  // (velocity rows) and, for the transposed application, G^T and D^T
  DevCsr<VT> Dc, Gc, GcT, DcT;
  int64_t nnz_D = 0, nnz_G = 0;
  int nv = 3, nn = 0;
  int order = 0;                 // 0 full, 1 lower
  const VT* MS = nullptr;        // pressure smoother when the pressure solve is one sweep
  ST *fu = nullptr, *fu2 = nullptr, *u1 = nullptr, *u = nullptr, *q = nullptr, *p = nullptr;
  Arena ar;
  int64_t nnzb = 0;

  void init(const HSchur& Hs, const HAmg& HA, const HAmg& HS, const PrecondOptions& o,
            cudaStream_t s) {
    nv = Hs.nvel;
    nn = Hs.C.nbr;
    nnzb = Hs.C.nnzb();
    order = o.schur_order;
    A.build(HA, o, s);
    std::vector<std::vector<VT>> keep;
    if (o.schur_p_smoother) {
      keep.push_back(cast_vec<VT>(Hs.MS));
      MS = ar.upload(keep.back().data(), keep.back().size(), s);
    } else {
      S.build(HS, o, s);
    }
    const HCsr Dh = to_scalar_csr(Hs.D), Gh = to_scalar_csr(Hs.G);
    nnz_D = (int64_t)Dh.col.size();
    nnz_G = (int64_t)Gh.col.size();
    Dc = upload_csr<VT>(ar, Dh, s, keep);
    Gc = upload_csr<VT>(ar, Gh, s, keep);
    if (o.tmaps) {
      GcT = upload_csr<VT>(ar, transpose(Gh), s, keep);
      DcT = upload_csr<VT>(ar, transpose(Dh), s, keep);
    }
    fu = ar.alloc<ST>((size_t)nn * nv);
    fu2 = ar.alloc<ST>((size_t)nn * nv);
    u1 = ar.alloc<ST>((size_t)nn * nv);
    u = ar.alloc<ST>((size_t)nn * nv);
    q = ar.alloc<ST>(nn);
    p = ar.alloc<ST>(nn);
    GBS_CUDA(cudaStreamSynchronize(s));
  }

  void pressure(const ST* qin, ST* pout, bool tr, cudaStream_t s) {
    if (MS) {
      ::gbs::launch_k(k_diag_apply<VT, ST>, grid_for(nn), 256, 0, s, nn, MS, qin, pout);
      GBS_LAUNCH_CHECK();
    } else {
      S.vcycle(qin, pout, tr, s);
    }
  }

  // Forward "full": u1 = V_A(r_u); q = r_p - D u1; p = V_S(q); u = V_A(r_u - G p).
  // Forward "lower": the same without the second velocity solve (u = u1).
  // Transposed "full": the same steps with A^T, S^T and G^T, D^T swapped.
  // Transposed "lower" (upper form on K^T): p = V_S^T(r_p); u = V_A^T(r_u - D^T p).
  template <int NV>
  void run(const double* r, double* z, bool tr, cudaStream_t s) {
    const unsigned g = grid_for((int64_t)nn * NV);
    const unsigned gn = grid_for(nn);
    ::gbs::launch_k(k_gather_u<NV, ST>, gn, 256, 0, s, nn, r, fu);
    GBS_LAUNCH_CHECK();
    const ST* uout = u;
    if (order == 1 && tr) {
      ::gbs::launch_k(k_gather_p<NV, ST>, gn, 256, 0, s, nn, r, q);
      GBS_LAUNCH_CHECK();
      pressure(q, p, true, s);
      ::gbs::launch_k(k_schur_u_csr<VT, ST>, g, 256, 0, s, DcT, fu, p, fu2);
      GBS_LAUNCH_CHECK();
      A.vcycle(fu2, u, true, s);
    } else {
      A.vcycle(fu, u1, tr, s);
      // forward: q = r_p - D u1; transposed: q = r_p - G^T u1
      ::gbs::launch_k(k_schur_q_csr<NV, VT, ST>, gn, 256, 0, s, tr ? GcT : Dc, r, u1, q);
      GBS_LAUNCH_CHECK();
      pressure(q, p, tr, s);
      if (order == 1) {
        uout = u1;
      } else {
        // forward: fu2 = fu - G p; transposed: fu2 = fu - D^T p
        ::gbs::launch_k(k_schur_u_csr<VT, ST>, g, 256, 0, s, tr ? DcT : Gc, fu, p, fu2);
        GBS_LAUNCH_CHECK();
        A.vcycle(fu2, u, tr, s);
      }
    }
    ::gbs::launch_k(k_scatter_z<NV, ST>, gn, 256, 0, s, nn, uout, p, z);
    GBS_LAUNCH_CHECK();
  }

  void apply(const double* r, double* z, bool tr, cudaStream_t s) override {
    NvtxRange range("Schur preconditioner");
    switch (nv) {
      case 1: run<1>(r, z, tr, s); break;
      case 2: run<2>(r, z, tr, s); break;
      case 3: run<3>(r, z, tr, s); break;
    }
  }
  int64_t bytes() const override { return A.ar.bytes + S.ar.bytes + ar.bytes; }
  void level_op(int which, int l, int op, const void* x, const void* f, void* y,
                cudaStream_t s) override {
    if (which == 1 && MS) throw SetupError{"level_op: the pressure solve is one sweep (no AMG)"};
    DevAmg<P>& H = which == 0 ? A : S;
    H.level_op((size_t)l, op, static_cast<const ST*>(x), static_cast<const ST*>(f),
               static_cast<ST*>(y), s);
  }
  int vector_bytes() const override { return (int)sizeof(ST); }
  int level_layout(int which, int l) const override {
    return which == 0 ? A.layout((size_t)l) : S.layout((size_t)l);
  }
  int nlevels(int which) const override {
    return which == 0 ? (int)A.lev.size() : (int)S.lev.size();
  }
  int64_t level_rows(int which, int l) const override {
    return which == 0 ? A.lev[l].n / A.B : S.lev[l].n;
  }
  int64_t level_nnzb(int which, int l) const override {
    return which == 0 ? A.lev[l].nnzb_A : S.lev[l].nnzb_A;
  }
  double bytes_per_apply() const override {
    const double sv = sizeof(VT), sx = sizeof(ST);
    double b = (order == 1 ? 1 : 2) * A.bytes_per_cycle();
    b += MS ? nn * (sv + 2 * sx) : S.bytes_per_cycle();
    // gather, two couplings (scalar CSR of their nonzeros), scatter
    b += nn * nv * (8 + sx);
    b += nnz_D * (sv + 4) + 4.0 * (nn + 1) + nn * nv * sx + nn * (8 + sx);
    b += nnz_G * (sv + 4) + 4.0 * (nn * nv + 1) + nn * sx + 2.0 * nn * nv * sx;
    b += nn * (nv + 1) * 8 + nn * (nv + 1) * sx;
    return b;
  }
};

}  // namespace gbs
