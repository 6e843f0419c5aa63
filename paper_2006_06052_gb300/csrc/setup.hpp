// Host-side hierarchy construction (not on the solve path).
//
// The paper's AMGCL builds the multigrid hierarchy on builtin host
// structures and then moves it to the backend (Section 2).  This file
// declares that host step: smoothed-aggregation coarsening, SPAI0 /
// damped-Jacobi blocks, the dense coarse inverse and the Schur split
// (Eq. SchurPC / Eq. SchurApprox).
#pragma once

#include <cstdint>
#include <string>
#include <vector>

namespace gbs {

// Block-CSR on the host, FP64 values, (br x bc) blocks, row-major blocks.
struct HBsr {
  int nbr = 0, nbc = 0, br = 1, bc = 1;
  std::vector<int32_t> ptr, col;
  std::vector<double> val;
  int64_t nnzb() const { return (int64_t)col.size(); }
  int bsz() const { return br * bc; }
};

struct AmgSetupParams {
  double eps_strong = 0.08;
  int coarse_enough = 1000;
  int max_levels = 10;
  int relax = 0;           // 0 SPAI0, 1 damped Jacobi, 2 ILUT
  double jacobi_omega = 0.72;
  bool smooth_P = true;
  int power_iters = 20;
  double ilut_p = 2.0;     // ILUT fill factor
  double ilut_tau = 1e-2;  // ILUT drop tolerance
};

// Scalar CSR (declared here for the ILUT factors; see to_scalar_csr).
struct HCsr {
  int n = 0, ncols = 0;
  std::vector<int32_t> ptr, col;
  std::vector<double> val;
};

// ILUT factors of a scalar matrix: A ~ (I + L)(D + U), L strictly lower,
// U strictly upper, D = diag(d).
struct HIlu {
  HCsr L, U;
  std::vector<double> d;
};

struct HLevel {
  HBsr A, P, R;
  std::vector<double> M;   // n_brows * B * B smoother blocks (SPAI0 / Jacobi)
  HIlu ilu;                // ILUT relaxation factors (relax = 2)
  std::vector<int32_t> agg;
  double omega = 0.0;
};

struct HAmg {
  int B = 1;
  std::vector<HLevel> levels;   // all but the coarsest
  HBsr Ac;                      // coarsest operator
  std::vector<double> Ainv;     // dense inverse of Ac, row-major
};

struct SetupError {
  std::string msg;
};

// Structural validation of a caller matrix (throws SetupError).
void validate(const HBsr& A, bool square);

// Full setup of one AMG hierarchy (throws SetupError).
HAmg build_amg(const HBsr& A, const AmgSetupParams& prm);

// Pieces exposed for tests / export.
std::vector<int32_t> aggregate(const HBsr& A, double eps, int* n_agg);
std::vector<double> spai0(const HBsr& A);
std::vector<double> jacobi(const HBsr& A, double omega);

// A M for a block-diagonal M (n_brows * B * B blocks): block (i, j) of the
// result is A_ij M_j, on A's pattern.  With x = M f, the residual f - A x of
// a zero-guess smoothing step is f - (A M) f, one product with f.
HBsr scale_columns(const HBsr& A, const std::vector<double>& M);

// Scalar CSR of the nonzero entries of a block matrix (columns sorted per
// row); fill = nonzeros / stored block values.
HCsr to_scalar_csr(const HBsr& A);

// Blocks that are scalar multiples of the identity.  is_iso: A has square
// B x B blocks (B >= 2), every stored block has zero off-diagonal entries
// and B bitwise-equal diagonal entries, so A = S (x) I_B.  iso_scalar: S as
// scalar CSR of its nonzeros (one entry per nonzero block, columns sorted).
// is_iso_blocks / iso_diag: the same test and the per-node value for a
// block-diagonal smoother (n * B * B values).
bool is_iso(const HBsr& A);
bool is_iso_blocks(const std::vector<double>& M, int B);
HCsr iso_scalar(const HBsr& A);
std::vector<double> iso_diag(const std::vector<double>& M, int B);

// Saad's dual-threshold ILUT (Section 4's velocity smoother), row by row
// in natural order: eliminate the row's lower entries in increasing
// column order (fill included), dropping an entry below tau * ||a_i||_2
// (tested before its division by the pivot, so that the test is
// scale-free) with its update; drop upper entries below the same bound;
// keep the floor(p * count) largest of the lower and of the upper
// entries, count being the row's own lower / upper nonzeros (ties to the
// smaller column); a zero pivot becomes tau * ||a_i||_2 (1 if that is
// zero).
HIlu ilut(const HCsr& A, double p, double tau);
// Transpose of a scalar CSR matrix (columns sorted per row).
HCsr transpose(const HCsr& A);
double block_fill(const HBsr& A);

// Sliced scalar CSR: the rows of component c (c < B) of 32 consecutive
// nodes form slice q = 32-node group * B + c, stored column-major -- entry
// k of the row of lane i at (off[q] + k) * 32 + i -- and padded to the
// slice's longest row with column -1 (value 0).  Rows of one component have
// equal lengths away from boundaries, so a warp walks its slice with every
// lane busy and each load instruction reads one contiguous run.
//
// A slice whose rows share their column offsets (col - row) -- a stencil
// level, where a slice's rows differ only by missing entries at the
// boundary -- is "uniform": the union of its rows' offsets is at most an
// eighth wider than its longest row, entry k of every lane sits at column
// row + uoff[k], and bit lane of umask[k] says whether that lane has it.
// The kernels then need no column loads for it: the gather address comes
// from the row index, not from memory.
struct HSell {
  int n = 0, B = 1, nslices = 0;
  std::vector<int32_t> off;   // nslices + 1, in columns of 32 entries
  std::vector<int32_t> col;   // off[nslices] * 32
  std::vector<double> val;
  std::vector<int64_t> src;   // entry -> index into the CSR arrays, -1 for padding
  std::vector<int32_t> cinfo; // per slice: 0 explicit, -1 - (first uoff index) uniform
  std::vector<int32_t> uoff;  // uniform slices: column offset of each slice column
  std::vector<uint32_t> umask;
  // Sorted form (irregular operators): the node of lane i of group g is
  // node[g * 32 + i] (-1: none) instead of g * 32 + i -- nodes sorted by
  // their rows' total length within windows of 1024 nodes, so that a
  // slice's rows have nearly equal lengths.  Empty: natural order.
  std::vector<int32_t> node;
};
// Stored entries / nonzeros - 1 of the sliced form (B must divide C.n),
// in natural or sorted node order.
double sell_padding(const HCsr& C, int B, bool sorted = false);
HSell to_sell(const HCsr& C, int B, bool sorted = false);

// Block-row slices of a square block matrix (the FP64 block levels): the
// block rows are sorted by length (longest first, stable) within windows
// of `window` slices, and each run of R = 32 / B consecutive sorted rows
// forms a slice that one warp owns with one lane per scalar row -- no lane
// shares a row, so no cross-lane sums, and the rows of a slice have
// nearly equal lengths, so few lanes idle.  Each slice is padded to its
// longest row.  Entry k of slot i of slice q is block e = (off[q] + k) * R
// + i: column col[e], values val[e * B * B ...] row-major, so a warp's
// loads of entry k read R consecutive blocks.  Padding entries repeat the
// slot's own block row as column with zero values; empty slots (the last
// slice) have perm -1.
struct HBSell {
  int nbr = 0, B = 1, R = 8, nslices = 0;
  std::vector<int32_t> perm;   // nslices * R: block row of each slot, -1 if none
  std::vector<int32_t> off;    // nslices + 1, in entries of R blocks
  std::vector<int32_t> col;    // off[nslices] * R
  std::vector<double> val;     // off[nslices] * R * B * B
};
HBSell to_bsell(const HBsr& A, int window);
// Stored blocks / stored blocks of A - 1 of that layout.
double bsell_padding(const HBsr& A, int window);

// Schur split of node blocks (nvel+1)^2 into A (nvel^2), G (nvel x 1),
// D (1 x nvel), C (1x1) on K's block pattern, and S_hat of Eq. SchurApprox.
struct HSchur {
  HBsr A, G, D, C, S;
  int nvel = 3;
  std::vector<double> MS;   // pressure smoother on S (when the pressure solve is one sweep)
};
HSchur schur_split(const HBsr& K, int nvel);

// Transpose map of a structurally symmetric pattern: tmap[k] = index of
// block (j, i) for block k = (i, j).  Returns false if not symmetric.
bool transpose_map(const HBsr& A, std::vector<int32_t>& tmap);

}  // namespace gbs
