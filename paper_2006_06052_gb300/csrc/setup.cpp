// Host-side hierarchy construction: smoothed aggregation, SPAI0 /
// damped Jacobi, Galerkin products, dense coarse inverse, Schur split.
//
// Algorithm (the paper composes AMG from smoothed-aggregation coarsening
// and the SPAI0 smoother, Section 2.1, Listing "composition", with the
// strong-coupling threshold of Listing "params"; it leaves the inner
// steps to the AMG literature, so these are the readings used):
//  - strength: ||A_ij||_F^2 > (eps^2 ||A_ii||_F) ||A_jj||_F, eps halved per
//    level, squares summed over the block in row-major order;
//  - greedy aggregation: roots in ascending order when all strong
//    neighbours are free; leftovers join the pass-1 aggregate of their
//    strongest neighbour (ties to the smaller aggregate id);
//  - P = (I - omega D^-1 A) P_tent, omega = 4 / (3 rho(D^-1 A)), rho by
//    power iteration from x_i = frac(0.6180339887498949 i) - 0.5;
//  - R = P^T, A_c = R A P;
//  - SPAI0 (Broker & Grote): M_i = A_ii^T (sum_j A_ij A_ij^T)^-1;
//    damped Jacobi: M_i = omega A_ii^-1;
//  - coarsest level: dense LU with partial pivoting, explicit inverse.
// This translation unit must be compiled with -ffp-contract=off so the
// strength test rounds like plain IEEE multiply and add.
#include "setup.hpp"

#include <algorithm>
#include <functional>
#include <cmath>
#include <cstring>

namespace gbs {

namespace {

[[noreturn]] void fail(const std::string& m) { throw SetupError{m}; }

// C = A * B for B x B blocks (row-major), accumulated into C.
inline void blk_mul_add(int B, const double* a, const double* b, double* c) {
  for (int i = 0; i < B; ++i)
    for (int k = 0; k < B; ++k) {
      double aik = a[i * B + k];
      for (int j = 0; j < B; ++j) c[i * B + j] += aik * b[k * B + j];
    }
}

// Gauss-Jordan inverse with partial pivoting; false if singular.
bool blk_inv(int B, const double* a, double* out) {
  double m[16 * 2];
  const int W = 2 * B;
  for (int i = 0; i < B; ++i)
    for (int j = 0; j < W; ++j) m[i * W + j] = j < B ? a[i * B + j] : (j - B == i ? 1.0 : 0.0);
  for (int c = 0; c < B; ++c) {
    int p = c;
    for (int r = c + 1; r < B; ++r)
      if (std::fabs(m[r * W + c]) > std::fabs(m[p * W + c])) p = r;
    if (m[p * W + c] == 0.0) return false;
    if (p != c)
      for (int j = 0; j < W; ++j) std::swap(m[p * W + j], m[c * W + j]);
    double d = m[c * W + c];
    for (int j = 0; j < W; ++j) m[c * W + j] /= d;
    for (int r = 0; r < B; ++r) {
      if (r == c) continue;
      double f = m[r * W + c];
      if (f == 0.0) continue;
      for (int j = 0; j < W; ++j) m[r * W + j] -= f * m[c * W + j];
    }
  }
  for (int i = 0; i < B; ++i)
    for (int j = 0; j < B; ++j) out[i * B + j] = m[i * W + B + j];
  return true;
}

int find_col(const HBsr& A, int row, int col) {
  auto b = A.col.begin() + A.ptr[row];
  auto e = A.col.begin() + A.ptr[row + 1];
  auto it = std::lower_bound(b, e, col);
  if (it != e && *it == col) return (int)(it - A.col.begin());
  return -1;
}

std::vector<int> diag_pos(const HBsr& A) {
  std::vector<int> d(A.nbr);
  for (int i = 0; i < A.nbr; ++i) {
    d[i] = find_col(A, i, i);
    if (d[i] < 0) fail("block row " + std::to_string(i) + " has no stored diagonal block");
  }
  return d;
}

std::vector<double> block_fro2(const HBsr& A) {
  const int bs = A.bsz();
  std::vector<double> s(A.nnzb());
  for (int64_t k = 0; k < A.nnzb(); ++k) {
    double acc = 0.0;
    const double* v = &A.val[k * bs];
    for (int e = 0; e < bs; ++e) acc = acc + v[e] * v[e];
    s[k] = acc;
  }
  return s;
}

std::vector<double> block_diag_inv(const HBsr& A) {
  const int B = A.br, bs = B * B;
  auto d = diag_pos(A);
  std::vector<double> inv((size_t)A.nbr * bs);
  for (int i = 0; i < A.nbr; ++i)
    if (!blk_inv(B, &A.val[(size_t)d[i] * bs], &inv[(size_t)i * bs]))
      fail("singular diagonal block at row " + std::to_string(i));
  return inv;
}

void spmv(const HBsr& A, const std::vector<double>& x, std::vector<double>& y) {
  const int br = A.br, bc = A.bc, bs = br * bc;
  y.assign((size_t)A.nbr * br, 0.0);
  for (int i = 0; i < A.nbr; ++i)
    for (int a = 0; a < br; ++a) {
      double acc = 0.0;
      for (int k = A.ptr[i]; k < A.ptr[i + 1]; ++k) {
        const double* v = &A.val[(size_t)k * bs + a * bc];
        const double* xv = &x[(size_t)A.col[k] * bc];
        for (int c = 0; c < bc; ++c) acc += v[c] * xv[c];
      }
      y[(size_t)i * br + a] = acc;
    }
}

double norm2(const std::vector<double>& v) {
  double s = 0.0;
  for (double e : v) s += e * e;
  return std::sqrt(s);
}

double spectral_radius(const HBsr& A, int iters) {
  const size_t n = (size_t)A.nbr * A.br;
  std::vector<double> x(n), y;
  for (size_t i = 0; i < n; ++i) x[i] = std::fmod((double)i * 0.6180339887498949, 1.0) - 0.5;
  double nx = norm2(x);
  for (auto& e : x) e = e / nx;
  double rho = 0.0;
  for (int it = 0; it < iters; ++it) {
    spmv(A, x, y);
    rho = norm2(y);
    if (rho == 0.0) break;
    for (size_t i = 0; i < n; ++i) x[i] = y[i] / rho;
  }
  return rho;
}

HBsr transpose(const HBsr& A) {
  HBsr T;
  T.nbr = A.nbc;
  T.nbc = A.nbr;
  T.br = A.bc;
  T.bc = A.br;
  const int bs = A.bsz();
  T.ptr.assign(T.nbr + 1, 0);
  for (auto c : A.col) T.ptr[c + 1]++;
  for (int i = 0; i < T.nbr; ++i) T.ptr[i + 1] += T.ptr[i];
  T.col.resize(A.col.size());
  T.val.resize(A.val.size());
  std::vector<int32_t> pos(T.ptr.begin(), T.ptr.end() - 1);
  for (int i = 0; i < A.nbr; ++i)
    for (int k = A.ptr[i]; k < A.ptr[i + 1]; ++k) {
      int p = pos[A.col[k]]++;
      T.col[p] = i;
      for (int a = 0; a < A.br; ++a)
        for (int c = 0; c < A.bc; ++c)
          T.val[(size_t)p * bs + c * A.br + a] = A.val[(size_t)k * bs + a * A.bc + c];
    }
  return T;
}

// C = A * B (square blocks of size Bk), Gustavson row by row.
HBsr spgemm(const HBsr& A, const HBsr& Bm) {
  const int B = A.br, bs = B * B;
  HBsr C;
  C.nbr = A.nbr;
  C.nbc = Bm.nbc;
  C.br = C.bc = B;
  C.ptr.assign(C.nbr + 1, 0);
  std::vector<int> mark(C.nbc, -1);
  std::vector<int> cols;
  std::vector<double> acc;
  for (int i = 0; i < A.nbr; ++i) {
    cols.clear();
    acc.clear();
    for (int k = A.ptr[i]; k < A.ptr[i + 1]; ++k) {
      int j = A.col[k];
      for (int kk = Bm.ptr[j]; kk < Bm.ptr[j + 1]; ++kk) {
        int c = Bm.col[kk];
        if (mark[c] < 0) {
          mark[c] = (int)cols.size();
          cols.push_back(c);
          acc.resize(acc.size() + bs, 0.0);
        }
        blk_mul_add(B, &A.val[(size_t)k * bs], &Bm.val[(size_t)kk * bs], &acc[(size_t)mark[c] * bs]);
      }
    }
    std::vector<int> order(cols.size());
    for (size_t t = 0; t < order.size(); ++t) order[t] = (int)t;
    std::sort(order.begin(), order.end(), [&](int a, int b) { return cols[a] < cols[b]; });
    for (int t : order) {
      C.col.push_back(cols[t]);
      C.val.insert(C.val.end(), acc.begin() + (size_t)t * bs, acc.begin() + (size_t)(t + 1) * bs);
    }
    for (int c : cols) mark[c] = -1;
    C.ptr[i + 1] = (int32_t)C.col.size();
  }
  return C;
}

std::vector<double> dense_inverse(const HBsr& A) {
  const int B = A.br;
  const int n = A.nbr * B;
  std::vector<double> a((size_t)n * n, 0.0);
  for (int i = 0; i < A.nbr; ++i)
    for (int k = A.ptr[i]; k < A.ptr[i + 1]; ++k)
      for (int r = 0; r < B; ++r)
        for (int c = 0; c < B; ++c)
          a[(size_t)(i * B + r) * n + A.col[k] * B + c] = A.val[(size_t)k * B * B + r * B + c];
  // LU with partial pivoting, in place
  std::vector<int> piv(n);
  for (int c = 0; c < n; ++c) {
    int p = c;
    for (int r = c + 1; r < n; ++r)
      if (std::fabs(a[(size_t)r * n + c]) > std::fabs(a[(size_t)p * n + c])) p = r;
    if (a[(size_t)p * n + c] == 0.0) fail("singular coarsest-level matrix");
    piv[c] = p;
    if (p != c)
      for (int j = 0; j < n; ++j) std::swap(a[(size_t)p * n + j], a[(size_t)c * n + j]);
    double d = a[(size_t)c * n + c];
    for (int r = c + 1; r < n; ++r) {
      double f = a[(size_t)r * n + c] / d;
      a[(size_t)r * n + c] = f;
      if (f == 0.0) continue;
      double* rr = &a[(size_t)r * n];
      const double* cr = &a[(size_t)c * n];
      for (int j = c + 1; j < n; ++j) rr[j] -= f * cr[j];
    }
  }
  // solve L U X = P I column by column; store X row-major
  std::vector<double> inv((size_t)n * n), col(n);
  for (int e = 0; e < n; ++e) {
    std::fill(col.begin(), col.end(), 0.0);
    col[e] = 1.0;
    for (int c = 0; c < n; ++c) std::swap(col[c], col[piv[c]]);
    for (int r = 0; r < n; ++r) {
      double s = col[r];
      for (int j = 0; j < r; ++j) s -= a[(size_t)r * n + j] * col[j];
      col[r] = s;
    }
    for (int r = n - 1; r >= 0; --r) {
      double s = col[r];
      for (int j = r + 1; j < n; ++j) s -= a[(size_t)r * n + j] * col[j];
      col[r] = s / a[(size_t)r * n + r];
    }
    for (int r = 0; r < n; ++r) inv[(size_t)r * n + e] = col[r];
  }
  return inv;
}

}  // namespace

void validate(const HBsr& A, bool square) {
  if (A.nbr < 0 || A.nbc < 0) fail("negative dimension");
  if (A.br < 1 || A.br > 4 || A.bc < 1 || A.bc > 4) fail("bdim must be in 1..4");
  if ((int)A.ptr.size() != A.nbr + 1) fail("row_ptr has the wrong length");
  if (A.ptr[0] != 0) fail("row_ptr[0] != 0");
  for (int i = 0; i < A.nbr; ++i)
    if (A.ptr[i + 1] < A.ptr[i]) fail("row_ptr is not monotone at row " + std::to_string(i));
  if ((int64_t)A.ptr[A.nbr] != A.nnzb()) fail("row_ptr[n] != nnzb");
  if ((int64_t)A.val.size() != A.nnzb() * A.bsz()) fail("vals has the wrong length");
  for (int i = 0; i < A.nbr; ++i)
    for (int k = A.ptr[i]; k < A.ptr[i + 1]; ++k) {
      if (A.col[k] < 0 || A.col[k] >= A.nbc)
        fail("column index out of range in row " + std::to_string(i));
      if (k > A.ptr[i] && A.col[k] <= A.col[k - 1])
        fail("columns not strictly increasing in row " + std::to_string(i));
    }
  for (double v : A.val)
    if (!std::isfinite(v)) fail("non-finite matrix value");
  if (square && (A.nbr != A.nbc || A.br != A.bc)) fail("matrix must be square");
}

std::vector<int32_t> aggregate(const HBsr& A, double eps, int* n_agg_out) {
  auto s = block_fro2(A);
  auto dp = diag_pos(A);
  std::vector<double> d(A.nbr);
  for (int i = 0; i < A.nbr; ++i) d[i] = std::sqrt(s[dp[i]]);
  const double e2 = eps * eps;
  std::vector<char> strong(A.nnzb(), 0);
  for (int i = 0; i < A.nbr; ++i)
    for (int k = A.ptr[i]; k < A.ptr[i + 1]; ++k) {
      int j = A.col[k];
      if (j == i) continue;
      double thr = e2 * d[i];
      strong[k] = s[k] > thr * d[j];
    }
  std::vector<int32_t> agg(A.nbr, -1);
  int n_agg = 0;
  for (int i = 0; i < A.nbr; ++i) {
    if (agg[i] != -1) continue;
    bool free_nb = true;
    for (int k = A.ptr[i]; k < A.ptr[i + 1] && free_nb; ++k)
      if (strong[k] && agg[A.col[k]] != -1) free_nb = false;
    if (!free_nb) continue;
    agg[i] = n_agg;
    for (int k = A.ptr[i]; k < A.ptr[i + 1]; ++k)
      if (strong[k]) agg[A.col[k]] = n_agg;
    ++n_agg;
  }
  std::vector<int32_t> agg1 = agg;
  for (int i = 0; i < A.nbr; ++i) {
    if (agg[i] != -1) continue;
    double best_s = 0.0;
    int best_a = -1;
    for (int k = A.ptr[i]; k < A.ptr[i + 1]; ++k) {
      if (!strong[k]) continue;
      int a = agg1[A.col[k]];
      if (a < 0) continue;
      if (best_a < 0 || s[k] > best_s || (s[k] == best_s && a < best_a)) {
        best_s = s[k];
        best_a = a;
      }
    }
    if (best_a < 0) fail("aggregation left a node without an aggregated neighbour");
    agg[i] = best_a;
  }
  *n_agg_out = n_agg;
  return agg;
}

std::vector<double> spai0(const HBsr& A) {
  const int B = A.br, bs = B * B;
  auto dp = diag_pos(A);
  std::vector<double> M((size_t)A.nbr * bs);
  std::vector<double> G(bs), Gi(bs);
  for (int i = 0; i < A.nbr; ++i) {
    std::fill(G.begin(), G.end(), 0.0);
    for (int k = A.ptr[i]; k < A.ptr[i + 1]; ++k) {
      const double* a = &A.val[(size_t)k * bs];
      for (int r = 0; r < B; ++r)
        for (int c = 0; c < B; ++c) {
          double acc = 0.0;
          for (int t = 0; t < B; ++t) acc += a[r * B + t] * a[c * B + t];
          G[r * B + c] += acc;
        }
    }
    if (!blk_inv(B, G.data(), Gi.data()))
      fail("SPAI0 Gram matrix is singular at row " + std::to_string(i) + " (zero row?)");
    const double* d = &A.val[(size_t)dp[i] * bs];
    double* m = &M[(size_t)i * bs];
    for (int r = 0; r < B; ++r)
      for (int c = 0; c < B; ++c) {
        double acc = 0.0;
        for (int t = 0; t < B; ++t) acc += d[t * B + r] * Gi[t * B + c];
        m[r * B + c] = acc;
      }
  }
  return M;
}

std::vector<double> jacobi(const HBsr& A, double omega) {
  auto M = block_diag_inv(A);
  for (auto& v : M) v *= omega;
  return M;
}

HAmg build_amg(const HBsr& A0, const AmgSetupParams& prm) {
  validate(A0, true);
  HAmg H;
  H.B = A0.br;
  const int B = H.B, bs = B * B;
  HBsr A = A0;
  int l = 0;
  while ((int64_t)A.nbr * B > prm.coarse_enough && l < prm.max_levels - 1) {
    int n_agg = 0;
    auto agg = aggregate(A, std::ldexp(prm.eps_strong, -l), &n_agg);
    if (n_agg >= A.nbr) break;
    HLevel lev;
    lev.agg = agg;
    // smoothed prolongator, row by row
    HBsr P;
    P.nbr = A.nbr;
    P.nbc = n_agg;
    P.br = P.bc = B;
    P.ptr.assign(A.nbr + 1, 0);
    double omega = 0.0;
    std::vector<double> DinvA;
    if (prm.smooth_P) {
      auto Dinv = block_diag_inv(A);
      HBsr DA = A;
      for (int i = 0; i < A.nbr; ++i)
        for (int k = A.ptr[i]; k < A.ptr[i + 1]; ++k) {
          std::fill(&DA.val[(size_t)k * bs], &DA.val[(size_t)(k + 1) * bs], 0.0);
          blk_mul_add(B, &Dinv[(size_t)i * bs], &A.val[(size_t)k * bs], &DA.val[(size_t)k * bs]);
        }
      double rho = spectral_radius(DA, prm.power_iters);
      if (!(rho > 0.0)) fail("spectral radius estimate is zero");
      omega = (4.0 / 3.0) / rho;
      std::vector<int> mark(n_agg, -1);
      std::vector<int> cols;
      std::vector<double> acc;
      for (int i = 0; i < A.nbr; ++i) {
        cols.clear();
        acc.clear();
        for (int k = A.ptr[i]; k < A.ptr[i + 1]; ++k) {
          int a = agg[A.col[k]];
          if (mark[a] < 0) {
            mark[a] = (int)cols.size();
            cols.push_back(a);
            acc.resize(acc.size() + bs, 0.0);
          }
          double* t = &acc[(size_t)mark[a] * bs];
          const double* v = &DA.val[(size_t)k * bs];
          for (int e = 0; e < bs; ++e) t[e] += v[e];
        }
        std::vector<int> order(cols.size());
        for (size_t t = 0; t < order.size(); ++t) order[t] = (int)t;
        std::sort(order.begin(), order.end(), [&](int a, int b) { return cols[a] < cols[b]; });
        for (int t : order) {
          int a = cols[t];
          P.col.push_back(a);
          for (int r = 0; r < B; ++r)
            for (int c = 0; c < B; ++c) {
              double id = (a == agg[i] && r == c) ? 1.0 : 0.0;
              P.val.push_back(id - omega * acc[(size_t)t * bs + r * B + c]);
            }
        }
        for (int a : cols) mark[a] = -1;
        P.ptr[i + 1] = (int32_t)P.col.size();
      }
    } else {
      for (int i = 0; i < A.nbr; ++i) {
        P.col.push_back(agg[i]);
        for (int r = 0; r < B; ++r)
          for (int c = 0; c < B; ++c) P.val.push_back(r == c ? 1.0 : 0.0);
        P.ptr[i + 1] = i + 1;
      }
    }
    lev.omega = omega;
    HBsr R = transpose(P);
    HBsr AP = spgemm(A, P);
    HBsr Ac = spgemm(R, AP);
    if (prm.relax == 2) lev.ilu = ilut(to_scalar_csr(A), prm.ilut_p, prm.ilut_tau);
    else lev.M = prm.relax == 0 ? spai0(A) : jacobi(A, prm.jacobi_omega);
    lev.A = std::move(A);
    lev.P = std::move(P);
    lev.R = std::move(R);
    H.levels.push_back(std::move(lev));
    A = std::move(Ac);
    ++l;
  }
  if ((int64_t)A.nbr * B > 8192)
    fail("coarsest level has " + std::to_string((int64_t)A.nbr * B) +
         " unknowns (> 8192); raise max_levels or coarse_enough");
  H.Ainv = dense_inverse(A);
  H.Ac = std::move(A);
  return H;
}

HSchur schur_split(const HBsr& K, int nvel) {
  validate(K, true);
  const int B = nvel + 1;
  if (K.br != B) fail("Schur split needs bdim = nvel + 1");
  HSchur S;
  S.nvel = nvel;
  auto mk = [&](int br, int bc) {
    HBsr M;
    M.nbr = K.nbr;
    M.nbc = K.nbc;
    M.br = br;
    M.bc = bc;
    M.ptr = K.ptr;
    M.col = K.col;
    M.val.resize((size_t)K.nnzb() * br * bc);
    return M;
  };
  S.A = mk(nvel, nvel);
  S.G = mk(nvel, 1);
  S.D = mk(1, nvel);
  S.C = mk(1, 1);
  const int bs = B * B;
  for (int64_t k = 0; k < K.nnzb(); ++k) {
    const double* v = &K.val[(size_t)k * bs];
    for (int r = 0; r < nvel; ++r) {
      for (int c = 0; c < nvel; ++c) S.A.val[(size_t)k * nvel * nvel + r * nvel + c] = v[r * B + c];
      S.G.val[(size_t)k * nvel + r] = v[r * B + nvel];
      S.D.val[(size_t)k * nvel + r] = v[nvel * B + r];
    }
    S.C.val[k] = v[nvel * B + nvel];
  }
  // S_hat = C - diag(D diag(A)^-1 G)   (Eq. SchurApprox)
  auto dp = diag_pos(S.A);
  std::vector<double> dA((size_t)K.nbr * nvel);
  for (int i = 0; i < K.nbr; ++i)
    for (int c = 0; c < nvel; ++c) {
      dA[(size_t)i * nvel + c] = S.A.val[(size_t)dp[i] * nvel * nvel + c * nvel + c];
      if (dA[(size_t)i * nvel + c] == 0.0) fail("zero on the velocity diagonal");
    }
  S.S = S.C;
  auto dpc = diag_pos(S.C);
  for (int i = 0; i < K.nbr; ++i) {
    double corr = 0.0;
    for (int k = K.ptr[i]; k < K.ptr[i + 1]; ++k) {
      int j = K.col[k];
      int kt = find_col(K, j, i);
      if (kt < 0) continue;
      for (int c = 0; c < nvel; ++c)
        corr += S.D.val[(size_t)k * nvel + c] * (1.0 / dA[(size_t)j * nvel + c]) *
                S.G.val[(size_t)kt * nvel + c];
    }
    S.S.val[dpc[i]] -= corr;
  }
  return S;
}

HBsr scale_columns(const HBsr& A, const std::vector<double>& M) {
  if (A.br != A.bc) fail("scale_columns needs square blocks");
  const int B = A.br, bs = B * B;
  if ((int64_t)M.size() != (int64_t)A.nbc * bs) fail("scale_columns: M has the wrong size");
  HBsr C = A;
  for (int i = 0; i < A.nbr; ++i)
    for (int k = A.ptr[i]; k < A.ptr[i + 1]; ++k) {
      const double* a = &A.val[(size_t)k * bs];
      const double* m = &M[(size_t)A.col[k] * bs];
      double* c = &C.val[(size_t)k * bs];
      for (int r = 0; r < B; ++r)
        for (int cc = 0; cc < B; ++cc) {
          double acc = 0.0;
          for (int t = 0; t < B; ++t) acc += a[r * B + t] * m[t * B + cc];
          c[r * B + cc] = acc;
        }
    }
  return C;
}

HCsr to_scalar_csr(const HBsr& A) {
  HCsr C;
  C.n = A.nbr * A.br;
  C.ncols = A.nbc * A.bc;
  C.ptr.assign(C.n + 1, 0);
  const int bs = A.bsz();
  for (int i = 0; i < A.nbr; ++i)
    for (int a = 0; a < A.br; ++a) {
      const int row = i * A.br + a;
      for (int k = A.ptr[i]; k < A.ptr[i + 1]; ++k)
        for (int c = 0; c < A.bc; ++c) {
          const double v = A.val[(size_t)k * bs + a * A.bc + c];
          if (v == 0.0) continue;
          C.col.push_back(A.col[k] * A.bc + c);
          C.val.push_back(v);
        }
      C.ptr[row + 1] = (int32_t)C.col.size();
    }
  return C;
}

namespace {
bool same_bits(double a, double b) {
  uint64_t x, y;
  std::memcpy(&x, &a, 8);
  std::memcpy(&y, &b, 8);
  return x == y;
}
// One B x B row-major block: zero off the diagonal, equal diagonal.
bool iso_block(const double* v, int B) {
  for (int a = 0; a < B; ++a)
    for (int c = 0; c < B; ++c) {
      const double e = v[a * B + c];
      if (a == c ? !same_bits(e, v[0]) : e != 0.0) return false;
    }
  return true;
}
}  // namespace

bool is_iso(const HBsr& A) {
  if (A.br != A.bc || A.br < 2) return false;
  const int B = A.br, bs = B * B;
  for (size_t k = 0; k < A.col.size(); ++k)
    if (!iso_block(&A.val[k * bs], B)) return false;
  return true;
}

bool is_iso_blocks(const std::vector<double>& M, int B) {
  if (B < 2 || M.size() % ((size_t)B * B) != 0) return false;
  for (size_t k = 0; k < M.size(); k += (size_t)B * B)
    if (!iso_block(&M[k], B)) return false;
  return true;
}

HCsr iso_scalar(const HBsr& A) {
  HCsr C;
  C.n = A.nbr;
  C.ncols = A.nbc;
  C.ptr.assign(C.n + 1, 0);
  const int bs = A.bsz();
  for (int i = 0; i < A.nbr; ++i) {
    for (int k = A.ptr[i]; k < A.ptr[i + 1]; ++k) {
      const double v = A.val[(size_t)k * bs];
      if (v == 0.0) continue;
      C.col.push_back(A.col[k]);
      C.val.push_back(v);
    }
    C.ptr[i + 1] = (int32_t)C.col.size();
  }
  return C;
}

std::vector<double> iso_diag(const std::vector<double>& M, int B) {
  std::vector<double> m(M.size() / ((size_t)B * B));
  for (size_t i = 0; i < m.size(); ++i) m[i] = M[i * B * B];
  return m;
}

namespace {
// Layout of each slice of the sliced form: its width, and for a uniform
// slice the sorted union of its rows' column offsets (col - row).  A slice
// is uniform when that union is at most an eighth wider than its longest
// row (one more column at least); its entry k then sits at column
// row + union[k] in every lane.
struct SellPlan {
  std::vector<int32_t> width;
  std::vector<std::vector<int32_t>> uni;   // empty: explicit slice
};
// node of slot p (lane p % 32 of 32-node group p / 32); -1 past the end
inline int slot_node(const std::vector<int32_t>& ord, int p, int nn) {
  if (p >= nn) return -1;
  return ord.empty() ? p : ord[p];
}
SellPlan sell_plan(const HCsr& C, int B, const std::vector<int32_t>& ord) {
  const int nn = C.n / B;
  const int ng = (nn + 31) / 32;
  SellPlan P;
  P.width.assign((size_t)ng * B, 0);
  P.uni.assign((size_t)ng * B, {});
  std::vector<int32_t> offs;
  for (int g = 0; g < ng; ++g)
    for (int c = 0; c < B; ++c) {
      const size_t q = (size_t)g * B + c;
      int wmax = 0;
      offs.clear();
      for (int p = g * 32; p < std::min(nn, g * 32 + 32); ++p) {
        const int row = slot_node(ord, p, nn) * B + c;
        wmax = std::max(wmax, C.ptr[row + 1] - C.ptr[row]);
        for (int k = C.ptr[row]; k < C.ptr[row + 1]; ++k) offs.push_back(C.col[k] - row);
      }
      std::sort(offs.begin(), offs.end());
      offs.erase(std::unique(offs.begin(), offs.end()), offs.end());
      const int wu = (int)offs.size();
      if (wmax > 0 && wu <= wmax + std::max(1, wmax / 8)) {
        P.width[q] = wu;
        P.uni[q] = offs;
      } else {
        P.width[q] = wmax;
      }
    }
  return P;
}
// Nodes sorted by their rows' total length, longest first, within windows
// of 32 groups (1024 nodes; stable, so equal lengths keep their order).
std::vector<int32_t> sell_order(const HCsr& C, int B) {
  const int nn = C.n / B;
  std::vector<int32_t> ord(nn);
  std::vector<int32_t> len(nn);
  for (int i = 0; i < nn; ++i) {
    ord[i] = i;
    len[i] = C.ptr[(i + 1) * B] - C.ptr[i * B];
  }
  constexpr int W = 32 * 32;
  for (int w0 = 0; w0 < nn; w0 += W)
    std::stable_sort(ord.begin() + w0, ord.begin() + std::min(nn, w0 + W),
                     [&](int a, int b) { return len[a] > len[b]; });
  return ord;
}
}  // namespace

double sell_padding(const HCsr& C, int B, bool sorted) {
  if (B < 1 || C.n % B != 0 || C.col.empty()) return 0.0;
  int64_t slots = 0;
  const std::vector<int32_t> ord = sorted ? sell_order(C, B) : std::vector<int32_t>();
  for (int32_t w : sell_plan(C, B, ord).width) slots += (int64_t)w * 32;
  return (double)slots / (double)C.col.size() - 1.0;
}

HSell to_sell(const HCsr& C, int B, bool sorted) {
  if (B < 1 || C.n % B != 0) throw SetupError{"sliced CSR needs whole nodes"};
  HSell S;
  S.n = C.n;
  S.B = B;
  const int nn = C.n / B;
  std::vector<int32_t> ord;
  if (sorted) {
    ord = sell_order(C, B);
    S.node = ord;
    S.node.resize((size_t)((nn + 31) / 32) * 32, -1);
  }
  const SellPlan P = sell_plan(C, B, ord);
  S.nslices = (int)P.width.size();
  S.off.assign(S.nslices + 1, 0);
  S.cinfo.assign(S.nslices, 0);
  for (int q = 0; q < S.nslices; ++q) {
    if ((int64_t)S.off[q] + P.width[q] > INT32_MAX / 32) throw SetupError{"sliced CSR too large"};
    S.off[q + 1] = S.off[q] + P.width[q];
    if (!P.uni[q].empty()) {
      S.cinfo[q] = -1 - (int32_t)S.uoff.size();
      S.uoff.insert(S.uoff.end(), P.uni[q].begin(), P.uni[q].end());
      S.umask.insert(S.umask.end(), P.uni[q].size(), 0u);
    }
  }
  const size_t slots = (size_t)S.off[S.nslices] * 32;
  S.col.assign(slots, -1);
  S.val.assign(slots, 0.0);
  S.src.assign(slots, -1);
  for (int p = 0; p < nn; ++p)
    for (int c = 0; c < B; ++c) {
      const int row = slot_node(ord, p, nn) * B + c;
      const int q = (p / 32) * B + c, lane = p % 32;
      const std::vector<int32_t>& u = P.uni[q];
      size_t kk = 0;   // position in the union (uniform slices)
      for (int k = C.ptr[row]; k < C.ptr[row + 1]; ++k) {
        size_t pos = (size_t)(k - C.ptr[row]);
        if (!u.empty()) {
          while (u[kk] != C.col[k] - row) ++kk;
          pos = kk;
          S.umask[(size_t)(-1 - S.cinfo[q]) + kk] |= 1u << lane;
        }
        const size_t e = ((size_t)S.off[q] + pos) * 32 + lane;
        S.col[e] = C.col[k];
        S.val[e] = C.val[k];
        S.src[e] = k;
      }
    }
  return S;
}

namespace {
// Slot order of to_bsell: rows sorted by length, longest first, within
// windows of window * R rows (stable, so equal lengths keep row order).
std::vector<int32_t> bsell_order(const HBsr& A, int R, int window) {
  std::vector<int32_t> ord(A.nbr);
  for (int i = 0; i < A.nbr; ++i) ord[i] = i;
  const int W = std::max(1, window) * R;
  for (int w0 = 0; w0 < A.nbr; w0 += W) {
    const int w1 = std::min(A.nbr, w0 + W);
    std::stable_sort(ord.begin() + w0, ord.begin() + w1, [&](int a, int b) {
      return A.ptr[a + 1] - A.ptr[a] > A.ptr[b + 1] - A.ptr[b];
    });
  }
  return ord;
}
}  // namespace

double bsell_padding(const HBsr& A, int window) {
  if (A.br != A.bc || A.nnzb() == 0) return 0.0;
  const int R = 32 / A.br;
  const std::vector<int32_t> ord = bsell_order(A, R, window);
  int64_t slots = 0;
  for (int q0 = 0; q0 < A.nbr; q0 += R) {
    int w = 0;
    for (int i = q0; i < std::min(A.nbr, q0 + R); ++i)
      w = std::max(w, A.ptr[ord[i] + 1] - A.ptr[ord[i]]);
    slots += (int64_t)w * R;
  }
  return (double)slots / (double)A.nnzb() - 1.0;
}

HBSell to_bsell(const HBsr& A, int window) {
  if (A.br != A.bc || A.br < 1 || A.br > 4) throw SetupError{"block slices need square blocks"};
  HBSell S;
  S.nbr = A.nbr;
  S.B = A.br;
  S.R = 32 / A.br;
  const int R = S.R, bs = A.bsz();
  const std::vector<int32_t> ord = bsell_order(A, R, window);
  S.nslices = (A.nbr + R - 1) / R;
  S.perm.assign((size_t)S.nslices * R, -1);
  S.off.assign(S.nslices + 1, 0);
  for (int q = 0; q < S.nslices; ++q) {
    int w = 0;
    for (int i = 0; i < R && q * R + i < A.nbr; ++i) {
      const int row = ord[q * R + i];
      S.perm[(size_t)q * R + i] = row;
      w = std::max(w, A.ptr[row + 1] - A.ptr[row]);
    }
    if ((int64_t)S.off[q] + w > INT32_MAX / (32 * 16)) throw SetupError{"block slices too large"};
    S.off[q + 1] = S.off[q] + w;
  }
  const size_t nb = (size_t)S.off[S.nslices] * R;
  S.col.assign(nb, 0);
  S.val.assign(nb * bs, 0.0);
  for (int q = 0; q < S.nslices; ++q)
    for (int i = 0; i < R; ++i) {
      const int row = S.perm[(size_t)q * R + i];
      const int w = S.off[q + 1] - S.off[q];
      for (int k = 0; k < w; ++k) {
        const size_t e = ((size_t)S.off[q] + k) * R + i;
        if (row < 0) continue;
        const int len = A.ptr[row + 1] - A.ptr[row];
        if (k < len) {
          const int src = A.ptr[row] + k;
          S.col[e] = A.col[src];
          std::copy(A.val.begin() + (size_t)src * bs, A.val.begin() + (size_t)(src + 1) * bs,
                    S.val.begin() + e * bs);
        } else {
          S.col[e] = row;   // zero block on the row's own column
        }
      }
    }
  return S;
}

HIlu ilut(const HCsr& A, double p, double tau) {
  const int n = A.n;
  if (A.ncols != n) fail("ILUT needs a square matrix");
  HIlu F;
  F.L.n = F.U.n = n;
  F.L.ncols = F.U.ncols = n;
  F.L.ptr.assign(n + 1, 0);
  F.U.ptr.assign(n + 1, 0);
  F.d.assign(n, 0.0);
  std::vector<double> w(n, 0.0);
  std::vector<char> present(n, 0);
  std::vector<int> cols;
  std::vector<std::pair<int, double>> lower, upper;
  auto keep = [](std::vector<std::pair<int, double>>& e, int count) {
    if ((int)e.size() > count) {
      std::sort(e.begin(), e.end(), [](const std::pair<int, double>& a,
                                       const std::pair<int, double>& b) {
        const double fa = std::fabs(a.second), fb = std::fabs(b.second);
        return fa > fb || (fa == fb && a.first < b.first);
      });
      e.resize(count < 0 ? 0 : count);
    }
    std::sort(e.begin(), e.end());
  };
  for (int i = 0; i < n; ++i) {
    cols.clear();
    int nzL = 0, nzU = 0;
    double s2 = 0.0;
    for (int k = A.ptr[i]; k < A.ptr[i + 1]; ++k) {
      const double v = A.val[k];
      if (v == 0.0) continue;
      const int j = A.col[k];
      w[j] = v;
      present[j] = 1;
      cols.push_back(j);
      s2 += v * v;
      if (j < i) ++nzL;
      else if (j > i) ++nzU;
    }
    const double tau_i = tau * std::sqrt(s2);
    // lower columns in increasing order, fill included (a min-heap)
    std::vector<int> heap;
    for (int j : cols)
      if (j < i) heap.push_back(j);
    std::make_heap(heap.begin(), heap.end(), std::greater<int>());
    while (!heap.empty()) {
      std::pop_heap(heap.begin(), heap.end(), std::greater<int>());
      const int k = heap.back();
      heap.pop_back();
      if (std::fabs(w[k]) < tau_i) {   // tested before the division (scale-free)
        w[k] = 0.0;
        continue;
      }
      const double wk = w[k] / F.d[k];
      w[k] = wk;
      for (int e = F.U.ptr[k]; e < F.U.ptr[k + 1]; ++e) {
        const int j = F.U.col[e];
        if (!present[j]) {
          present[j] = 1;
          w[j] = 0.0;
          cols.push_back(j);
          if (j < i) {
            heap.push_back(j);
            std::push_heap(heap.begin(), heap.end(), std::greater<int>());
          }
        }
        w[j] -= wk * F.U.val[e];
      }
    }
    lower.clear();
    upper.clear();
    for (int j : cols) {
      const double v = w[j];
      if (j == i || v == 0.0) continue;
      if (j < i) lower.emplace_back(j, v);   // multipliers, tested during elimination
      else if (std::fabs(v) >= tau_i) upper.emplace_back(j, v);
    }
    keep(lower, (int)std::floor(p * nzL));
    keep(upper, (int)std::floor(p * nzU));
    for (const auto& e : lower) {
      F.L.col.push_back(e.first);
      F.L.val.push_back(e.second);
    }
    for (const auto& e : upper) {
      F.U.col.push_back(e.first);
      F.U.val.push_back(e.second);
    }
    F.L.ptr[i + 1] = (int32_t)F.L.col.size();
    F.U.ptr[i + 1] = (int32_t)F.U.col.size();
    double di = present[i] ? w[i] : 0.0;
    if (di == 0.0) di = tau_i != 0.0 ? tau_i : 1.0;
    F.d[i] = di;
    for (int j : cols) {
      w[j] = 0.0;
      present[j] = 0;
    }
  }
  return F;
}

HCsr transpose(const HCsr& A) {
  HCsr T;
  T.n = A.ncols;
  T.ncols = A.n;
  T.ptr.assign(T.n + 1, 0);
  for (int32_t c : A.col) ++T.ptr[c + 1];
  for (int i = 0; i < T.n; ++i) T.ptr[i + 1] += T.ptr[i];
  T.col.resize(A.col.size());
  T.val.resize(A.val.size());
  std::vector<int32_t> next(T.ptr.begin(), T.ptr.end() - 1);
  for (int i = 0; i < A.n; ++i)
    for (int k = A.ptr[i]; k < A.ptr[i + 1]; ++k) {
      const int32_t at = next[A.col[k]]++;
      T.col[at] = i;
      T.val[at] = A.val[k];
    }
  return T;
}

double block_fill(const HBsr& A) {
  if (A.val.empty()) return 1.0;
  size_t nz = 0;
  for (double v : A.val) nz += v != 0.0;
  return (double)nz / (double)A.val.size();
}

bool transpose_map(const HBsr& A, std::vector<int32_t>& tmap) {
  tmap.assign(A.nnzb(), -1);
  for (int i = 0; i < A.nbr; ++i)
    for (int k = A.ptr[i]; k < A.ptr[i + 1]; ++k) {
      int j = A.col[k];
      if (j >= A.nbr) return false;
      int t = find_col(A, j, i);
      if (t < 0) return false;
      tmap[k] = t;
    }
  return true;
}

}  // namespace gbs
