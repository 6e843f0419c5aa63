// C ABI (include/gbstokes.h): hierarchy build/import, BiCGStab and
// GMRES drivers on the FP64 outer operator, adjoint solve, sampled outer
// product.  The Krylov loops run on the host and launch device kernels;
// iteration scalars stay on the device and one small device-to-host read
// per iteration decides convergence.  Optionally each BiCGStab iteration
// is replayed from a captured CUDA graph.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <memory>
#include <string>
#include <vector>

#include "../../include/gbstokes.h"
#include "amg_dev.cuh"
#include "device.hpp"
#include "outer.cuh"
#include "setup.hpp"

namespace gbs {

thread_local std::string g_err;
static std::atomic<int64_t> g_launches{0};
void count_launch(int64_t k) { g_launches.fetch_add(k, std::memory_order_relaxed); }
int64_t launch_count() { return g_launches.load(std::memory_order_relaxed); }

struct Handle {
  gbs_params prm{};
  int B = 1;
  int64_t n = 0;
  HBsr Kh;                       // host copy of K (pattern + FP64 values)
  DevBsr<double> K;
  double* Kval = nullptr;
  // K as scalar CSR of its build-time nonzeros (per-level format choice);
  // the block form stays the source of truth for updates and K^T
  DevCsr<double> Kc;
  DevSell<double> Ks;            // the same nonzeros in uniform 32-node slices (k_sell)
  bool k_csr = false;
  bool k_sell = false;
  bool k_check_pending = false;
  int* kmap = nullptr;          // CSR entry -> flat block-value index
  int64_t kmap_n = 0;
  double* kcval = nullptr;
  unsigned* kzero = nullptr;    // bit i: block value i is outside the CSR pattern
  int* kflag = nullptr;
  std::unique_ptr<DevPrecond> pc;
  bool schur = false;
  HAmg H, HA, HS;                // host hierarchies (export)
  HSchur Sh;
  Arena ar;
  // work vectors
  double *r, *rhat, *p, *ph, *v, *s, *sh, *t, *xi, *bi;
  double *V = nullptr, *hcol, *hcol2, *ydev, *z, *u;
  double *Pidr = nullptr, *Gidr = nullptr, *Uidr = nullptr;  // IDR(s): s x n each
  int m = 30;
  double* sc;
  double* sc_host = nullptr;     // pinned
  double* h_host = nullptr;      // pinned
  Red red;
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
  cudaStream_t cap = nullptr;
  cudaGraphExec_t gexec[2] = {nullptr, nullptr};  // BiCGStab iteration, fwd / adjoint
  int64_t gnodes[2] = {0, 0};                     // kernels per graph replay
  // GMRES: the device part of Arnoldi step j (basis size j + 1), fwd / adjoint
  std::vector<cudaGraphExec_t> garn[2];
  std::vector<int64_t> garn_nodes[2];
  void drop_graphs() {
    for (auto& g : gexec)
      if (g) cudaGraphExecDestroy(g), g = nullptr;
    for (auto& v : garn)
      for (auto& g : v)
        if (g) cudaGraphExecDestroy(g), g = nullptr;
  }
  ~Handle() {
    drop_graphs();
    if (cap) cudaStreamDestroy(cap);
    if (ev0) cudaEventDestroy(ev0);
    if (ev1) cudaEventDestroy(ev1);
    if (sc_host) cudaFreeHost(sc_host);
    if (h_host) cudaFreeHost(h_host);
  }
};

namespace {

cudaStream_t S(void* s) { return reinterpret_cast<cudaStream_t>(s); }

std::vector<double> idr_shadow_space(int64_t n, int s, uint64_t seed);

// Grid of an elementwise kernel: one thread per element up to `cap` CTAs of
// 256 threads (the device's resident CTAs, Red::cap).
unsigned vgrid(int64_t n, int cap) {
  return (unsigned)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, cap));
}

HBsr from_c(const gbs_bsr* A) {
  if (!A) throw SetupError{"null matrix"};
  if (A->n_brows < 0 || A->n_bcols < 0 || A->nnzb < 0 || A->bdim < 1 || A->bdim > 4)
    throw SetupError{"bad matrix dimensions"};
  if (!A->row_ptr || (A->nnzb > 0 && (!A->col_idx || !A->vals)))
    throw SetupError{"null matrix array"};
  if (A->nnzb > INT32_MAX) throw SetupError{"nnzb exceeds int32 range"};
  HBsr H;
  H.nbr = A->n_brows;
  H.nbc = A->n_bcols;
  H.br = H.bc = A->bdim;
  H.ptr.assign(A->row_ptr, A->row_ptr + A->n_brows + 1);
  if (H.ptr.back() != A->nnzb) throw SetupError{"row_ptr[n_brows] != nnzb"};
  H.col.assign(A->col_idx, A->col_idx + A->nnzb);
  H.val.assign(A->vals, A->vals + A->nnzb * A->bdim * A->bdim);
  return H;
}

void check_params(const gbs_params* p) {
  if (!p) throw SetupError{"null params"};
  if (p->precond != GBS_PC_AMG && p->precond != GBS_PC_SCHUR) throw SetupError{"bad precond"};
  if (p->krylov != GBS_BICGSTAB && p->krylov != GBS_GMRES && p->krylov != GBS_IDRS)
    throw SetupError{"bad krylov"};
  if (p->krylov == GBS_IDRS && (p->idr_s < 1 || p->idr_s > 8)) throw SetupError{"idr_s must be in 1..8"};
  if (p->restart < 1 || p->restart > 64) throw SetupError{"restart must be in 1..64"};
  if (!(p->tol > 0.0)) throw SetupError{"tol must be > 0"};
  if (p->maxiter < 1) throw SetupError{"maxiter must be >= 1"};
  if (p->replace_every < 1) throw SetupError{"replace_every must be >= 1"};
  if (p->precision < GBS_FP64 || p->precision > GBS_BF16) throw SetupError{"bad precision"};
  if (p->npre < 0 || p->npost < 1) throw SetupError{"need npre >= 0 and npost >= 1"};
  if (p->relax != GBS_SPAI0 && p->relax != GBS_JACOBI && p->relax != GBS_ILUT)
    throw SetupError{"bad relax"};
  if (p->relax_p != GBS_SPAI0 && p->relax_p != GBS_JACOBI && p->relax_p != GBS_ILUT)
    throw SetupError{"bad relax_p"};
  if (p->precond == GBS_PC_SCHUR && p->schur_p == 1 && p->relax_p == GBS_ILUT)
    throw SetupError{"the single-sweep pressure solve (schur_p = 1) takes SPAI0 or Jacobi"};
  if (!(p->ilut_p >= 0.0) || !(p->ilut_tau >= 0.0) || !(p->ilut_omega > 0.0) ||
      p->ilut_sweeps < 0 || p->ilut_sweeps > 16)
    throw SetupError{"bad ILUT parameters (p >= 0, tau >= 0, omega > 0, sweeps 0..16)"};
  if (p->max_levels < 1 || p->coarse_enough < 1) throw SetupError{"bad level limits"};
  if (p->precond == GBS_PC_SCHUR && (p->nvel < 1 || p->nvel > 3))
    throw SetupError{"nvel must be in 1..3"};
  if (p->level_format < 0 || p->level_format > 3) throw SetupError{"level_format must be 0..3"};
  if (p->schur_p < 0 || p->schur_p > 1) throw SetupError{"schur_p must be 0 or 1"};
  if (p->schur_order < 0 || p->schur_order > 1) throw SetupError{"schur_order must be 0 or 1"};
  if (p->gmres_reorth < 0 || p->gmres_reorth > 2) throw SetupError{"gmres_reorth must be 0, 1 or 2"};
  if (p->wait_log2 < 0 || p->wait_log2 > 40) throw SetupError{"wait_log2 must be in 0..40"};
  if (p->iso_blocks < 0 || p->iso_blocks > 1) throw SetupError{"iso_blocks must be 0 or 1"};
}

AmgSetupParams amg_prm(const gbs_params* p, int relax) {
  AmgSetupParams a;
  a.eps_strong = p->eps_strong;
  a.coarse_enough = p->coarse_enough;
  a.max_levels = p->max_levels;
  a.relax = relax;
  a.jacobi_omega = p->jacobi_omega;
  a.smooth_P = p->smooth_P != 0;
  a.power_iters = p->power_iters;
  a.ilut_p = p->ilut_p;
  a.ilut_tau = p->ilut_tau;
  return a;
}

PrecondOptions pc_opts(const gbs_params* p) {
  PrecondOptions o;
  o.precision = p->precision;
  o.npre = p->npre;
  o.npost = p->npost;
  o.tmaps = p->enable_adjoint != 0;
  o.level_format = p->level_format;
  o.schur_order = p->schur_order;
  o.schur_p_smoother = p->schur_p == 1;
  o.ilut_sweeps = p->ilut_sweeps;
  o.ilut_omega = p->ilut_omega;
  o.wait_cycles = 1LL << p->wait_log2;
  o.iso = p->iso_blocks != 0;
  return o;
}

void alloc_work(Handle& h, cudaStream_t s) {
  Arena& a = h.ar;
  const int64_t n = h.n;
  const std::vector<double> kv = padded_vals<double>(h.Kh.val);   // see CHUNK_PAD
  h.Kval = a.upload(kv.data(), kv.size(), s);
  h.K.nbr = h.Kh.nbr;
  h.K.nbc = h.Kh.nbc;
  h.K.rp = a.upload(h.Kh.ptr.data(), h.Kh.ptr.size(), s);
  const std::vector<int32_t> kc = padded_cols(h.Kh.col);
  h.K.col = a.upload(kc.data(), kc.size(), s);
  h.K.val = h.Kval;
  switch (h.B) {
    case 1: h.K.G = choose_group<1, double, double>(h.Kh.nbr, h.Kh.nnzb()); break;
    case 2: h.K.G = choose_group<2, double, double>(h.Kh.nbr, h.Kh.nnzb()); break;
    case 3: h.K.G = choose_group<3, double, double>(h.Kh.nbr, h.Kh.nnzb()); break;
    default: h.K.G = choose_group<4, double, double>(h.Kh.nbr, h.Kh.nnzb()); break;
  }
  if (h.K.G == 256) h.K.G = 32;  // the outer SpMV keeps lane groups inside a warp
  if (const char* e = std::getenv("GBS_SPMV_GROUP")) {  // tuning override
    int g = std::atoi(e);
    if (g == 0 || g == 8 || g == 16 || g == 32) h.K.G = g;
    if (h.K.G == 256) h.K.G = 32;
  }
  if (use_scalar_csr(h.Kh, h.prm.level_format)) {
    HCsr c = to_scalar_csr(h.Kh);
    std::vector<int32_t> map;
    std::vector<unsigned> zero((h.Kh.val.size() + 31) / 32, 0u);
    const int bs = h.Kh.bsz();
    map.reserve(c.col.size());
    for (int i = 0; i < h.Kh.nbr; ++i)
      for (int a = 0; a < h.Kh.br; ++a)
        for (int k = h.Kh.ptr[i]; k < h.Kh.ptr[i + 1]; ++k)
          for (int cc = 0; cc < h.Kh.bc; ++cc) {
            const size_t flat = (size_t)k * bs + a * h.Kh.bc + cc;
            if (h.Kh.val[flat] != 0.0) map.push_back((int32_t)flat);
            else zero[flat >> 5] |= 1u << (flat & 31);
          }
    HSell S;
    bool sliced = false;
    if (use_sell(c, h.B, h.prm.level_format) == 1) {   // K: stencil slices only
      S = to_sell(c, h.B);
      int64_t uni = 0;
      for (int32_t ci : S.cinfo) uni += ci < 0;
      // only a stencil K gains: its slices need no column loads
      sliced = level_format_of(h.prm.level_format) == 3 || uni * 10 >= (int64_t)S.nslices * 9;
    }
    if (sliced) {
      std::vector<int32_t> smap(S.src.size());
      for (size_t e = 0; e < S.src.size(); ++e) smap[e] = S.src[e] >= 0 ? map[S.src[e]] : -1;
      std::vector<std::vector<double>> keep;
      h.Ks = upload_sell<double>(a, S, h.sc + S_ERR, 1LL << 31, s, keep);
      h.kcval = const_cast<double*>(h.Ks.val);
      h.kmap = a.upload(smap.data(), smap.size(), s);
      h.kmap_n = (int64_t)smap.size();
      h.k_sell = true;
      GBS_CUDA(cudaStreamSynchronize(s));   // host staging dies here
    } else {
      h.Kc.n = c.n;
      h.Kc.rp = a.upload(c.ptr.data(), c.ptr.size(), s);
      h.Kc.col = a.upload(c.col.data(), c.col.size(), s);
      h.kcval = a.upload(c.val.data(), c.val.size(), s);
      h.Kc.val = h.kcval;
      h.Kc.S = csr_split(c.n, (int64_t)c.col.size());
      h.kmap = a.upload(map.data(), map.size(), s);
      h.kmap_n = (int64_t)map.size();
    }
    h.kzero = a.upload(zero.data(), zero.size(), s);
    h.kflag = a.alloc<int>(1);
    GBS_CUDA(cudaMemsetAsync(h.kflag, 0, sizeof(int), s));
    h.k_csr = true;
  }
  if (h.prm.enable_adjoint) {
    std::vector<int32_t> tm;
    if (!transpose_map(h.Kh, tm))
      throw SetupError{"K's block pattern is not structurally symmetric (needed for the adjoint)"};
    h.K.tmap = a.upload(tm.data(), tm.size(), s);
  }
  for (double** q : {&h.r, &h.rhat, &h.p, &h.ph, &h.v, &h.s, &h.sh, &h.t, &h.xi, &h.bi})
    *q = a.alloc<double>(n);
  h.m = h.prm.restart;
  if (h.prm.krylov == GBS_GMRES) {
    h.V = a.alloc<double>((size_t)(h.m + 1) * n);
    h.z = a.alloc<double>(n);
    h.u = a.alloc<double>(n);
  }
  if (h.prm.krylov == GBS_IDRS) {
    const int sdim = h.prm.idr_s;
    std::vector<double> P = idr_shadow_space(n, sdim, (uint64_t)(uint32_t)h.prm.idr_seed);
    h.Pidr = a.upload(P.data(), P.size(), s);
    h.Gidr = a.alloc<double>((size_t)sdim * n);
    h.Uidr = a.alloc<double>((size_t)sdim * n);
  }
  h.hcol = a.alloc<double>(MAX_DOTS);
  h.hcol2 = a.alloc<double>(MAX_DOTS);
  h.ydev = a.alloc<double>(MAX_DOTS);
  GBS_CUDA(cudaMemsetAsync(h.sc, 0, sizeof(double) * S_COUNT, s));
  h.red.sc = h.sc;
  // reduction partials for one wave of 256-thread CTAs on this device
  int dev = 0, sms = 0;
  GBS_CUDA(cudaGetDevice(&dev));
  GBS_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  h.red.cap = std::max(1, sms) * (2048 / RED_THREADS);
  h.red.partials = a.alloc<double>((size_t)h.red.cap * MAX_DOTS);
  h.red.counter = a.alloc<unsigned>(16);
  GBS_CUDA(cudaMemsetAsync(h.red.counter, 0, sizeof(unsigned) * 16, s));
  GBS_CUDA(cudaMallocHost(&h.sc_host, sizeof(double) * S_COUNT));
  GBS_CUDA(cudaMallocHost(&h.h_host, sizeof(double) * MAX_DOTS));
  GBS_CUDA(cudaEventCreate(&h.ev0));
  GBS_CUDA(cudaEventCreate(&h.ev1));
  GBS_CUDA(cudaStreamCreateWithFlags(&h.cap, cudaStreamNonBlocking));
  GBS_CUDA(cudaStreamSynchronize(s));
}

// ----------------------------------------------------------- outer kernels
template <bool TR, int MODE>
void outer_B(const Handle& h, const double* x, const double* f, double* y, const double* w0,
             int self_dot, int slot, int op, bool reduce, cudaStream_t s) {
  const Red& R = h.red;
#define GBS_OUTG(BB, GG) \
  launch_resident(k_outer<BB, GG, TR, MODE>, h.red.cap, s, h.K, x, f, y, w0, self_dot, R, slot, \
                                                                op, reduce)
#define GBS_OUT(BB)                                                                        \
  switch (h.K.G) {                                                                         \
    case 0:                                                                                \
      launch_resident(k_outer_n<BB, TR, MODE>, h.red.cap / 2, s, h.K, x, f, y, w0, self_dot, R, \
                                                                  slot, op, reduce);       \
      break;                                                                               \
    case 8: GBS_OUTG(BB, 8); break;                                                        \
    case 16: GBS_OUTG(BB, 16); break;                                                      \
    default: GBS_OUTG(BB, 32); break;                                                      \
  }
  switch (h.B) {
    case 1: GBS_OUT(1); break;
    case 2: GBS_OUT(2); break;
    case 3: GBS_OUT(3); break;
    case 4: GBS_OUT(4); break;
  }
#undef GBS_OUT
#undef GBS_OUTG
  GBS_LAUNCH_CHECK();
}
// y = K x or f - K x (K^T when tr); d0 = y . w0 (w0 != y), d1 = y . y if self_dot.
template <int MODE>
void outer_csr(const Handle& h, const double* x, const double* f, double* y, const double* w0,
               int self_dot, int slot, int op, bool reduce, cudaStream_t s) {
  const Red& R = h.red;
  switch (h.Kc.S) {
    case 2: launch_resident(k_outer_csr<2, MODE>, h.red.cap, s, h.Kc, x, f, y, w0, self_dot, R, slot, op, reduce); break;
    case 4: launch_resident(k_outer_csr<4, MODE>, h.red.cap, s, h.Kc, x, f, y, w0, self_dot, R, slot, op, reduce); break;
    case 8: launch_resident(k_outer_csr<8, MODE>, h.red.cap, s, h.Kc, x, f, y, w0, self_dot, R, slot, op, reduce); break;
    default: launch_resident(k_outer_csr<1, MODE>, h.red.cap, s, h.Kc, x, f, y, w0, self_dot, R, slot, op, reduce);
  }
  GBS_LAUNCH_CHECK();
}

void outer(const Handle& h, bool tr, int mode, const double* x, const double* f, double* y,
           const double* w0, int self_dot, int slot, int op, bool reduce, cudaStream_t s) {
  NvtxRange range(mode == SPMV_RESID ? "outer residual" : "outer SpMV");
  if (!tr && h.k_csr && h.k_sell) {
#define GBS_OSELL(MM, BB)                                                                      \
  launch_resident(k_outer_sell<MM, BB>, h.red.cap, s, h.Ks, x, f, y, w0, self_dot, h.red, slot, \
                  op, (int)reduce)
    const bool res = mode == SPMV_RESID;
    switch (h.B) {
      case 1: if (res) GBS_OSELL(SPMV_RESID, 1); else GBS_OSELL(SPMV_SET, 1); break;
      case 2: if (res) GBS_OSELL(SPMV_RESID, 2); else GBS_OSELL(SPMV_SET, 2); break;
      case 3: if (res) GBS_OSELL(SPMV_RESID, 3); else GBS_OSELL(SPMV_SET, 3); break;
      default: if (res) GBS_OSELL(SPMV_RESID, 4); else GBS_OSELL(SPMV_SET, 4); break;
    }
#undef GBS_OSELL
    GBS_LAUNCH_CHECK();
    return;
  }
  if (!tr && h.k_csr) {
    if (mode == SPMV_RESID) outer_csr<SPMV_RESID>(h, x, f, y, w0, self_dot, slot, op, reduce, s);
    else outer_csr<SPMV_SET>(h, x, f, y, w0, self_dot, slot, op, reduce, s);
    return;
  }
  if (tr) {
    if (mode == SPMV_RESID) outer_B<true, SPMV_RESID>(h, x, f, y, w0, self_dot, slot, op, reduce, s);
    else outer_B<true, SPMV_SET>(h, x, f, y, w0, self_dot, slot, op, reduce, s);
  } else {
    if (mode == SPMV_RESID) outer_B<false, SPMV_RESID>(h, x, f, y, w0, self_dot, slot, op, reduce, s);
    else outer_B<false, SPMV_SET>(h, x, f, y, w0, self_dot, slot, op, reduce, s);
  }
}

void read_scalars(Handle& h, cudaStream_t s) {
  GBS_CUDA(cudaMemcpyAsync(h.sc_host, h.sc, sizeof(double) * S_COUNT, cudaMemcpyDeviceToHost, s));
  GBS_CUDA(cudaStreamSynchronize(s));
  if (h.sc_host[S_ERR] != 0.0) {
    GBS_CUDA(cudaMemsetAsync(h.sc + S_ERR, 0, sizeof(double), s));
    GBS_CUDA(cudaStreamSynchronize(s));
    throw CudaError{"a pipelined SpMV kernel timed out waiting for its copies"};
  }
}

// One BiCGStab iteration (all device work, no host reads).
void bicg_iteration(Handle& h, bool tr, cudaStream_t s) {
  NvtxRange range("BiCGStab iteration");
  const int64_t n = h.n;
  const unsigned g = vgrid(n, h.red.cap);
  ::gbs::launch_k(k_bicg_p, g, 256, 0, s, n, h.r, h.v, h.p, h.sc);
  GBS_LAUNCH_CHECK();
  h.pc->apply(h.p, h.ph, tr, s);
  outer(h, tr, SPMV_SET, h.ph, nullptr, h.v, h.rhat, 0, 0, FIN_ALPHA, true, s);
  ::gbs::launch_k(k_bicg_s, g, 256, 0, s, n, h.r, h.v, h.s, h.sc);
  GBS_LAUNCH_CHECK();
  h.pc->apply(h.s, h.sh, tr, s);
  outer(h, tr, SPMV_SET, h.sh, nullptr, h.t, h.s, 1, 1, FIN_OMEGA, true, s);
  launch_resident(k_bicg_xr, h.red.cap, s, n, h.xi, h.ph, h.sh, h.s, h.t, h.r, h.rhat, h.red, 2);
  GBS_LAUNCH_CHECK();
}

// Run body(stream) on s from a CUDA graph, captured on h.cap at the first
// call and kept in ge (nodes: kernels a replay launches).
template <class F>
void replay(Handle& h, cudaGraphExec_t& ge, int64_t& nodes, cudaStream_t s, F&& body) {
  if (!ge) {
    cudaGraph_t g = nullptr;
    GBS_CUDA(cudaStreamBeginCapture(h.cap, cudaStreamCaptureModeThreadLocal));
    const int64_t before = launch_count();
    try {
      body(h.cap);
    } catch (...) {
      cudaStreamEndCapture(h.cap, &g);
      if (g) cudaGraphDestroy(g);
      throw;
    }
    nodes = launch_count() - before;
    count_launch(-nodes);  // captured, not executed
    GBS_CUDA(cudaStreamEndCapture(h.cap, &g));
    cudaError_t e = cudaGraphInstantiate(&ge, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) {
      ge = nullptr;
      throw CudaError{std::string("cudaGraphInstantiate: ") + cudaGetErrorString(e)};
    }
  }
  GBS_CUDA(cudaGraphLaunch(ge, s));
  count_launch(nodes);
}

void run_iteration(Handle& h, bool tr, cudaStream_t s) {
  if (!h.prm.use_graph) {
    bicg_iteration(h, tr, s);
    return;
  }
  replay(h, h.gexec[tr ? 1 : 0], h.gnodes[tr ? 1 : 0], s,
         [&](cudaStream_t cs) { bicg_iteration(h, tr, cs); });
}

gbs_status finish(Handle& h, gbs_info* info, int iters, int repl, double rel, bool conv,
                  std::vector<double>& hist, cudaStream_t s) {
  GBS_CUDA(cudaEventRecord(h.ev1, s));
  GBS_CUDA(cudaEventSynchronize(h.ev1));
  float ms = 0.f;
  cudaEventElapsedTime(&ms, h.ev0, h.ev1);
  if (info) {
    info->iters = iters;
    info->replacements = repl;
    info->converged = conv ? 1 : 0;
    info->rel_res = rel;
    info->ms = ms;
    info->history_len = 0;
    if (info->history && info->history_cap > 0) {
      int nh = std::min<int>(info->history_cap, (int)hist.size());
      std::memcpy(info->history, hist.data(), sizeof(double) * nh);
      info->history_len = nh;
    }
  }
  if (!std::isfinite(rel)) {
    g_err = "NaN or Inf in the residual norm";
    return GBS_ERR_NAN;
  }
  return conv ? GBS_OK : GBS_NOT_CONVERGED;
}

gbs_status solve_bicgstab(Handle& h, const double* b, double* x, bool tr, cudaStream_t s,
                          gbs_info* info) {
  const int64_t n = h.n;
  std::vector<double> hist;
  GBS_CUDA(cudaEventRecord(h.ev0, s));
  GBS_CUDA(cudaMemcpyAsync(h.bi, b, sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
  GBS_CUDA(cudaMemcpyAsync(h.xi, x, sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
  launch_resident(k_dot2, h.red.cap, s, n, h.bi, h.bi, nullptr, h.red, 3, FIN_BB);
  GBS_LAUNCH_CHECK();
  outer(h, tr, SPMV_RESID, h.xi, h.bi, h.r, nullptr, 1, 4, FIN_INIT, true, s);
  GBS_CUDA(cudaMemcpyAsync(h.rhat, h.r, sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
  read_scalars(h, s);
  const double bb = h.sc_host[S_BB];
  if (!std::isfinite(bb)) {
    g_err = "NaN or Inf in b";
    return GBS_ERR_NAN;
  }
  if (bb == 0.0) {
    GBS_CUDA(cudaMemsetAsync(x, 0, sizeof(double) * n, s));
    return finish(h, info, 0, 0, 0.0, true, hist, s);
  }
  const double nb = std::sqrt(bb);
  double rel = std::sqrt(h.sc_host[S_RR]) / nb;
  int it = 0, repl = 0;
  bool conv = rel <= h.prm.tol;
  bool breakdown = false;
  while (!conv && it < h.prm.maxiter) {
    ++it;
    run_iteration(h, tr, s);
    read_scalars(h, s);
    const double* c = h.sc_host;
    if (c[S_BREAK] != 0.0) {
      breakdown = true;
      break;
    }
    double res = std::sqrt(c[S_RR]) / nb;
    if (!std::isfinite(res)) {
      rel = res;
      break;
    }
    hist.push_back(res);
    const bool claim = res <= h.prm.tol;
    if (claim || it % h.prm.replace_every == 0) {
      outer(h, tr, SPMV_RESID, h.xi, h.bi, h.r, h.rhat, 1, 4, FIN_REPLACE, true, s);
      read_scalars(h, s);
      ++repl;
      rel = std::sqrt(h.sc_host[S_RR]) / nb;
      if (rel <= h.prm.tol) {
        conv = true;
        break;
      }
      if (claim) {
        GBS_CUDA(cudaMemcpyAsync(h.rhat, h.r, sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
        ::gbs::launch_k(k_set_restart, 1, 1, 0, s, h.sc);
        GBS_LAUNCH_CHECK();
      }
      if (h.sc_host[S_OMEGA] == 0.0 && !claim) {
        breakdown = true;
        break;
      }
    } else if (c[S_OMEGA] == 0.0 || c[S_RHO] == 0.0) {
      breakdown = true;
      break;
    }
  }
  if (!conv) {
    outer(h, tr, SPMV_RESID, h.xi, h.bi, h.r, nullptr, 1, 4, FIN_RR, true, s);
    read_scalars(h, s);
    rel = std::sqrt(h.sc_host[S_RR]) / nb;
    conv = rel <= h.prm.tol;
  }
  GBS_CUDA(cudaMemcpyAsync(x, h.xi, sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
  gbs_status st = finish(h, info, it, repl, rel, conv, hist, s);
  if (breakdown && !conv && st == GBS_NOT_CONVERGED) {
    g_err = "BiCGStab breakdown";
    return GBS_ERR_BREAKDOWN;
  }
  return st;
}

// SplitMix64 (Steele, Lea & Flood 2014) as a counter-based generator.
inline uint64_t splitmix64(uint64_t counter, uint64_t seed) {
  uint64_t z = seed + (counter + 1) * 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

// s orthonormal shadow vectors (rows): entry (j, i) = u - 1/2, u the top
// 53 bits of splitmix64(j*n + i) over 2^53, then modified Gram-Schmidt.
std::vector<double> idr_shadow_space(int64_t n, int s, uint64_t seed) {
  std::vector<double> P((size_t)s * n);
  for (int64_t c = 0; c < (int64_t)s * n; ++c)
    P[c] = (double)(splitmix64((uint64_t)c, seed) >> 11) * (1.0 / 9007199254740992.0) - 0.5;
  for (int j = 0; j < s; ++j) {
    double* pj = &P[(size_t)j * n];
    for (int i = 0; i < j; ++i) {
      const double* pi = &P[(size_t)i * n];
      double d = 0.0;
      for (int64_t e = 0; e < n; ++e) d += pi[e] * pj[e];
      for (int64_t e = 0; e < n; ++e) pj[e] -= d * pi[e];
    }
    double nrm = 0.0;
    for (int64_t e = 0; e < n; ++e) nrm += pj[e] * pj[e];
    nrm = std::sqrt(nrm);
    for (int64_t e = 0; e < n; ++e) pj[e] /= nrm;
  }
  return P;
}

void givens(double a, double b, double& c, double& sn) {
  if (b == 0.0) {
    c = 1.0;
    sn = 0.0;
    return;
  }
  double r = std::hypot(a, b);
  c = a / r;
  sn = b / r;
}

// The device part of GMRES Arnoldi step j: w = K M^-1 v_j, its classical
// Gram-Schmidt coefficients against v_0 .. v_j (h[0..j], and ||w|| for
// h[j+1]), w -= V h, v_{j+1} = w / ||w||.
void arnoldi_step(Handle& h, int j, bool tr, cudaStream_t s) {
  const int64_t n = h.n;
  const unsigned g = vgrid(n, h.red.cap);
  double* w = h.V + (size_t)(j + 1) * n;
  h.pc->apply(h.V + (size_t)j * n, h.z, tr, s);
  outer(h, tr, SPMV_SET, h.z, nullptr, w, nullptr, 0, 0, FIN_STORE, false, s);
  const int J = j + 1;
  NvtxRange orth("GMRES orthogonalisation");
  launch_resident(k_multidot, h.red.cap, s, n, h.V, J, w, h.hcol, h.red, 5, nullptr);
  GBS_LAUNCH_CHECK();
  launch_resident(k_orth, h.red.cap, s, n, h.V, J, w, h.hcol, nullptr, h.red, 6, nullptr);
  GBS_LAUNCH_CHECK();
  if (h.prm.gmres_reorth != 0) {
    // the second pass: always, or when k_orth flagged a drop of ||w||
    const double* gate = h.prm.gmres_reorth == 2 ? nullptr : h.sc + S_REORTH;
    launch_resident(k_multidot, h.red.cap, s, n, h.V, J, w, h.hcol2, h.red, 7, gate);
    GBS_LAUNCH_CHECK();
    launch_resident(k_orth, h.red.cap, s, n, h.V, J, w, h.hcol2, h.hcol, h.red, 8, gate);
    GBS_LAUNCH_CHECK();
  }
  ::gbs::launch_k(k_normalize, g, 256, 0, s, n, w, h.sc, h.hcol + J);
  GBS_LAUNCH_CHECK();
}

// Arnoldi step j replayed from its own CUDA graph (one per basis size,
// captured the first time a solve reaches it), or launched directly when
// use_graph is 0.
void run_arnoldi(Handle& h, int j, bool tr, cudaStream_t s) {
  if (!h.prm.use_graph) {
    arnoldi_step(h, j, tr, s);
    return;
  }
  auto& ge = h.garn[tr ? 1 : 0];
  auto& nodes = h.garn_nodes[tr ? 1 : 0];
  if ((int)ge.size() < h.m) {
    ge.resize(h.m, nullptr);
    nodes.resize(h.m, 0);
  }
  replay(h, ge[j], nodes[j], s, [&](cudaStream_t cs) { arnoldi_step(h, j, tr, cs); });
}

gbs_status solve_gmres(Handle& h, const double* b, double* x, bool tr, cudaStream_t s,
                       gbs_info* info) {
  const int64_t n = h.n;
  const int m = h.m;
  const unsigned g = vgrid(n, h.red.cap);
  std::vector<double> hist;
  GBS_CUDA(cudaEventRecord(h.ev0, s));
  GBS_CUDA(cudaMemcpyAsync(h.bi, b, sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
  GBS_CUDA(cudaMemcpyAsync(h.xi, x, sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
  launch_resident(k_dot2, h.red.cap, s, n, h.bi, h.bi, nullptr, h.red, 3, FIN_BB);
  GBS_LAUNCH_CHECK();
  read_scalars(h, s);
  const double bb = h.sc_host[S_BB];
  if (!std::isfinite(bb)) {
    g_err = "NaN or Inf in b";
    return GBS_ERR_NAN;
  }
  if (bb == 0.0) {
    GBS_CUDA(cudaMemsetAsync(x, 0, sizeof(double) * n, s));
    return finish(h, info, 0, 0, 0.0, true, hist, s);
  }
  const double nb = std::sqrt(bb);
  std::vector<double> H((size_t)(m + 1) * m), cs(m), sn(m), gv(m + 1), y(m);
  int it = 0, repl = 0;
  double rel = INFINITY;
  bool conv = false;
  for (;;) {
    outer(h, tr, SPMV_RESID, h.xi, h.bi, h.r, nullptr, 1, 4, FIN_RR, true, s);
    read_scalars(h, s);
    ++repl;
    const double beta = std::sqrt(h.sc_host[S_RR]);
    rel = beta / nb;
    if (!std::isfinite(rel)) break;
    if (rel <= h.prm.tol) {
      conv = true;
      break;
    }
    if (it >= h.prm.maxiter) break;
    ::gbs::launch_k(k_scale_rr, g, 256, 0, s, n, h.r, h.V, h.sc);
    GBS_LAUNCH_CHECK();
    std::fill(H.begin(), H.end(), 0.0);
    std::fill(gv.begin(), gv.end(), 0.0);
    gv[0] = beta;
    int j = 0;
    while (j < m && it < h.prm.maxiter) {
      NvtxRange step("GMRES Arnoldi step");
      const int J = j + 1;
      run_arnoldi(h, j, tr, s);
      GBS_CUDA(cudaMemcpyAsync(h.h_host, h.hcol, sizeof(double) * (J + 1), cudaMemcpyDeviceToHost, s));
      GBS_CUDA(cudaStreamSynchronize(s));
      for (int i = 0; i <= J; ++i) H[(size_t)i * m + j] = h.h_host[i];
      for (int i = 0; i < j; ++i) {
        double a = H[(size_t)i * m + j], c = H[(size_t)(i + 1) * m + j];
        H[(size_t)i * m + j] = cs[i] * a + sn[i] * c;
        H[(size_t)(i + 1) * m + j] = -sn[i] * a + cs[i] * c;
      }
      givens(H[(size_t)j * m + j], H[(size_t)(j + 1) * m + j], cs[j], sn[j]);
      H[(size_t)j * m + j] = cs[j] * H[(size_t)j * m + j] + sn[j] * H[(size_t)(j + 1) * m + j];
      H[(size_t)(j + 1) * m + j] = 0.0;
      gv[j + 1] = -sn[j] * gv[j];
      gv[j] = cs[j] * gv[j];
      ++it;
      ++j;
      double est = std::fabs(gv[j]) / nb;
      hist.push_back(est);
      if (!std::isfinite(est) || est <= h.prm.tol) break;
    }
    for (int i = j - 1; i >= 0; --i) {
      double acc = gv[i];
      for (int k = i + 1; k < j; ++k) acc -= H[(size_t)i * m + k] * y[k];
      y[i] = acc / H[(size_t)i * m + i];
    }
    GBS_CUDA(cudaMemcpyAsync(h.ydev, y.data(), sizeof(double) * j, cudaMemcpyHostToDevice, s));
    ::gbs::launch_k(k_combine, g, 256, 0, s, n, h.V, j, h.ydev, h.u);
    GBS_LAUNCH_CHECK();
    h.pc->apply(h.u, h.z, tr, s);
    ::gbs::launch_k(k_axpy, g, 256, 0, s, n, 1.0, h.z, h.xi);
    GBS_LAUNCH_CHECK();
    GBS_CUDA(cudaStreamSynchronize(s));  // y is a pageable host buffer
  }
  GBS_CUDA(cudaMemcpyAsync(x, h.xi, sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
  return finish(h, info, it, repl, rel, conv, hist, s);
}

void need_aligned(const void* p, const char* what) {
  if (reinterpret_cast<uintptr_t>(p) % 16 != 0)
    throw SetupError{std::string(what) + " is not 16-byte aligned"};
}

void need_device(const Handle& h) {
  if (!h.pc) throw SetupError{"hierarchy was built with setup_only (no device data)"};
}

// After gbs_update_values: if a new nonzero fell outside K's CSR pattern,
// K runs in block form from now on.  Reads one device flag (synchronises s).
void settle_k_format(Handle& h, cudaStream_t s) {
  if (!h.k_csr || !h.k_check_pending) return;
  int flag = 0;
  GBS_CUDA(cudaMemcpyAsync(&flag, h.kflag, sizeof(int), cudaMemcpyDeviceToHost, s));
  GBS_CUDA(cudaStreamSynchronize(s));
  h.k_check_pending = false;
  if (flag) {
    h.k_csr = false;
    // captured iterations launch the CSR kernel: capture again
    h.drop_graphs();
  }
}

// Right-preconditioned IDR(s), bi-orthogonal variant (van Gijzen & Sonneveld
// 2011): s inner steps keep the residual orthogonal to the shadow space P,
// then a minimal-residual dimension-reduction step ("maintaining
// convergence" omega, kappa = 0.7).  The small s x s systems live on the
// host; every vector operation is a device kernel.  Iterations count
// applications of K.
gbs_status solve_idrs(Handle& h, const double* b, double* x, bool tr, cudaStream_t s,
                      gbs_info* info) {
  const int64_t n = h.n;
  const int sd = h.prm.idr_s;
  const unsigned g = vgrid(n, h.red.cap);
  std::vector<double> hist;
  GBS_CUDA(cudaEventRecord(h.ev0, s));
  GBS_CUDA(cudaMemcpyAsync(h.bi, b, sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
  GBS_CUDA(cudaMemcpyAsync(h.xi, x, sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
  launch_resident(k_dot2, h.red.cap, s, n, h.bi, h.bi, nullptr, h.red, 3, FIN_BB);
  GBS_LAUNCH_CHECK();
  outer(h, tr, SPMV_RESID, h.xi, h.bi, h.r, nullptr, 1, 4, FIN_RR, true, s);
  read_scalars(h, s);
  const double bb = h.sc_host[S_BB];
  if (!std::isfinite(bb)) {
    g_err = "NaN or Inf in b";
    return GBS_ERR_NAN;
  }
  if (bb == 0.0) {
    GBS_CUDA(cudaMemsetAsync(x, 0, sizeof(double) * n, s));
    return finish(h, info, 0, 0, 0.0, true, hist, s);
  }
  const double nb = std::sqrt(bb);
  double rel = std::sqrt(h.sc_host[S_RR]) / nb;
  int it = 0, repl = 0;
  bool conv = rel <= h.prm.tol, breakdown = false;
  GBS_CUDA(cudaMemsetAsync(h.Gidr, 0, sizeof(double) * n * sd, s));
  GBS_CUDA(cudaMemsetAsync(h.Uidr, 0, sizeof(double) * n * sd, s));
  std::vector<double> Mm((size_t)sd * sd, 0.0), f(sd), c(sd), d(sd), al(sd);
  for (int i = 0; i < sd; ++i) Mm[(size_t)i * sd + i] = 1.0;
  double om = 1.0;
  double cur = rel;  // relative norm of the current residual r
  auto MM = [&](int i, int j) -> double& { return Mm[(size_t)i * sd + j]; };
  auto rownorm = [&]() {
    read_scalars(h, s);
    return std::sqrt(h.sc_host[S_RR]) / nb;
  };
  // confirm a recurrence claim with the true residual (which replaces r)
  auto confirm = [&](double res) {
    hist.push_back(res);
    cur = res;
    if (!(res <= h.prm.tol)) return false;
    outer(h, tr, SPMV_RESID, h.xi, h.bi, h.r, nullptr, 1, 4, FIN_RR, true, s);
    ++repl;
    rel = rownorm();
    cur = rel;
    return rel <= h.prm.tol;
  };
  auto multidot_P = [&](const double* w, std::vector<double>& out) {
    launch_resident(k_multidot, h.red.cap, s, n, h.Pidr, sd, w, h.hcol, h.red, 5, nullptr);
    GBS_LAUNCH_CHECK();
    GBS_CUDA(cudaMemcpyAsync(h.h_host, h.hcol, sizeof(double) * sd, cudaMemcpyDeviceToHost, s));
    GBS_CUDA(cudaStreamSynchronize(s));
    for (int i = 0; i < sd; ++i) out[i] = h.h_host[i];
  };
  while (!conv && it < h.prm.maxiter && !breakdown) {
    multidot_P(h.r, f);
    for (int k = 0; k < sd && !conv && it < h.prm.maxiter; ++k) {
      for (int i = 0; i < sd - k; ++i) {  // lower-triangular Mm[k:, k:] c = f[k:]
        double acc = f[k + i];
        for (int j = 0; j < i; ++j) acc -= MM(k + i, k + j) * c[j];
        c[i] = acc / MM(k + i, k + i);
      }
      Coefs cn{}, cp{};
      for (int i = 0; i < sd - k; ++i) {
        cn.c[i] = -c[i];
        cp.c[i] = c[i];
      }
      double* Gk = h.Gidr + (size_t)k * n;
      double* Uk = h.Uidr + (size_t)k * n;
      ::gbs::launch_k(k_idr_comb, g, 256, 0, s, n, h.v, 1.0, h.r, Gk, sd - k, cn);   // v = r - G[k:] c
      GBS_LAUNCH_CHECK();
      h.pc->apply(h.v, h.ph, tr, s);                                   // v = M^-1 v
      ::gbs::launch_k(k_idr_comb, g, 256, 0, s, n, Uk, om, h.ph, Uk, sd - k, cp);    // U_k = U[k:] c + om v
      GBS_LAUNCH_CHECK();
      outer(h, tr, SPMV_SET, Uk, nullptr, Gk, nullptr, 0, 0, FIN_STORE, false, s);  // G_k = K U_k
      ++it;
      multidot_P(Gk, d);
      for (int i = 0; i < k; ++i) {  // bi-orthogonalise G_k against P[:k]
        double acc = d[i];
        for (int j = 0; j < i; ++j) acc -= MM(i, j) * al[j];
        al[i] = acc / MM(i, i);
      }
      if (k > 0) {
        Coefs ca{};
        for (int i = 0; i < k; ++i) ca.c[i] = -al[i];
        ::gbs::launch_k(k_idr_comb, g, 256, 0, s, n, Gk, 1.0, Gk, h.Gidr, k, ca);
        GBS_LAUNCH_CHECK();
        ::gbs::launch_k(k_idr_comb, g, 256, 0, s, n, Uk, 1.0, Uk, h.Uidr, k, ca);
        GBS_LAUNCH_CHECK();
      }
      for (int i = k; i < sd; ++i) {
        double acc = d[i];
        for (int j = 0; j < k; ++j) acc -= MM(i, j) * al[j];
        MM(i, k) = acc;
      }
      if (MM(k, k) == 0.0) {
        breakdown = true;
        break;
      }
      const double beta = f[k] / MM(k, k);
      launch_resident(k_idr_update, h.red.cap, s, n, h.r, h.xi, Gk, Uk, beta, h.red, 4);
      GBS_LAUNCH_CHECK();
      const double res = rownorm();
      if (!std::isfinite(res)) {
        rel = res;
        breakdown = true;
        break;
      }
      if (confirm(res)) {
        conv = true;
        break;
      }
      for (int i = k + 1; i < sd; ++i) f[i] -= beta * MM(i, k);
    }
    if (conv || breakdown || it >= h.prm.maxiter) break;
    h.pc->apply(h.r, h.ph, tr, s);                                     // v = M^-1 r
    outer(h, tr, SPMV_SET, h.ph, nullptr, h.t, h.r, 1, 1, FIN_STORE, true, s);  // t = K v, t.r, t.t
    ++it;
    read_scalars(h, s);
    const double ts = h.sc_host[S_D0], tt = h.sc_host[S_D1];
    om = tt > 0.0 ? ts / tt : 0.0;
    // ||r|| of the current residual for the kappa rule
    const double rn = cur * nb;
    const double rho = (tt > 0.0 && rn > 0.0) ? std::fabs(ts) / (std::sqrt(tt) * rn) : 0.0;
    if (rho > 0.0 && rho < 0.7) om = om * 0.7 / rho;
    if (om == 0.0 || !std::isfinite(om)) {
      breakdown = true;
      break;
    }
    launch_resident(k_idr_update, h.red.cap, s, n, h.r, h.xi, h.t, h.ph, om, h.red, 4);
    GBS_LAUNCH_CHECK();
    const double res = rownorm();
    if (confirm(res)) conv = true;
    else rel = cur;
  }
  if (!conv) {
    outer(h, tr, SPMV_RESID, h.xi, h.bi, h.r, nullptr, 1, 4, FIN_RR, true, s);
    rel = rownorm();
    conv = rel <= h.prm.tol;
  }
  GBS_CUDA(cudaMemcpyAsync(x, h.xi, sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
  gbs_status st = finish(h, info, it, repl, rel, conv, hist, s);
  if (breakdown && !conv && st == GBS_NOT_CONVERGED) {
    g_err = "IDR(s) breakdown";
    return GBS_ERR_BREAKDOWN;
  }
  return st;
}

gbs_status solve(Handle& h, const double* b, double* x, bool tr, cudaStream_t s, gbs_info* info) {
  need_device(h);
  settle_k_format(h, s);
  if (!b || !x) throw SetupError{"null vector"};
  need_aligned(b, "b");
  need_aligned(x, "x");
  if (tr && !h.prm.enable_adjoint) throw SetupError{"hierarchy was built without enable_adjoint"};
  if (h.prm.krylov == GBS_GMRES) return solve_gmres(h, b, x, tr, s, info);
  if (h.prm.krylov == GBS_IDRS) return solve_idrs(h, b, x, tr, s, info);
  return solve_bicgstab(h, b, x, tr, s, info);
}

void init_device() {
  int nd = 0;
  cudaError_t e = cudaGetDeviceCount(&nd);
  if (e != cudaSuccess || nd == 0)
    throw CudaError{std::string("no CUDA device: ") + cudaGetErrorString(e)};
}

void finish_build(Handle& h, cudaStream_t s) {
  // the scalar block first: pipelined kernels report a timed-out wait in it
  h.sc = h.ar.alloc<double>(S_COUNT);
  GBS_CUDA(cudaMemsetAsync(h.sc, 0, sizeof(double) * S_COUNT, s));
  PrecondOptions o = pc_opts(&h.prm);
  o.err = h.sc + S_ERR;
  if (h.schur) h.pc = make_schur_precond(h.Sh, h.HA, h.HS, o, s);
  else h.pc = make_amg_precond(h.H, o, s);
  alloc_work(h, s);
}

template <class F>
gbs_status guarded(F&& f) {
  try {
    g_err.clear();
    return f();
  } catch (const SetupError& e) {
    g_err = e.msg;
    return GBS_ERR_INVALID;
  } catch (const CudaError& e) {
    g_err = e.msg;
    return e.msg.find("cudaMalloc") != std::string::npos ? GBS_ERR_OOM : GBS_ERR_CUDA;
  } catch (const std::bad_alloc&) {
    g_err = "host allocation failed";
    return GBS_ERR_OOM;
  } catch (const std::exception& e) {
    g_err = e.what();
    return GBS_ERR_INVALID;
  }
}

// One caller-supplied hierarchy (gbs_levels) on the host, checked level by
// level; ILUT factors are this library's own, from each imported operator.
HAmg import_amg(const gbs_levels& L, int B, const gbs_params& prm, int relax) {
  const int nlev = L.nlev;
  if (nlev < 1 || !L.A || !L.Ainv ||
      (nlev > 1 && (!L.P || !L.R || (!L.M && relax != GBS_ILUT))))
    throw SetupError{"bad level arrays"};
  HAmg H;
  H.B = B;
  for (int l = 0; l + 1 < nlev; ++l) {
    HLevel V;
    V.A = from_c(&L.A[l]);
    V.P = from_c(&L.P[l]);
    V.R = from_c(&L.R[l]);
    validate(V.A, true);
    validate(V.P, false);
    validate(V.R, false);
    HBsr An = from_c(&L.A[l + 1]);
    if (V.A.br != B || V.P.br != B || V.R.br != B || An.br != B)
      throw SetupError{"all levels need the same bdim"};
    if (V.P.nbr != V.A.nbr || V.P.nbc != An.nbr || V.R.nbr != An.nbr || V.R.nbc != V.A.nbr)
      throw SetupError{"level " + std::to_string(l) + ": P/R shapes do not match A"};
    if (relax == GBS_ILUT) {
      V.ilu = ilut(to_scalar_csr(V.A), prm.ilut_p, prm.ilut_tau);
    } else {
      if (!L.M[l]) throw SetupError{"null smoother blocks"};
      V.M.assign(L.M[l], L.M[l] + (size_t)V.A.nbr * B * B);
    }
    H.levels.push_back(std::move(V));
  }
  H.Ac = from_c(&L.A[nlev - 1]);
  validate(H.Ac, true);
  if (H.Ac.br != B) throw SetupError{"all levels need the same bdim"};
  const size_t nc = (size_t)H.Ac.nbr * B;
  if (nc > 8192) throw SetupError{"coarsest level too large for a dense inverse"};
  H.Ainv.assign(L.Ainv, L.Ainv + nc * nc);
  return H;
}

}  // namespace

std::unique_ptr<DevPrecond> make_amg_precond(const HAmg& H, const PrecondOptions& o,
                                             cudaStream_t s) {
  switch (o.precision) {
    case 1: return make_amg_fp32(H, o, s);
    case 2: return make_amg_bf16(H, o, s);
    default: return make_amg_fp64(H, o, s);
  }
}
std::unique_ptr<DevPrecond> make_schur_precond(const HSchur& Sc, const HAmg& HA, const HAmg& HS,
                                               const PrecondOptions& o, cudaStream_t s) {
  switch (o.precision) {
    case 1: return make_schur_fp32(Sc, HA, HS, o, s);
    case 2: return make_schur_bf16(Sc, HA, HS, o, s);
    default: return make_schur_fp64(Sc, HA, HS, o, s);
  }
}

}  // namespace gbs

using namespace gbs;

struct gbs_hierarchy {
  Handle h;
};

extern "C" {

const char* gbs_last_error(void) { return g_err.c_str(); }

int64_t gbs_kernel_launches(void) { return launch_count(); }

gbs_status gbs_params_default(gbs_params* p) {
  if (!p) {
    g_err = "null params";
    return GBS_ERR_INVALID;
  }
  std::memset(p, 0, sizeof(*p));
  p->precond = GBS_PC_AMG;
  p->krylov = GBS_BICGSTAB;
  p->restart = 30;
  p->tol = 1e-8;
  p->maxiter = 1000;
  p->replace_every = 50;
  p->precision = GBS_FP64;
  p->eps_strong = 0.08;
  p->coarse_enough = 1000;
  p->max_levels = 10;
  p->npre = 1;
  p->npost = 1;
  p->relax = GBS_SPAI0;
  p->relax_p = GBS_SPAI0;
  p->jacobi_omega = 0.72;
  p->smooth_P = 1;
  p->power_iters = 20;
  p->nvel = 3;
  p->use_graph = 1;
  p->enable_adjoint = 1;
  p->setup_only = 0;
  p->level_format = 0;
  p->schur_p = 0;
  p->schur_order = 0;
  p->idr_s = 5;
  p->idr_seed = 0;
  p->ilut_p = 2.0;
  p->ilut_tau = 1e-2;
  p->ilut_sweeps = 2;
  p->ilut_omega = 1.0;
  p->gmres_reorth = 0;
  p->wait_log2 = 31;
  p->iso_blocks = 1;
  return GBS_OK;
}

gbs_status gbs_build_hierarchy(const gbs_bsr* A, const gbs_params* params, void* stream,
                               gbs_hierarchy** out) {
  return guarded([&]() -> gbs_status {
    if (!out) throw SetupError{"null output handle"};
    *out = nullptr;
    check_params(params);
    HBsr K = from_c(A);
    validate(K, true);
    if (!params->setup_only) init_device();
    auto hh = std::make_unique<gbs_hierarchy>();
    Handle& h = hh->h;
    h.prm = *params;
    h.B = K.br;
    h.n = (int64_t)K.nbr * K.br;
    if (params->precond == GBS_PC_SCHUR) {
      h.schur = true;
      if (K.br != params->nvel + 1) throw SetupError{"Schur needs bdim = nvel + 1"};
      h.Sh = schur_split(K, params->nvel);
      h.HA = build_amg(h.Sh.A, amg_prm(params, params->relax));
      if (params->schur_p == 1)
        h.Sh.MS = params->relax_p == GBS_SPAI0 ? spai0(h.Sh.S) : jacobi(h.Sh.S, params->jacobi_omega);
      else
        h.HS = build_amg(h.Sh.S, amg_prm(params, params->relax_p));
    } else {
      h.H = build_amg(K, amg_prm(params, params->relax));
    }
    h.Kh = std::move(K);
    if (!params->setup_only) finish_build(h, S(stream));
    *out = hh.release();
    return GBS_OK;
  });
}

gbs_status gbs_import_hierarchy(const gbs_bsr* A, const gbs_bsr* P, const gbs_bsr* R,
                                const double* const* M, const double* Ainv, int32_t nlev,
                                const gbs_params* params, void* stream, gbs_hierarchy** out) {
  return guarded([&]() -> gbs_status {
    if (!out) throw SetupError{"null output handle"};
    *out = nullptr;
    check_params(params);
    if (params->precond != GBS_PC_AMG)
      throw SetupError{"gbs_import_hierarchy takes the AMG preconditioner (Schur: gbs_import_schur)"};
    if (nlev < 1 || !A) throw SetupError{"bad level arrays"};
    if (params->setup_only) throw SetupError{"import needs device upload (setup_only = 0)"};
    init_device();
    auto hh = std::make_unique<gbs_hierarchy>();
    Handle& h = hh->h;
    h.prm = *params;
    HBsr K = from_c(&A[0]);
    validate(K, true);
    h.B = K.br;
    h.n = (int64_t)K.nbr * K.br;
    const gbs_levels L{A, P, R, M, Ainv, nlev};
    h.H = import_amg(L, K.br, *params, params->relax);
    h.Kh = std::move(K);
    finish_build(h, S(stream));
    *out = hh.release();
    return GBS_OK;
  });
}

gbs_status gbs_import_schur(const gbs_bsr* Kc, const gbs_levels* vel, const gbs_levels* pres,
                            const double* pres_smoother, const gbs_params* params, void* stream,
                            gbs_hierarchy** out) {
  return guarded([&]() -> gbs_status {
    if (!out) throw SetupError{"null output handle"};
    *out = nullptr;
    check_params(params);
    if (params->precond != GBS_PC_SCHUR) throw SetupError{"gbs_import_schur needs GBS_PC_SCHUR"};
    if (params->setup_only) throw SetupError{"import needs device upload (setup_only = 0)"};
    if (!vel) throw SetupError{"null velocity hierarchy"};
    if (params->schur_p == 0 && !pres) throw SetupError{"null pressure hierarchy (schur_p = 0)"};
    if (params->schur_p == 1 && !pres_smoother)
      throw SetupError{"null pressure smoother (schur_p = 1)"};
    HBsr K = from_c(Kc);
    validate(K, true);
    if (K.br != params->nvel + 1) throw SetupError{"Schur needs bdim = nvel + 1"};
    init_device();
    auto hh = std::make_unique<gbs_hierarchy>();
    Handle& h = hh->h;
    h.prm = *params;
    h.schur = true;
    h.B = K.br;
    h.n = (int64_t)K.nbr * K.br;
    h.Sh = schur_split(K, params->nvel);
    h.HA = import_amg(*vel, params->nvel, *params, params->relax);
    const HBsr& A0 = h.HA.levels.empty() ? h.HA.Ac : h.HA.levels[0].A;
    if (A0.nbr != K.nbr || A0.nbc != K.nbc)
      throw SetupError{"velocity level 0 does not match K's block rows"};
    if (params->schur_p == 1) {
      h.Sh.MS.assign(pres_smoother, pres_smoother + K.nbr);
    } else {
      h.HS = import_amg(*pres, 1, *params, params->relax_p);
      const HBsr& S0 = h.HS.levels.empty() ? h.HS.Ac : h.HS.levels[0].A;
      if (S0.nbr != K.nbr || S0.nbc != K.nbc)
        throw SetupError{"pressure level 0 does not match K's block rows"};
    }
    h.Kh = std::move(K);
    finish_build(h, S(stream));
    *out = hh.release();
    return GBS_OK;
  });
}

gbs_status gbs_solve(gbs_hierarchy* hh, const double* b, double* x, void* stream, gbs_info* info) {
  return guarded([&]() -> gbs_status {
    if (!hh) throw SetupError{"null handle"};
    return solve(hh->h, b, x, false, S(stream), info);
  });
}

gbs_status gbs_solve_adjoint(gbs_hierarchy* hh, const double* g, double* lam, void* stream,
                             gbs_info* info) {
  return guarded([&]() -> gbs_status {
    if (!hh) throw SetupError{"null handle"};
    return solve(hh->h, g, lam, true, S(stream), info);
  });
}

gbs_status gbs_sampled_outer(const gbs_hierarchy* hh, const double* lam, const double* x,
                             double alpha, double* grad, void* stream) {
  return guarded([&]() -> gbs_status {
    if (!hh || !lam || !x || !grad) throw SetupError{"null argument"};
    const Handle& h = hh->h;
    need_device(h);
    need_aligned(lam, "lam");
    need_aligned(x, "x");
    need_aligned(grad, "grad");
    cudaStream_t s = S(stream);
#define GBS_SO(BB)                                                                    \
  ::gbs::launch_k(k_sampled_outer<BB>, grid_for(row_threads<BB>(h.K.nbr)), 256, 0, s, h.K, lam, x, \
                                                                         alpha, grad)
    switch (h.B) {
      case 1: GBS_SO(1); break;
      case 2: GBS_SO(2); break;
      case 3: GBS_SO(3); break;
      case 4: GBS_SO(4); break;
    }
#undef GBS_SO
    GBS_LAUNCH_CHECK();
    return GBS_OK;
  });
}

gbs_status gbs_update_values(gbs_hierarchy* hh, const double* vals, void* stream) {
  return guarded([&]() -> gbs_status {
    if (!hh || !vals) throw SetupError{"null argument"};
    Handle& h = hh->h;
    need_device(h);
    need_aligned(vals, "vals");
    cudaStream_t s = S(stream);
    GBS_CUDA(cudaMemcpyAsync(h.Kval, vals, sizeof(double) * h.Kh.val.size(),
                             cudaMemcpyDeviceToDevice, s));
    if (h.k_csr) {
      if (h.k_sell)
        ::gbs::launch_k(k_gather_sell, vgrid(h.kmap_n, h.red.cap), 256, 0, s, h.kmap_n, h.kmap, h.Kval, h.kcval);
      else
        ::gbs::launch_k(k_gather_vals, vgrid((int64_t)h.Kh.val.size(), h.red.cap), 256, 0, s, h.kmap_n, h.kmap, h.Kval, h.kcval);
      GBS_LAUNCH_CHECK();
      ::gbs::launch_k(k_check_outside, vgrid((int64_t)h.Kh.val.size(), h.red.cap), 256, 0, s, (int64_t)h.Kh.val.size(), h.kzero,
                                                                      h.Kval, h.kflag);
      GBS_LAUNCH_CHECK();
      h.k_check_pending = true;
    }
    return GBS_OK;
  });
}

gbs_status gbs_spmv(const gbs_hierarchy* hh, const double* x, double* y, int32_t transpose,
                    void* stream) {
  return guarded([&]() -> gbs_status {
    if (!hh || !x || !y) throw SetupError{"null argument"};
    Handle& h = const_cast<gbs_hierarchy*>(hh)->h;
    need_device(h);
    settle_k_format(h, S(stream));
    need_aligned(x, "x");
    need_aligned(y, "y");
    if (transpose && !h.K.tmap) throw SetupError{"built without enable_adjoint"};
    if (x == y) throw SetupError{"x and y must not alias"};
    outer(h, transpose != 0, SPMV_SET, x, nullptr, y, nullptr, 0, 0, FIN_STORE, false, S(stream));
    return GBS_OK;
  });
}

gbs_status gbs_apply_precond(gbs_hierarchy* hh, const double* r, double* z, int32_t transpose,
                             void* stream) {
  return guarded([&]() -> gbs_status {
    if (!hh || !r || !z) throw SetupError{"null argument"};
    Handle& h = hh->h;
    need_device(h);
    need_aligned(r, "r");
    need_aligned(z, "z");
    if (r == z) throw SetupError{"r and z must not alias"};
    if (transpose && !h.prm.enable_adjoint) throw SetupError{"built without enable_adjoint"};
    h.pc->apply(r, z, transpose != 0, S(stream));
    return GBS_OK;
  });
}

gbs_status gbs_hierarchy_info(const gbs_hierarchy* hh, int32_t which, int32_t* nlevels,
                              int32_t* n_brows, int64_t* nnzb, int32_t cap, int64_t* bytes) {
  return guarded([&]() -> gbs_status {
    if (!hh || !nlevels) throw SetupError{"null argument"};
    const Handle& h = hh->h;
    if (which < 0 || which > 1 || (which == 1 && !h.schur)) throw SetupError{"bad hierarchy id"};
    if (which == 1 && h.prm.schur_p == 1)
      throw SetupError{"the pressure solve is one smoother application (no pressure AMG)"};
    const HAmg& H = h.schur ? (which == 0 ? h.HA : h.HS) : h.H;
    const int nl = (int)H.levels.size() + 1;
    *nlevels = nl;
    for (int l = 0; l < nl && l < cap; ++l) {
      const HBsr& A = l + 1 == nl ? H.Ac : H.levels[l].A;
      if (n_brows) n_brows[l] = A.nbr;
      if (nnzb) nnzb[l] = A.nnzb();
    }
    if (bytes) *bytes = h.pc ? h.pc->bytes() + h.ar.bytes : 0;
    return GBS_OK;
  });
}

gbs_status gbs_level_apply(gbs_hierarchy* hh, int32_t which, int32_t level, int32_t op,
                           const void* x, const void* f, void* y, void* stream) {
  return guarded([&]() -> gbs_status {
    if (!hh || !x || !f || !y) throw SetupError{"null argument"};
    Handle& h = hh->h;
    need_device(h);
    if (which < 0 || which > 1 || (which == 1 && !h.schur)) throw SetupError{"bad hierarchy id"};
    if (level < 0 || level + 1 >= h.pc->nlevels(which))
      throw SetupError{"level must be below the coarsest"};
    if (x == y || f == y) throw SetupError{"y must not alias x or f"};
    need_aligned(x, "x");
    need_aligned(f, "f");
    need_aligned(y, "y");
    h.pc->level_op(which, level, op, x, f, y, S(stream));
    return GBS_OK;
  });
}

gbs_status gbs_level_format(const gbs_hierarchy* hh, int32_t which, int32_t level,
                            int32_t* format) {
  return guarded([&]() -> gbs_status {
    if (!hh || !format) throw SetupError{"null argument"};
    const Handle& h = hh->h;
    need_device(h);
    if (which < 0 || which > 1 || (which == 1 && !h.schur)) throw SetupError{"bad hierarchy id"};
    if (level < 0 || level + 1 >= h.pc->nlevels(which))
      throw SetupError{"level must be below the coarsest"};
    *format = h.pc->level_layout(which, level);
    return GBS_OK;
  });
}

gbs_status gbs_outer_format(const gbs_hierarchy* hh, int32_t* format, int64_t* stored) {
  return guarded([&]() -> gbs_status {
    if (!hh || !format || !stored) throw SetupError{"null argument"};
    const Handle& h = hh->h;
    if (h.k_csr) {
      *format = h.k_sell ? 2 : 1;
      *stored = h.kmap_n;
    } else {
      *format = 0;
      *stored = (int64_t)h.Kh.val.size();
    }
    return GBS_OK;
  });
}

gbs_status gbs_precond_bytes(const gbs_hierarchy* hh, double* bytes) {
  return guarded([&]() -> gbs_status {
    if (!hh || !bytes) throw SetupError{"null argument"};
    need_device(hh->h);
    *bytes = hh->h.pc->bytes_per_apply();
    return GBS_OK;
  });
}

gbs_status gbs_export_level(const gbs_hierarchy* hh, int32_t which, int32_t level, int32_t part,
                            int32_t* n_brows, int32_t* n_bcols, int64_t* nnzb, int32_t* row_ptr,
                            int32_t* col_idx, double* vals) {
  return guarded([&]() -> gbs_status {
    if (!hh || !n_brows || !n_bcols || !nnzb) throw SetupError{"null argument"};
    const Handle& h = hh->h;
    if (which < 0 || which > 1 || (which == 1 && !h.schur)) throw SetupError{"bad hierarchy id"};
    if (which == 1 && h.prm.schur_p == 1)
      throw SetupError{"the pressure solve is one smoother application (no pressure AMG)"};
    const HAmg& H = h.schur ? (which == 0 ? h.HA : h.HS) : h.H;
    const int nl = (int)H.levels.size() + 1;
    if (level < 0 || level >= nl) throw SetupError{"bad level"};
    const bool coarsest = level == nl - 1;
    const HBsr* M = nullptr;
    if (part == 0) M = coarsest ? &H.Ac : &H.levels[level].A;
    else if (part == 1 || part == 2) {
      if (coarsest) throw SetupError{"the coarsest level has no P/R"};
      M = part == 1 ? &H.levels[level].P : &H.levels[level].R;
    }
    if (M) {
      *n_brows = M->nbr;
      *n_bcols = M->nbc;
      *nnzb = M->nnzb();
      if (row_ptr) std::memcpy(row_ptr, M->ptr.data(), sizeof(int32_t) * M->ptr.size());
      if (col_idx) std::memcpy(col_idx, M->col.data(), sizeof(int32_t) * M->col.size());
      if (vals) std::memcpy(vals, M->val.data(), sizeof(double) * M->val.size());
      return GBS_OK;
    }
    if (part == 3 || part == 4) {
      if (coarsest) throw SetupError{"the coarsest level has no smoother/aggregates"};
      const HLevel& L = H.levels[level];
      *n_brows = L.A.nbr;
      *n_bcols = part == 3 ? H.B : 1;
      *nnzb = 0;
      if (part == 3 && vals) std::memcpy(vals, L.M.data(), sizeof(double) * L.M.size());
      if (part == 4 && col_idx) std::memcpy(col_idx, L.agg.data(), sizeof(int32_t) * L.agg.size());
      return GBS_OK;
    }
    if (part >= 6 && part <= 8) {
      if (coarsest) throw SetupError{"the coarsest level has no smoother"};
      const HIlu& F = H.levels[level].ilu;
      if (F.d.empty()) throw SetupError{"the level is not relaxed by ILUT"};
      const int n = (int)F.d.size();
      *n_brows = n;
      *n_bcols = part == 8 ? 1 : n;
      if (part == 8) {
        *nnzb = 0;
        if (vals) std::memcpy(vals, F.d.data(), sizeof(double) * F.d.size());
        return GBS_OK;
      }
      const HCsr& C = part == 6 ? F.L : F.U;
      *nnzb = (int64_t)C.col.size();
      if (row_ptr) std::memcpy(row_ptr, C.ptr.data(), sizeof(int32_t) * C.ptr.size());
      if (col_idx) std::memcpy(col_idx, C.col.data(), sizeof(int32_t) * C.col.size());
      if (vals) std::memcpy(vals, C.val.data(), sizeof(double) * C.val.size());
      return GBS_OK;
    }
    if (part == 5) {
      if (!coarsest) throw SetupError{"the dense inverse lives on the coarsest level"};
      *n_brows = H.Ac.nbr * H.B;
      *n_bcols = H.Ac.nbr * H.B;
      *nnzb = 0;
      if (vals) std::memcpy(vals, H.Ainv.data(), sizeof(double) * H.Ainv.size());
      return GBS_OK;
    }
    throw SetupError{"bad part"};
  });
}

gbs_status gbs_destroy(gbs_hierarchy* hh) {
  return guarded([&]() -> gbs_status {
    if (!hh) return GBS_OK;
    if (hh->h.pc) cudaDeviceSynchronize();
    delete hh;
    return GBS_OK;
  });
}

}  // extern "C"
