"""Smoothed-aggregation AMG with SPAI0 relaxation (FP64 oracle).

The paper composes its preconditioner as AMG with smoothed-aggregation
coarsening and the SPAI0 smoother (Section 2.1, Listing "composition";
the strong-coupling threshold eps_strong is set in Listing "params").
It names these components but leaves their inner steps to the AMG
literature; the readings used here (each one a choice where the paper is
silent) are:

1. Strength: block nodes i != j are strongly coupled iff
       ||A_ij||_F^2 > eps_l^2 ||A_ii||_F ||A_jj||_F,  eps_l = eps * 0.5^l,
   with ||.||_F^2 accumulated over the block in row-major order.
2. Aggregation, deterministic greedy:
   pass 1 visits nodes in ascending order; a node whose strong
   neighbours are all unaggregated becomes a root and forms an aggregate
   with them (no strong neighbours -> singleton);
   pass 2 attaches each remaining node to the pass-1 aggregate of its
   strongest strongly-coupled neighbour (ties -> smaller aggregate id).
3. Tentative prolongator: identity block at (i, aggregate(i)).
4. Smoothed prolongator P = (I - omega D^-1 A) P_tent, D = block
   diagonal of A, omega = (4/3) / rho with rho the spectral radius of
   D^-1 A estimated by 20 power iterations from the deterministic start
   x_i = frac(0.6180339887498949 i) - 0.5 (the infinity-norm bound is
   ~40x too large on the saddle-point blocks, which turns smoothing off).
5. R = P^T, A_{l+1} = R A_l P (Galerkin).  Coarsening stops when the
   next level would have <= coarse_enough scalar unknowns, or at
   max_levels, or when aggregation no longer shrinks the level; the
   coarsest matrix is inverted densely (LU with partial pivoting).
6. SPAI0 (Broker & Grote, Section 4's reference for the smoother):
   scalar m_i = a_ii / sum_j a_ij^2; for blocks the minimiser of
   ||I - M A||_F over block-diagonal M, M_i = A_ii^T (sum_j A_ij A_ij^T)^-1.
   Damped Jacobi (PETSc's choice in Section 4) is M_i = omega A_ii^-1.
   ILUT (the paper's velocity smoother, Listings V2-V4) is in ilut.py: there
   the step x += S (f - A x) uses the approximate (LU)^-1 of that file in
   place of the block-diagonal M.
7. V-cycle: 1 pre-sweep from a zero guess (x = M f), residual,
   restriction, recursive coarse correction, prolongation, 1 post-sweep
   x += M (f - A x); the transposed cycle uses A^T, M^T, the same P and
   R (R = P^T), the transposed coarse inverse and swapped sweep counts.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np
import scipy.sparse as sp

from . import ilut as ilut_mod
from .bsr import Bsr, from_scipy, spmv
from .precision import round_to


@dataclass
class AmgParams:
    eps_strong: float = 0.08
    coarse_enough: int = 1000        # scalar unknowns on the coarsest level
    max_levels: int = 10
    npre: int = 1
    npost: int = 1
    relax: str = "spai0"             # "spai0" | "jacobi" | "ilut"
    jacobi_omega: float = 0.72
    smooth_P: bool = True
    ilut_p: float = 2.0              # ILUT fill factor (ilut.py reading 1)
    ilut_tau: float = 1e-2           # ILUT drop tolerance
    ilut_sweeps: int = 2             # Jacobi sweeps per triangular solve
    ilut_omega: float = 1.0          # ILUT relaxation damping


@dataclass
class Level:
    A: Bsr
    M: np.ndarray        # [n_brows, B, B] smoother blocks (SPAI0 / Jacobi)
    P: Bsr               # n x n_c
    R: Bsr               # n_c x n
    agg: np.ndarray      # aggregate id of every block node
    S: object = None     # ilut.Ilu when the level is relaxed by ILUT


@dataclass
class Hierarchy:
    levels: list
    A_coarse: Bsr
    Ainv_coarse: np.ndarray
    params: AmgParams
    omegas: list = field(default_factory=list)

    @property
    def nlevels(self) -> int:
        return len(self.levels) + 1

    def A(self, l: int) -> Bsr:
        return self.levels[l].A if l < len(self.levels) else self.A_coarse


def block_fro2(data: np.ndarray) -> np.ndarray:
    """Squared Frobenius norm of each block, summed in row-major order."""
    s = np.zeros(data.shape[0])
    for a in range(data.shape[1]):
        for c in range(data.shape[2]):
            s = s + data[:, a, c] * data[:, a, c]
    return s


def diag_positions(A: Bsr) -> np.ndarray:
    rows = A.block_rows()
    mask = A.indices == rows
    pos = np.full(A.n_brows, -1, dtype=np.int64)
    pos[rows[mask]] = np.nonzero(mask)[0]
    if (pos < 0).any():
        raise ValueError("a block row has no stored diagonal block")
    return pos


def strong_couplings(A: Bsr, eps: float):
    """Boolean mask over stored blocks: True where the coupling is strong."""
    s = block_fro2(A.data)
    dpos = diag_positions(A)
    d = np.sqrt(s[dpos])
    rows = A.block_rows()
    cols = A.indices
    thr = (eps * eps) * d[rows]
    strong = (s > thr * d[cols]) & (rows != cols)
    return strong, s


def aggregate(A: Bsr, eps: float):
    """Greedy two-pass aggregation (reading 2 above).  Returns (agg, n_agg)."""
    strong, s = strong_couplings(A, eps)
    n = A.n_brows
    indptr = A.indptr.tolist()
    cols = A.indices.tolist()
    strong_l = strong.tolist()
    s_l = s.tolist()
    nbrs = []
    for i in range(n):
        nbrs.append([(cols[k], s_l[k]) for k in range(indptr[i], indptr[i + 1]) if strong_l[k]])
    agg = [-1] * n
    n_agg = 0
    # pass 1: roots with all strong neighbours still free
    for i in range(n):
        if agg[i] != -1:
            continue
        if all(agg[j] == -1 for j, _ in nbrs[i]):
            agg[i] = n_agg
            for j, _ in nbrs[i]:
                agg[j] = n_agg
            n_agg += 1
    agg1 = list(agg)
    # pass 2: attach the rest to the strongest aggregated neighbour
    for i in range(n):
        if agg[i] != -1:
            continue
        best = None
        for j, sij in nbrs[i]:
            a = agg1[j]
            if a < 0:
                continue
            if best is None or sij > best[0] or (sij == best[0] and a < best[1]):
                best = (sij, a)
        assert best is not None, "pass 1 leaves every free node next to an aggregate"
        agg[i] = best[1]
    return np.array(agg, dtype=np.int64), n_agg


def tentative_P(agg: np.ndarray, n_agg: int, B: int) -> Bsr:
    n = len(agg)
    data = np.broadcast_to(np.eye(B), (n, B, B)).copy()
    return Bsr(np.arange(n + 1, dtype=np.int64), agg.astype(np.int64), data, n_agg)


def block_diag_inv(A: Bsr) -> np.ndarray:
    D = A.data[diag_positions(A)]
    if np.any(np.abs(np.linalg.det(D)) == 0.0):
        raise ValueError("singular diagonal block")
    return np.linalg.inv(D)


POWER_ITERS = 20


def power_start(n: int) -> np.ndarray:
    """Deterministic start vector: x_i = frac(i * 0.6180339887498949) - 0.5."""
    i = np.arange(n, dtype=np.float64)
    return np.mod(i * 0.6180339887498949, 1.0) - 0.5


def spectral_radius(A: Bsr, iters: int) -> float:
    """Power-iteration estimate of rho(A): ||A x_k|| / ||x_k||, x_{k+1} = A x_k / ||A x_k||."""
    x = power_start(A.shape[0])
    x = x / np.linalg.norm(x)
    rho = 0.0
    for _ in range(iters):
        y = spmv(A, x)
        rho = np.linalg.norm(y)
        x = y / rho
    return float(rho)


def smoothed_P(A: Bsr, Pt: Bsr):
    """P = (I - omega D^-1 A) P_tent with omega = (4/3)/rho(D^-1 A)."""
    Dinv = block_diag_inv(A)
    rows = A.block_rows()
    DinvA_data = np.einsum("kab,kbc->kac", Dinv[rows], A.data)
    DinvA = Bsr(A.indptr, A.indices, DinvA_data, A.n_bcols)
    rho = spectral_radius(DinvA, POWER_ITERS)
    omega = (4.0 / 3.0) / rho
    S = DinvA.csr() @ Pt.csr()
    P = Pt.csr() - omega * S
    return from_scipy(P, A.br, A.bc), omega


def galerkin(R: Bsr, A: Bsr, P: Bsr) -> Bsr:
    return from_scipy(R.csr() @ A.csr() @ P.csr(), A.br, A.bc)


def spai0(A: Bsr) -> np.ndarray:
    """Block SPAI0: M_i = A_ii^T (sum_j A_ij A_ij^T)^-1 (scalar: a_ii / sum a_ij^2)."""
    rows = A.block_rows()
    B = A.br
    G = np.zeros((A.n_brows, B, B))
    np.add.at(G, rows, np.einsum("kab,kcb->kac", A.data, A.data))
    Aii = A.data[diag_positions(A)]
    if np.any(np.linalg.det(G) == 0.0):
        raise ValueError("SPAI0 Gram matrix is singular (zero row)")
    return np.einsum("iba,ibc->iac", Aii, np.linalg.inv(G))


def jacobi(A: Bsr, omega: float) -> np.ndarray:
    return omega * block_diag_inv(A)


def build_hierarchy(A: Bsr, prm: AmgParams | None = None) -> Hierarchy:
    prm = prm or AmgParams()
    B = A.br
    levels = []
    omegas = []
    l = 0
    while A.n_brows * B > prm.coarse_enough and l < prm.max_levels - 1:
        agg, n_agg = aggregate(A, prm.eps_strong * 0.5 ** l)
        if n_agg >= A.n_brows:
            break
        Pt = tentative_P(agg, n_agg, B)
        if prm.smooth_P:
            P, omega = smoothed_P(A, Pt)
        else:
            P, omega = Pt, 0.0
        R = from_scipy(P.csr().T, B, B)
        Ac = galerkin(R, A, P)
        S = None
        if prm.relax == "ilut":
            M = np.zeros((A.n_brows, B, B))
            As = sp.csr_matrix(A.scipy())
            As.eliminate_zeros()
            S = ilut_mod.build(As, prm.ilut_p, prm.ilut_tau, prm.ilut_sweeps, prm.ilut_omega)
        elif prm.relax == "spai0":
            M = spai0(A)
        else:
            M = jacobi(A, prm.jacobi_omega)
        levels.append(Level(A=A, M=M, P=P, R=R, agg=agg, S=S))
        omegas.append(omega)
        A = Ac
        l += 1
    Ainv = np.linalg.inv(A.dense())
    return Hierarchy(levels=levels, A_coarse=A, Ainv_coarse=Ainv, params=prm, omegas=omegas)


def apply_M(M: np.ndarray, v: np.ndarray, transpose: bool = False) -> np.ndarray:
    B = M.shape[1]
    vb = v.reshape(-1, B)
    if transpose:
        return np.einsum("iba,ib->ia", M, vb).reshape(-1)
    return np.einsum("iab,ib->ia", M, vb).reshape(-1)


def smooth(lev: Level, v: np.ndarray, transpose: bool = False) -> np.ndarray:
    """The level's relaxation operator applied to v: M v, or S v for ILUT."""
    if lev.S is not None:
        return lev.S.apply(v, transpose)
    return apply_M(lev.M, v, transpose)


def vcycle(H: Hierarchy, f: np.ndarray, l: int = 0, transpose: bool = False) -> np.ndarray:
    """One V-cycle x = V(f) from a zero initial guess (reading 7)."""
    if l == len(H.levels):
        Ainv = H.Ainv_coarse.T if transpose else H.Ainv_coarse
        return Ainv @ f
    lev = H.levels[l]
    A = lev.A.scipy()
    if transpose:
        A = A.T
    npre, npost = H.params.npre, H.params.npost
    if transpose:
        npre, npost = npost, npre
    x = np.zeros_like(f)
    for it in range(npre):
        if it == 0:
            x = smooth(lev, f, transpose)
        else:
            x = x + smooth(lev, f - A @ x, transpose)
    r = f - A @ x
    fc = spmv(lev.R, r)
    ec = vcycle(H, fc, l + 1, transpose)
    x = x + spmv(lev.P, ec)
    for it in range(npost):
        x = x + smooth(lev, f - A @ x, transpose)
    return x


def vcycle_dense(H: Hierarchy, transpose: bool = False) -> np.ndarray:
    """The V-cycle as a dense matrix (columns = images of unit vectors)."""
    n = H.A(0).shape[0]
    cols = [vcycle(H, e, 0, transpose) for e in np.eye(n)]
    return np.array(cols).T


def _rounded(A: Bsr, fmt: str) -> Bsr:
    return Bsr(A.indptr, A.indices, round_to(A.data, fmt), A.n_bcols)


def cast_values(H: Hierarchy, fmt: str) -> Hierarchy:
    """The hierarchy as a mixed-precision form stores it (Section 4's
    single-precision preconditioner, Listing V4, and its BF16 extension):
    A_l, P_l, R_l and the smoother blocks M_l rounded to `fmt` ("fp32" or
    "bf16"), the dense coarse inverse rounded to FP32 in both forms.  The
    result is an ordinary FP64 hierarchy holding those rounded values, so
    vcycle() on it differs from the GPU's mixed form only by the GPU's
    FP32 accumulation.  ILUT levels are not modelled."""
    levels = []
    for lev in H.levels:
        if lev.S is not None:
            raise ValueError("cast_values: ILUT levels are not modelled")
        levels.append(Level(A=_rounded(lev.A, fmt), M=round_to(lev.M, fmt),
                            P=_rounded(lev.P, fmt), R=_rounded(lev.R, fmt), agg=lev.agg))
    return Hierarchy(levels=levels, A_coarse=_rounded(H.A_coarse, fmt),
                     Ainv_coarse=round_to(H.Ainv_coarse, "fp32"), params=H.params,
                     omegas=list(H.omegas))
