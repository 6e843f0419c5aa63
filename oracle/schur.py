"""Schur pressure-correction preconditioner (FP64 oracle).

Section 4, Eq. SchurPC: for the saddle-point system [A G; D C] the
preconditioning step solves S p = r_p - D A^-1 r_u and then
A u = r_u - G p, each inner solve replaced by one application of a
preconditioner (the "preonly" reading: the overall preconditioner stays
linear).  Eq. SchurApprox gives the pressure operator
S_hat = C - diag(D diag(A)^-1 G), where diag(A) is the scalar diagonal
of the velocity block.  The paper writes B_c and B_c^T for D and G; on
the finite-difference stand-in D = -G^T.

Read literally, Eq. SchurPC applies the velocity preconditioner twice:
u* = V_A(r_u), p = V_S(r_p - D u*), u = V_A(r_u - G p) ("full").
Variants (the paper's own configurations):
* pressure solve = one application of the pressure smoother on S_hat
  (Section 4: one SPAI0 application as the approximation to S^-1, Listing
  V2's as_preconditioner + preonly) instead of an AMG V-cycle;
* "lower" ordering (the LOWER factorisation of the PETSc configuration in
  Section 4): u = V_A(r_u), p = V_S(r_p - D u), one velocity solve.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np
import scipy.sparse as sp

from . import amg
from .bsr import Bsr, from_scipy
from .precision import round_to


@dataclass
class SchurSplit:
    A: Bsr      # velocity block, nvel x nvel blocks
    G: Bsr      # velocity rows, pressure cols (nvel x 1 blocks)
    D: Bsr      # pressure rows, velocity cols (1 x nvel blocks)
    C: Bsr      # pressure block (1 x 1)
    nvel: int


def split(K: Bsr, nvel: int = 3) -> SchurSplit:
    """Split node blocks [(nvel+1) x (nvel+1)] into A, G, D, C (same block pattern)."""
    assert K.br == K.bc == nvel + 1
    d = K.data
    A = Bsr(K.indptr, K.indices, d[:, :nvel, :nvel].copy(), K.n_bcols)
    G = Bsr(K.indptr, K.indices, d[:, :nvel, nvel:].copy(), K.n_bcols)
    D = Bsr(K.indptr, K.indices, d[:, nvel:, :nvel].copy(), K.n_bcols)
    C = Bsr(K.indptr, K.indices, d[:, nvel:, nvel:].copy(), K.n_bcols)
    return SchurSplit(A, G, D, C, nvel)


def s_hat(S: SchurSplit) -> Bsr:
    """Eq. SchurApprox: S_hat = C - diag(D diag(A)^-1 G) on C's pattern."""
    dA = S.A.csr().diagonal()
    if np.any(dA == 0.0):
        raise ValueError("zero on the velocity diagonal")
    corr = (S.D.csr() @ sp.diags(1.0 / dA) @ S.G.csr()).diagonal()
    C = S.C.csr().astype(np.float64)
    Sh = C - sp.diags(corr)
    Sh = sp.csr_matrix(Sh)
    out = from_scipy(Sh, 1, 1)
    # keep C's stored pattern exactly (explicit zeros included)
    Cb = S.C
    data = Cb.data.copy()
    rows = Cb.block_rows()
    diag = rows == Cb.indices
    data[diag, 0, 0] = data[diag, 0, 0] - corr[rows[diag]]
    return Bsr(Cb.indptr, Cb.indices, data, Cb.n_bcols)


@dataclass
class SchurPrecond:
    split: SchurSplit
    S_hat: Bsr
    HA: amg.Hierarchy
    HS: amg.Hierarchy | None
    order: str = "full"            # "full" | "lower"
    M_S: np.ndarray | None = None  # pressure smoother (used when HS is None)

    def _pressure(self, q, transpose):
        if self.HS is not None:
            return amg.vcycle(self.HS, q, 0, transpose)
        return amg.apply_M(self.M_S, q, transpose)

    def apply(self, r: np.ndarray, transpose: bool = False) -> np.ndarray:
        """Eq. SchurPC with one preconditioner application per inner solve.
        The transposed application is the exact transpose: for "full" the
        same steps on K^T = [A^T D^T; G^T C^T] with transposed inner
        solves; for "lower" the upper-triangular steps p = S'^T r_p,
        u = A'^T (r_u - D^T p)."""
        nv = self.split.nvel
        rr = r.reshape(-1, nv + 1)
        ru = rr[:, :nv].reshape(-1).copy()
        rp = rr[:, nv].copy()
        if transpose:
            Dm = self.split.G.scipy().T      # acts as D' = G^T
            Gm = self.split.D.scipy().T      # acts as G' = D^T
        else:
            Dm = self.split.D.scipy()
            Gm = self.split.G.scipy()
        if self.order == "lower" and transpose:
            p = self._pressure(rp, True)
            u = amg.vcycle(self.HA, ru - Gm @ p, 0, True)
        else:
            u1 = amg.vcycle(self.HA, ru, 0, transpose)
            q = rp - Dm @ u1
            p = self._pressure(q, transpose)
            if self.order == "lower":
                u = u1
            else:
                u = amg.vcycle(self.HA, ru - Gm @ p, 0, transpose)
        z = np.empty_like(rr)
        z[:, :nv] = u.reshape(-1, nv)
        z[:, nv] = p
        return z.reshape(-1)


def build(K: Bsr, nvel: int = 3, prmA: amg.AmgParams | None = None,
          prmS: amg.AmgParams | None = None, order: str = "full",
          pressure: str = "amg") -> SchurPrecond:
    """pressure: "amg" (V-cycle on S_hat), or "spai0" / "jacobi" (one
    application of that smoother on S_hat)."""
    S = split(K, nvel)
    Sh = s_hat(S)
    HA = amg.build_hierarchy(S.A, prmA)
    if pressure == "amg":
        return SchurPrecond(S, Sh, HA, amg.build_hierarchy(Sh, prmS), order)
    prmS = prmS or amg.AmgParams()
    M = amg.spai0(Sh) if pressure == "spai0" else amg.jacobi(Sh, prmS.jacobi_omega)
    return SchurPrecond(S, Sh, HA, None, order, M)


def cast_values(pc: SchurPrecond, fmt: str) -> SchurPrecond:
    """The preconditioner as a mixed-precision form stores it: both inner
    hierarchies (amg.cast_values), the couplings G and D and the pressure
    smoother rounded to `fmt`.  C and S_hat enter only through the pressure
    hierarchy."""
    S = pc.split

    def rb(A):
        return Bsr(A.indptr, A.indices, round_to(A.data, fmt), A.n_bcols)

    sp_ = SchurSplit(S.A, rb(S.G), rb(S.D), S.C, S.nvel)
    return SchurPrecond(sp_, pc.S_hat, amg.cast_values(pc.HA, fmt),
                        amg.cast_values(pc.HS, fmt) if pc.HS is not None else None,
                        pc.order, round_to(pc.M_S, fmt) if pc.M_S is not None else None)
