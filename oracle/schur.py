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
u* = V_A(r_u), p = V_S(r_p - D u*), u = V_A(r_u - G p).
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np
import scipy.sparse as sp

from . import amg
from .bsr import Bsr, from_scipy


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
    HS: amg.Hierarchy

    def apply(self, r: np.ndarray, transpose: bool = False) -> np.ndarray:
        """Eq. SchurPC with one V-cycle per inner solve.  The transposed
        application is the same step on K^T = [A^T D^T; G^T C^T] with
        transposed V-cycles (it equals the exact transpose of ``apply``)."""
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
        u1 = amg.vcycle(self.HA, ru, 0, transpose)
        q = rp - Dm @ u1
        p = amg.vcycle(self.HS, q, 0, transpose)
        u = amg.vcycle(self.HA, ru - Gm @ p, 0, transpose)
        z = np.empty_like(rr)
        z[:, :nv] = u.reshape(-1, nv)
        z[:, nv] = p
        return z.reshape(-1)


def build(K: Bsr, nvel: int = 3, prmA: amg.AmgParams | None = None,
          prmS: amg.AmgParams | None = None) -> SchurPrecond:
    S = split(K, nvel)
    Sh = s_hat(S)
    HA = amg.build_hierarchy(S.A, prmA)
    HS = amg.build_hierarchy(Sh, prmS)
    return SchurPrecond(S, Sh, HA, HS)
