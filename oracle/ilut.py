"""ILUT relaxation (FP64 oracle).  Test infrastructure only.

The paper's velocity solver (Section 4, Listings V2-V4) is aggregation AMG
relaxed by ILUT, the dual-threshold incomplete LU of Saad (1994).  The
paper names the smoother but gives neither its parameters nor how its
triangular solves are carried out; the readings used here are:

1. Factorisation (Saad's ILUT), row by row on the scalar matrix of the
   level's nonzeros, rows and columns in their natural order:
     w = a_i;  tau_i = tau * ||a_i||_2 (sum of squares in column order);
     for k < i with w_k != 0, in increasing k (fill included):
         if |w_k| < tau_i: w_k = 0 and skip;  else w_k = w_k / u_kk;
         w_j -= w_k * u_kj for the strictly upper entries j of U's row k;
     drop every upper w_j (j > i) with |w_j| < tau_i;
   A lower entry is tested before its division by the pivot, in the units
   of a_i as the upper entries are: Saad tests the multiplier itself,
   which on a matrix whose entries are far from 1 (the FD levels scale as
   1/h^2) drops every multiplier and leaves no L at all.
     keep the floor(p * nnz_L(a_i)) largest |w_j|, j < i, and the
     floor(p * nnz_U(a_i)) largest, j > i (p a fill factor relative to
     the row's own lower / upper counts, so a row with no upper entries
     keeps no upper fill; ties to the smaller column);
     u_ii = w_i, replaced by tau_i (1 if tau_i = 0) when it is zero.
   Defaults p = 2, tau = 1e-2.
2. Triangular solves: m Jacobi sweeps each (Anzt, Chow & Dongarra 2015,
   iterative sparse triangular solves for preconditioning), m = 2:
     y_0 = r,  y_k = r - L y_{k-1}            (L strictly lower, unit diag)
     z_0 = D^-1 y,  z_k = D^-1 (y - U z_{k-1})  (U strictly upper, D diag)
   With m >= n the sweeps are exact (L and D^-1 U are nilpotent).
3. Relaxation x += omega S (f - A x), S = z(y(.)), omega = 1; the zero
   guess step is x = omega S f.  The transposed smoother is the exact
   transpose of S: v_0 = r, v_k = r - U^T D^-1 v_{k-1}, then D^-1 v_m;
   t_0 = that, t_k = t_0 - L^T t_{k-1}.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np
import scipy.sparse as sp


@dataclass
class Ilu:
    L: sp.csr_matrix      # strictly lower part of the unit lower factor
    d: np.ndarray         # diagonal of U
    U: sp.csr_matrix      # strictly upper part of U
    sweeps: int = 2
    omega: float = 1.0

    def apply(self, r: np.ndarray, transpose: bool = False) -> np.ndarray:
        m = self.sweeps
        if not transpose:
            y = r.copy()
            for _ in range(m):
                y = r - self.L @ y
            z = y / self.d
            for _ in range(m):
                z = (y - self.U @ z) / self.d
            return self.omega * z
        UT = self.U.T.tocsr()
        v = r.copy()
        for _ in range(m):
            v = r - UT @ (v / self.d)
        t0 = v / self.d
        t = t0.copy()
        LT = self.L.T.tocsr()
        for _ in range(m):
            t = t0 - LT @ t
        return self.omega * t


def _keep_largest(entries: list, count: int) -> list:
    """The `count` entries (j, v) of largest |v|, ties to the smaller j,
    returned in increasing j."""
    if count <= 0:
        return []
    ranked = sorted(entries, key=lambda e: (-abs(e[1]), e[0]))[:count]
    return sorted(ranked)


def ilut(A: sp.spmatrix, p: float = 2.0, tau: float = 1e-2) -> tuple:
    """Reading 1: returns (L strictly lower CSR, d, U strictly upper CSR)."""
    A = sp.csr_matrix(A, dtype=np.float64)
    A.sort_indices()
    n = A.shape[0]
    Lrows, Urows = [], []          # lists of (j, v) per row, increasing j
    d = np.zeros(n)
    for i in range(n):
        cols = A.indices[A.indptr[i]:A.indptr[i + 1]]
        vals = A.data[A.indptr[i]:A.indptr[i + 1]]
        nzL = nzU = 0
        s = 0.0
        w = {}
        for j, v in zip(cols, vals):
            if v == 0.0:
                continue
            w[int(j)] = float(v)
            s += float(v) * float(v)
            if j < i:
                nzL += 1
            elif j > i:
                nzU += 1
        tau_i = tau * math.sqrt(s)
        done = set()
        while True:
            pend = [k for k in w if k < i and k not in done]
            if not pend:
                break
            k = min(pend)
            done.add(k)
            if abs(w[k]) < tau_i:
                w[k] = 0.0
                continue
            wk = w[k] / d[k]
            w[k] = wk
            for j, ukj in Urows[k]:
                w[j] = w.get(j, 0.0) - wk * ukj
        lower = [(j, v) for j, v in w.items() if j < i and v != 0.0]
        upper = [(j, v) for j, v in w.items() if j > i and v != 0.0 and abs(v) >= tau_i]
        Lrows.append(_keep_largest(lower, int(math.floor(p * nzL))))
        Urows.append(_keep_largest(upper, int(math.floor(p * nzU))))
        di = w.get(i, 0.0)
        if di == 0.0:
            di = tau_i if tau_i != 0.0 else 1.0
        d[i] = di

    def csr(rows):
        ptr = np.zeros(n + 1, dtype=np.int64)
        ind, val = [], []
        for i, r in enumerate(rows):
            for j, v in r:
                ind.append(j)
                val.append(v)
            ptr[i + 1] = len(ind)
        return sp.csr_matrix((np.array(val, dtype=np.float64), np.array(ind, dtype=np.int64), ptr),
                             shape=(n, n))
    return csr(Lrows), d, csr(Urows)


def build(A: sp.spmatrix, p: float = 2.0, tau: float = 1e-2, sweeps: int = 2,
          omega: float = 1.0) -> Ilu:
    L, d, U = ilut(A, p, tau)
    return Ilu(L, d, U, sweeps, omega)
