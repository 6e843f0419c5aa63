"""Adjoint solve and sampled outer-product gradient (FP64 oracle).

For x = K^-1 b and a scalar loss L(x) with g = dL/dx, the adjoint
lambda = K^-T g gives dL/db = lambda and, for every stored block
k = (i, j) of K, dL/dK_ij = -lambda_i x_j^T (entry (a, c) of the block is
-lambda[B i + a] x[B j + c]), evaluated on the stored pattern only.
The adjoint solve uses the same Krylov method on K^T with the transposed
preconditioner.
"""
from __future__ import annotations

import numpy as np

from .bsr import Bsr


def sampled_outer(K: Bsr, lam: np.ndarray, x: np.ndarray, alpha: float = -1.0) -> np.ndarray:
    """grad[k, a, c] = alpha * lam[br*i + a] * x[bc*j + c] for stored block k = (i, j)."""
    rows = K.block_rows()
    lb = lam.reshape(-1, K.br)[rows]
    xb = x.reshape(-1, K.bc)[K.indices]
    return alpha * lb[:, :, None] * xb[:, None, :]


def sampled_outer_brute(K: Bsr, lam, x, alpha=-1.0):
    """Entry-by-entry loop form of ``sampled_outer`` (for tiny cases)."""
    out = np.zeros_like(K.data)
    for i in range(K.n_brows):
        for k in range(K.indptr[i], K.indptr[i + 1]):
            j = K.indices[k]
            for a in range(K.br):
                for c in range(K.bc):
                    out[k, a, c] = alpha * lam[K.br * i + a] * x[K.bc * j + c]
    return out
