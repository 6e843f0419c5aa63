"""CSR / block-CSR (BSR) containers for the oracle.

Section 4 of the paper defines the two storage formats with a worked
6x6 example: scalar CSR (ptr, col, val) and block-valued CSR whose
entries are small dense blocks (2x2 in the example; 3x3 for the velocity
sub-problem, Listing V3).  A BSR matrix here is (indptr, indices, data)
with data[k] the row-major dense block of stored block k.

Products use scipy.sparse as a library primitive; everything else is
written out.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np
import scipy.sparse as sp


@dataclass
class Bsr:
    indptr: np.ndarray      # int64 [n_brows + 1]
    indices: np.ndarray     # int64 [nnzb], sorted within each row
    data: np.ndarray        # f64 [nnzb, br, bc]
    n_bcols: int

    @property
    def n_brows(self) -> int:
        return len(self.indptr) - 1

    @property
    def br(self) -> int:
        return self.data.shape[1]

    @property
    def bc(self) -> int:
        return self.data.shape[2]

    @property
    def nnzb(self) -> int:
        return len(self.indices)

    @property
    def shape(self):
        return (self.n_brows * self.br, self.n_bcols * self.bc)

    def block_rows(self) -> np.ndarray:
        """Row index of every stored block."""
        return np.repeat(np.arange(self.n_brows), np.diff(self.indptr))

    def scipy(self) -> sp.bsr_matrix:
        return sp.bsr_matrix((self.data, self.indices, self.indptr), shape=self.shape)

    def csr(self) -> sp.csr_matrix:
        A = self.scipy().tocsr()
        A.sort_indices()
        return A

    def dense(self) -> np.ndarray:
        return self.scipy().toarray()


def from_scipy(A, br: int, bc: int, n_bcols: int | None = None) -> Bsr:
    """Convert any scipy sparse matrix to Bsr with (br x bc) blocks."""
    if br == 1 and bc == 1:
        C = sp.csr_matrix(A)
        C.sort_indices()
        return Bsr(C.indptr.astype(np.int64), C.indices.astype(np.int64),
                   C.data.reshape(-1, 1, 1).astype(np.float64), C.shape[1])
    Bm = sp.bsr_matrix(A, blocksize=(br, bc))
    Bm.sort_indices()
    return Bsr(Bm.indptr.astype(np.int64), Bm.indices.astype(np.int64),
               np.array(Bm.data, dtype=np.float64), Bm.shape[1] // bc)


def from_arrays(indptr, indices, data, bdim: int, n_bcols: int | None = None) -> Bsr:
    """Wrap caller arrays (bdim 1 accepts flat CSR values)."""
    indptr = np.asarray(indptr, dtype=np.int64)
    indices = np.asarray(indices, dtype=np.int64)
    data = np.asarray(data, dtype=np.float64).reshape(-1, bdim, bdim)
    if n_bcols is None:
        n_bcols = len(indptr) - 1
    return Bsr(indptr, indices, data, n_bcols)


def spmv(A: Bsr, x: np.ndarray) -> np.ndarray:
    """y = A x (scipy's sparse product, a library primitive)."""
    return A.scipy() @ x


def spmv_t(A: Bsr, x: np.ndarray) -> np.ndarray:
    """y = A^T x."""
    return A.scipy().T @ x


def residual(f: np.ndarray, A: Bsr, x: np.ndarray) -> np.ndarray:
    """r = f - A x: the backend residual primitive of Section 2.3."""
    return f - spmv(A, x)


def csr_to_bsr(indptr, indices, vals, n: int, B: int) -> Bsr:
    """Group a scalar CSR matrix (n x n) into B x B blocks, written out
    from the definition of the block-valued format (Section 4): block
    (I, J) is stored iff some scalar entry (i, j) with i // B == I and
    j // B == J is stored; absent entries inside a stored block are 0."""
    assert n % B == 0
    nb = n // B
    rows_blocks = []
    for I in range(nb):
        cols = set()
        for i in range(I * B, I * B + B):
            for k in range(indptr[i], indptr[i + 1]):
                cols.add(int(indices[k]) // B)
        rows_blocks.append(sorted(cols))
    bptr = np.zeros(nb + 1, dtype=np.int64)
    for I in range(nb):
        bptr[I + 1] = bptr[I] + len(rows_blocks[I])
    bcol = np.array([J for r in rows_blocks for J in r], dtype=np.int64)
    data = np.zeros((len(bcol), B, B))
    for I in range(nb):
        for i in range(I * B, I * B + B):
            for k in range(indptr[i], indptr[i + 1]):
                j = int(indices[k])
                J = j // B
                kb = bptr[I] + rows_blocks[I].index(J)
                data[kb, i - I * B, j - J * B] = vals[k]
    return Bsr(bptr, bcol, data, nb)


def bsr_to_csr(A: Bsr, drop_zeros: bool = False):
    """Expand BSR into scalar CSR arrays (row-major inside each block)."""
    ptr = [0]
    col = []
    val = []
    for I in range(A.n_brows):
        for a in range(A.br):
            for k in range(A.indptr[I], A.indptr[I + 1]):
                J = int(A.indices[k])
                for c in range(A.bc):
                    v = A.data[k, a, c]
                    if drop_zeros and v == 0.0:
                        continue
                    col.append(J * A.bc + c)
                    val.append(float(v))
            ptr.append(len(col))
    return np.array(ptr, dtype=np.int64), np.array(col, dtype=np.int64), np.array(val)


def transpose(A: Bsr) -> Bsr:
    """Explicit transpose (blocks transposed too)."""
    T = A.scipy().T.tocsr()
    return from_scipy(T, A.bc, A.br)


def transpose_map(A: Bsr) -> np.ndarray:
    """tmap[k] = index of block (j, i) for stored block k = (i, j).
    Requires a structurally symmetric block pattern (raises otherwise)."""
    rows = A.block_rows()
    key = {}
    for k in range(A.nnzb):
        key[(int(rows[k]), int(A.indices[k]))] = k
    tmap = np.empty(A.nnzb, dtype=np.int64)
    for k in range(A.nnzb):
        t = key.get((int(A.indices[k]), int(rows[k])))
        if t is None:
            raise ValueError("block pattern is not structurally symmetric")
        tmap[k] = t
    return tmap
