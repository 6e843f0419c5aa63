"""Oracle pins: storage formats and SpMV (CPU only)."""
import numpy as np

import stokes_inputs as si
from oracle import bsr

from conftest import load_golden


def _paper_example():
    g = load_golden("paper_block_example.txt")
    dense = np.array([g["dense%d" % i] for i in range(6)])
    return g, dense


def test_paper_worked_example_csr_to_bsr():
    """Section 4's 6x6 example: the printed CSR arrays group into the
    printed 2x2 block arrays."""
    g, dense = _paper_example()
    ptr = np.array(g["csr_ptr"], dtype=int)
    col = np.array(g["csr_col"], dtype=int)
    val = np.array(g["csr_val"])
    # the printed CSR arrays describe the printed dense matrix
    rebuilt = np.zeros((6, 6))
    for i in range(6):
        for k in range(ptr[i], ptr[i + 1]):
            rebuilt[i, col[k]] = val[k]
    np.testing.assert_array_equal(rebuilt, dense)
    B = bsr.csr_to_bsr(ptr, col, val, 6, 2)
    np.testing.assert_array_equal(B.indptr, np.array(g["bsr_ptr"], dtype=int))
    np.testing.assert_array_equal(B.indices, np.array(g["bsr_col"], dtype=int))
    np.testing.assert_array_equal(B.data.reshape(-1), np.array(g["bsr_val"]))
    np.testing.assert_array_equal(B.dense(), dense)
    # and back: block -> scalar CSR without stored zeros is the printed CSR
    p2, c2, v2 = bsr.bsr_to_csr(B, drop_zeros=True)
    np.testing.assert_array_equal(p2, ptr)
    np.testing.assert_array_equal(c2, col)
    np.testing.assert_array_equal(v2, val)


def test_paper_example_counts():
    """Section 4: the block form has half the rows and a quarter of the
    logical nonzeros of the scalar form."""
    g, _ = _paper_example()
    assert len(g["bsr_ptr"]) - 1 == (len(g["csr_ptr"]) - 1) // 2
    assert len(g["bsr_col"]) * 4 == len(g["csr_col"])


def test_spmv_matches_dense():
    for N in (3, 4):
        s = si.make_system("c2", N=N)
        A = bsr.from_arrays(s.indptr, s.indices, s.data, 4)
        x = np.random.default_rng(N).standard_normal(A.shape[1])
        Ad = A.dense()
        np.testing.assert_allclose(bsr.spmv(A, x), Ad @ x, rtol=1e-14, atol=1e-14 * np.abs(Ad).max())
        np.testing.assert_allclose(bsr.spmv_t(A, x), Ad.T @ x, rtol=1e-14, atol=1e-14 * np.abs(Ad).max())
        r = bsr.residual(s.b, A, x)
        np.testing.assert_allclose(r, s.b - Ad @ x, rtol=1e-14, atol=1e-13 * np.abs(Ad).max())


def test_transpose_map():
    s = si.make_system("c2", N=3)
    A = bsr.from_arrays(s.indptr, s.indices, s.data, 4)
    tm = bsr.transpose_map(A)
    rows = A.block_rows()
    for k in range(A.nnzb):
        t = tm[k]
        assert rows[t] == A.indices[k] and A.indices[t] == rows[k]
    AT = bsr.transpose(A)
    np.testing.assert_array_equal(AT.dense(), A.dense().T)
