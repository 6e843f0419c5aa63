"""Pins of the ILUT relaxation oracle (oracle/ilut.py) against what the
mathematics fixes: complete factorisations, the tridiagonal recurrence,
hand-computed dropping and fill limits, exactness of the Jacobi sweeps
once they outnumber the rows, and the transposed smoother."""
import numpy as np
import pytest
import scipy.linalg as sla
import scipy.sparse as sp

import stokes_inputs as si
from oracle import amg, bsr, ilut, schur


def _factors(L, d, U):
    n = len(d)
    Lf = np.eye(n) + L.toarray()
    Uf = np.diag(d) + U.toarray()
    return Lf, Uf


def _dd_matrix(n, density, seed):
    rng = np.random.default_rng(seed)
    M = sp.random(n, n, density=density, random_state=rng, format="csr")
    M.data = rng.standard_normal(M.nnz)
    M = M + sp.diags(np.abs(M).sum(axis=1).A1 + 1.0)
    return sp.csr_matrix(M)


def test_complete_factorisation_reproduces_A():
    """tau = 0 on a full matrix (every row's lower and upper counts are
    already the most a row can hold, so p = 1 limits nothing): ILUT is the
    complete LU without pivoting, so (I + L)(D + U) = A."""
    A = _dd_matrix(14, 1.0, 1)
    L, d, U = ilut.ilut(A, p=1.0, tau=0.0)
    Lf, Uf = _factors(L, d, U)
    Ad = A.toarray()
    assert np.abs(Lf @ Uf - Ad).max() <= 1e-13 * np.abs(Ad).max()
    assert np.allclose(np.tril(Lf, -1), L.toarray()) and np.allclose(np.triu(Uf, 1), U.toarray())


def test_tridiagonal_is_the_thomas_recurrence():
    """A tridiagonal matrix has no fill: l_i = a_{i,i-1} / u_{i-1},
    u_i = a_ii - l_i a_{i-1,i}, super-diagonal unchanged."""
    rng = np.random.default_rng(2)
    n = 25
    lo, up = rng.standard_normal(n - 1), rng.standard_normal(n - 1)
    dg = 4.0 + rng.random(n)
    A = sp.diags([lo, dg, up], [-1, 0, 1], format="csr")
    L, d, U = ilut.ilut(A, p=1.0, tau=0.0)
    u = np.empty(n)
    l = np.empty(n - 1)
    u[0] = dg[0]
    for i in range(1, n):
        l[i - 1] = lo[i - 1] / u[i - 1]
        u[i] = dg[i] - l[i - 1] * up[i - 1]
    np.testing.assert_array_equal(d, u)
    np.testing.assert_array_equal(L.diagonal(-1), l)
    np.testing.assert_array_equal(U.diagonal(1), up)
    assert L.nnz == n - 1 and U.nnz == n - 1


def test_drop_rule_hand_example():
    """Row 2's entry 0.02 (tested before the division by its pivot) is
    below tau ||a_2|| = 0.01 * sqrt(0.0004 + 1 + 16) = 0.0412 and is
    dropped with its update; the entry 1 survives, multiplier 1/3.75.  By
    hand: u_11 = 4 - 0.25 = 3.75, u_22 = 4 - 1/3.75."""
    A = sp.csr_matrix(np.array([[4.0, 1.0, 0.0], [1.0, 4.0, 1.0], [0.02, 1.0, 4.0]]))
    L, d, U = ilut.ilut(A, p=2.0, tau=0.01)
    np.testing.assert_allclose(d, [4.0, 3.75, 4.0 - 1.0 / 3.75], rtol=1e-15)
    Ld = L.toarray()
    assert Ld[1, 0] == 0.25 and Ld[2, 0] == 0.0
    assert abs(Ld[2, 1] - 1.0 / 3.75) <= 1e-16
    np.testing.assert_array_equal(U.toarray(), [[0, 1, 0], [0, 0, 1], [0, 0, 0]])


def test_fill_factor_keeps_the_largest_entries():
    """Row 3 = [1, 0, 0, 8] holds one lower entry.  By hand (tau = 0):
    column 0: multiplier 1/4, fill -0.25*2 = -0.5 at column 1 and
    -0.25*1 = -0.25 at column 2; column 1: multiplier -0.5/4 = -0.125,
    column 2 becomes -0.25 + 0.125 = -0.125; column 2: multiplier
    -0.125/4 = -0.03125.  With p = 1 only the largest lower entry (0.25)
    survives; with p = 3 all three do."""
    A = sp.csr_matrix(np.array([[4.0, 2.0, 1.0, 0.0],
                                [0.0, 4.0, 1.0, 0.0],
                                [0.0, 0.0, 4.0, 0.0],
                                [1.0, 0.0, 0.0, 8.0]]))
    L3, d3, U3 = ilut.ilut(A, p=3.0, tau=0.0)
    np.testing.assert_allclose(L3.toarray()[3, :3], [0.25, -0.125, -0.03125], rtol=0, atol=1e-16)
    assert d3[3] == 8.0
    L1, d1, U1 = ilut.ilut(A, p=1.0, tau=0.0)
    np.testing.assert_array_equal(L1.toarray()[3, :3], [0.25, 0.0, 0.0])
    assert d1[3] == 8.0


def test_lower_drop_test_is_scale_free():
    """Scaling A by 2^-14 (exact in binary) scales U and D by 2^-14 and
    leaves L unchanged bit for bit: the lower entries are tested before
    the division by the pivot, so every decision compares quantities of
    the same scale."""
    s = si.make_system("c3", N=5)
    A = schur.split(bsr.from_arrays(s.indptr, s.indices, s.data, 4), 3).A.csr()
    A = sp.csr_matrix(A)
    A.eliminate_zeros()
    L1, d1, U1 = ilut.ilut(A)
    sc = 2.0 ** -14
    L2, d2, U2 = ilut.ilut(A * sc)
    assert L1.nnz > 0 and L1.nnz == L2.nnz and (L1 != L2).nnz == 0
    np.testing.assert_array_equal(d2, d1 * sc)
    np.testing.assert_array_equal(U2.toarray(), U1.toarray() * sc)


def test_sweeps_are_exact_once_they_outnumber_the_rows():
    A = _dd_matrix(15, 0.3, 3)
    L, d, U = ilut.ilut(A, p=2.0, tau=1e-2)
    Lf, Uf = _factors(L, d, U)
    r = np.random.default_rng(4).standard_normal(15)
    S = ilut.Ilu(L, d, U, sweeps=15)
    ref = sla.solve_triangular(Uf, sla.solve_triangular(Lf, r, lower=True, unit_diagonal=True))
    np.testing.assert_allclose(S.apply(r), ref, rtol=1e-12, atol=1e-14)
    refT = sla.solve_triangular(Lf.T, sla.solve_triangular(Uf.T, r, lower=True),
                                lower=False, unit_diagonal=True)
    np.testing.assert_allclose(S.apply(r, transpose=True), refT, rtol=1e-12, atol=1e-14)


def test_zero_sweeps_is_jacobi():
    A = _dd_matrix(10, 0.4, 5)
    L, d, U = ilut.ilut(A)
    r = np.random.default_rng(6).standard_normal(10)
    S = ilut.Ilu(L, d, U, sweeps=0, omega=0.8)
    np.testing.assert_allclose(S.apply(r), 0.8 * r / d, rtol=1e-15)
    np.testing.assert_allclose(S.apply(r, transpose=True), 0.8 * r / d, rtol=1e-15)


@pytest.mark.parametrize("sweeps", [1, 2, 3])
def test_transposed_smoother_is_the_exact_transpose(sweeps):
    A = _dd_matrix(18, 0.25, 7)
    S = ilut.build(A, p=2.0, tau=1e-2, sweeps=sweeps)
    E = np.eye(18)
    Sf = np.array([S.apply(e) for e in E]).T
    St = np.array([S.apply(e, transpose=True) for e in E]).T
    np.testing.assert_allclose(St, Sf.T, rtol=1e-13, atol=1e-15)


def test_ilut_vcycle_transpose_and_convergence():
    """Velocity block of the C3 recipe at N=6 with ILUT relaxation: the
    transposed V-cycle is the transpose of the V-cycle, and the V-cycle
    contracts the error of A u = f."""
    s = si.make_system("c3", N=6)
    K = bsr.from_arrays(s.indptr, s.indices, s.data, 4)
    A = schur.split(K, 3).A
    H = amg.build_hierarchy(A, amg.AmgParams(coarse_enough=60, relax="ilut", smooth_P=False))
    assert len(H.levels) >= 1 and all(lev.S is not None for lev in H.levels)
    V = amg.vcycle_dense(H)
    VT = amg.vcycle_dense(H, transpose=True)
    np.testing.assert_allclose(VT, V.T, rtol=1e-12, atol=1e-14 * np.abs(V).max())
    Ad = A.dense()
    rho = np.abs(np.linalg.eigvals(np.eye(len(Ad)) - V @ Ad)).max()
    assert rho < 0.9, rho
