"""Oracle pins: smoothed-aggregation setup, SPAI0 and the V-cycle (CPU only).

Each check is independent of the oracle's own code path: closed forms,
hand-computed aggregates, dense re-derivations of the operators, or
variational/linear-algebra invariants.
"""
import numpy as np
import pytest
import scipy.sparse as sp

import stokes_inputs as si
from oracle import amg, bsr


def poisson1d(n, scale=1.0):
    A = sp.diags([-np.ones(n - 1), 2 * np.ones(n), -np.ones(n - 1)], [-1, 0, 1]) * scale
    return bsr.from_scipy(sp.csr_matrix(A), 1, 1)


def stokes_bsr(N, name="c2"):
    s = si.make_system(name, N=N)
    return bsr.from_arrays(s.indptr, s.indices, s.data, 4)


def test_strength_threshold_closed_form():
    # 3x3 scalar matrix: |a01|^2 = 0.25 vs eps^2 |a00||a11| = 0.01*4*1
    A = bsr.from_scipy(sp.csr_matrix(np.array([[4.0, 0.5, 0.01], [0.5, 1.0, 0.0], [0.01, 0.0, 1.0]])), 1, 1)
    strong, s = amg.strong_couplings(A, 0.1)
    rows = A.block_rows()
    got = {(int(rows[k]), int(A.indices[k])) for k in range(A.nnzb) if strong[k]}
    # 0.0001 < 0.01*sqrt(16)*sqrt(1)*... -> (0,2) weak; (0,1),(1,0) strong
    assert got == {(0, 1), (1, 0)}


def test_aggregation_chain_hand_computed():
    """1D chain of 7 nodes, all couplings strong and equal.  Pass 1: root 0
    takes {0,1}; node 2 sees aggregated 1 and is skipped; root 3 takes
    {2,3,4}; node 5 sees aggregated 4; root 6 takes {5,6}.  Pass 2 has
    nothing left."""
    A = poisson1d(7)
    agg, n_agg = amg.aggregate(A, 0.08)
    # node 2 is taken by root 3's aggregate in pass 1 (it is 3's neighbour)
    assert n_agg == 3
    assert agg.tolist() == [0, 0, 1, 1, 1, 2, 2]


def test_aggregation_pass2_tie_breaks_to_smaller_id():
    """A path whose middle node is left over after pass 1, adjacent to two
    aggregates with equal coupling strength: it joins the smaller id."""
    M = np.zeros((5, 5))
    for i in range(5):
        M[i, i] = 2.0
    for a, b in ((0, 1), (1, 2), (2, 3), (3, 4)):
        M[a, b] = M[b, a] = -1.0
    # order 4 < 2 is needed for 4 to become root first: relabel 2 <-> 4
    perm = [0, 1, 4, 3, 2]
    Mp = M[np.ix_(perm, perm)]
    A = bsr.from_scipy(sp.csr_matrix(Mp), 1, 1)
    agg, n_agg = amg.aggregate(A, 0.08)
    # new labels: 0-1, 1-4, 4-3, 3-2.  pass 1: 0 -> {0,1}; 2 -> {2,3};
    # 4 sees 1 (agg 0) and 3 (agg 1) with equal strength -> agg 0
    assert agg.tolist() == [0, 0, 1, 1, 0]


@pytest.mark.parametrize("N", [3, 5])
def test_aggregates_partition_and_are_strongly_connected(N):
    A = stokes_bsr(N)
    agg, n_agg = amg.aggregate(A, 0.08)
    assert set(agg.tolist()) == set(range(n_agg))
    strong, _ = amg.strong_couplings(A, 0.08)
    rows = A.block_rows()
    # every aggregate with >1 node is connected through strong couplings
    adj = {}
    for k in np.nonzero(strong)[0]:
        adj.setdefault(int(rows[k]), set()).add(int(A.indices[k]))
    for a in range(n_agg):
        members = set(np.nonzero(agg == a)[0].tolist())
        if len(members) == 1:
            continue
        start = next(iter(members))
        seen, stack = {start}, [start]
        while stack:
            v = stack.pop()
            for w in adj.get(v, ()):
                if w in members and w not in seen:
                    seen.add(w)
                    stack.append(w)
        assert seen == members


def test_tentative_P_partitions_nodes():
    A = stokes_bsr(4)
    agg, n_agg = amg.aggregate(A, 0.08)
    Pt = amg.tentative_P(agg, n_agg, 4).dense()
    # each scalar row has exactly one 1; row sums are 1; columns are disjoint
    assert np.all(Pt.sum(axis=1) == 1.0)
    assert np.all((Pt == 0) | (Pt == 1))
    G = Pt.T @ Pt
    assert np.all(G == np.diag(np.diag(G)))


def test_spai0_closed_forms():
    # diagonal matrix: M = A^-1
    A = bsr.from_scipy(sp.diags([2.0, 4.0, 5.0]).tocsr(), 1, 1)
    np.testing.assert_allclose(amg.spai0(A).reshape(-1), [0.5, 0.25, 0.2], rtol=1e-15)
    # 1D Laplacian interior row (-1, 2, -1): 2 / (1 + 4 + 1) = 1/3
    M = amg.spai0(poisson1d(5)).reshape(-1)
    assert abs(M[2] - 1.0 / 3.0) < 1e-15
    assert abs(M[0] - 2.0 / 5.0) < 1e-15
    # block-diagonal matrix with dense blocks: M_i = A_ii^-1
    rng = np.random.default_rng(0)
    blocks = rng.standard_normal((3, 4, 4)) + 4 * np.eye(4)
    Ab = bsr.Bsr(np.arange(4), np.arange(3), blocks, 3)
    np.testing.assert_allclose(amg.spai0(Ab), np.linalg.inv(blocks), rtol=1e-12, atol=1e-14)


def test_spai0_block_is_frobenius_minimiser():
    """M minimises ||I - M A||_F over block-diagonal M: any perturbation
    of any block increases the objective (first-order optimality)."""
    A = stokes_bsr(3)
    M = amg.spai0(A)
    Ad = A.dense()
    n = Ad.shape[0]

    def obj(Mb):
        Md = sp.block_diag(list(Mb)).toarray()
        return np.linalg.norm(np.eye(n) - Md @ Ad) ** 2

    f0 = obj(M)
    rng = np.random.default_rng(1)
    for _ in range(5):
        D = rng.standard_normal(M.shape) * 1e-3 * np.abs(M).max()
        assert obj(M + D) > f0
        assert obj(M - D) > f0


def test_jacobi_is_scaled_block_inverse():
    A = stokes_bsr(3)
    M = amg.jacobi(A, 0.72)
    D = A.data[amg.diag_positions(A)]
    np.testing.assert_allclose(np.einsum("iab,ibc->iac", M, D),
                               np.broadcast_to(0.72 * np.eye(4), D.shape), atol=1e-13)


def test_spectral_radius_estimate():
    # D^-1 A of the 1D Laplacian has eigenvalues 1 - cos(k pi/(n+1))
    n = 40
    A = poisson1d(n)
    DA = bsr.Bsr(A.indptr, A.indices, A.data / 2.0, A.n_bcols)
    true = 1 + np.cos(np.pi / (n + 1))
    est = amg.spectral_radius(DA, 20)
    assert 0.9 * true <= est <= true * (1 + 1e-12)


def test_smoothed_P_dense_formula():
    A = stokes_bsr(4)
    agg, n_agg = amg.aggregate(A, 0.08)
    Pt = amg.tentative_P(agg, n_agg, 4)
    P, omega = amg.smoothed_P(A, Pt)
    Ad = A.dense()
    D = np.zeros_like(Ad)
    for i in range(A.n_brows):
        D[4 * i:4 * i + 4, 4 * i:4 * i + 4] = Ad[4 * i:4 * i + 4, 4 * i:4 * i + 4]
    DinvA = np.linalg.solve(D, Ad)
    rho = np.abs(np.linalg.eigvals(DinvA)).max()
    assert 0.8 * rho <= 4.0 / 3.0 / omega <= rho * (1 + 1e-9)
    expect = (np.eye(Ad.shape[0]) - omega * DinvA) @ Pt.dense()
    np.testing.assert_allclose(P.dense(), expect, atol=1e-12)


def test_galerkin_triple_product_and_R_is_P_transpose():
    A = stokes_bsr(5)
    H = amg.build_hierarchy(A, amg.AmgParams(coarse_enough=40, relax="jacobi"))
    assert len(H.levels) >= 2
    for l, lev in enumerate(H.levels):
        Ad = lev.A.dense()
        Pd = lev.P.dense()
        Rd = lev.R.dense()
        np.testing.assert_array_equal(Rd, Pd.T)
        Ac = H.A(l + 1).dense()
        ref = Pd.T @ Ad @ Pd
        np.testing.assert_allclose(Ac, ref, atol=1e-13 * np.abs(ref).max())
    np.testing.assert_allclose(H.Ainv_coarse @ H.A_coarse.dense(), np.eye(H.A_coarse.shape[0]),
                               atol=1e-10)


def test_vcycle_one_level_is_exact_inverse():
    A = stokes_bsr(3)
    H = amg.build_hierarchy(A, amg.AmgParams(coarse_enough=1000))
    assert len(H.levels) == 0
    f = np.random.default_rng(2).standard_normal(A.shape[0])
    np.testing.assert_allclose(A.dense() @ amg.vcycle(H, f), f, atol=1e-10)


@pytest.mark.parametrize("relax", ["spai0", "jacobi"])
def test_vcycle_two_level_dense_formula(relax):
    """With one pre-sweep from zero and one post-sweep the V-cycle is
    B = M + (I - M A) M + (I - M A) P Ac^-1 R (I - A M)."""
    A = stokes_bsr(3)
    H = amg.build_hierarchy(A, amg.AmgParams(coarse_enough=60, relax=relax))
    assert len(H.levels) == 1
    lev = H.levels[0]
    Ad = A.dense()
    n = Ad.shape[0]
    Md = sp.block_diag(list(lev.M)).toarray()
    Pd, Rd = lev.P.dense(), lev.R.dense()
    Aci = np.linalg.inv(H.A_coarse.dense())
    I = np.eye(n)
    B = Md + (I - Md @ Ad) @ Md + (I - Md @ Ad) @ Pd @ Aci @ Rd @ (I - Ad @ Md)
    V = amg.vcycle_dense(H)
    np.testing.assert_allclose(V, B, atol=1e-12 * np.abs(B).max())
    VT = amg.vcycle_dense(H, transpose=True)
    np.testing.assert_allclose(VT, B.T, atol=1e-12 * np.abs(B).max())


def test_vcycle_multilevel_linear_and_transposed():
    A = stokes_bsr(4)
    H = amg.build_hierarchy(A, amg.AmgParams(coarse_enough=30, relax="jacobi"))
    assert len(H.levels) >= 2
    rng = np.random.default_rng(5)
    a, b = rng.standard_normal((2, A.shape[0]))
    Va, Vb = amg.vcycle(H, a), amg.vcycle(H, b)
    np.testing.assert_allclose(amg.vcycle(H, 2.0 * a - 3.0 * b), 2.0 * Va - 3.0 * Vb,
                               atol=1e-12 * np.abs(Va).max())
    # <V^T a, b> == <a, V b>
    lhs = amg.vcycle(H, a, transpose=True) @ b
    rhs = a @ Vb
    assert abs(lhs - rhs) <= 1e-11 * abs(rhs) + 1e-11


def test_two_grid_contracts_on_poisson():
    A = poisson1d(63, scale=64.0 ** 2)
    H = amg.build_hierarchy(A, amg.AmgParams(coarse_enough=30))
    assert len(H.levels) >= 1
    V = amg.vcycle_dense(H)
    E = np.eye(63) - V @ A.dense()
    assert np.abs(np.linalg.eigvals(E)).max() < 0.9


def test_plain_aggregation_prolongator_is_tentative():
    A = stokes_bsr(4)
    H = amg.build_hierarchy(A, amg.AmgParams(coarse_enough=30, smooth_P=False, relax="jacobi"))
    for lev in H.levels:
        Pt = amg.tentative_P(lev.agg, lev.P.n_bcols, 4)
        np.testing.assert_array_equal(lev.P.dense(), Pt.dense())


# ------------------------------------------------------- level schedule
def chain8(weak):
    """8-node scalar chain, diagonal 4; strong pairs (0,1), (2,3), (4,5),
    (6,7) coupled by -2.5 and the pairs between them by `weak`."""
    M = 4.0 * np.eye(8)
    for i in range(7):
        c = -2.5 if i % 2 == 0 else weak
        M[i, i + 1] = M[i + 1, i] = c
    return bsr.from_scipy(sp.csr_matrix(M), 1, 1)


def test_level_schedule_hand_computed_three_levels():
    """The strength threshold is eps at level 0 and eps/2 at level 1
    (eps_l = eps 0.5^l).  eps = 0.5, plain aggregation (P = P_tent), so the
    coarse operators are sums of entries.

    Level 0: a coupling c is strong iff c^2 > 0.25 * 4 * 4 = 4.
      6.25 > 4: strong; 1.5625 <= 4: weak.  Pass 1 gives {0,1} {2,3}
      {4,5} {6,7}.  (At eps/2 the threshold would be 1 and the weak
      pairs would be strong.)
    Level 1: A_1 = P^T A_0 P is tridiagonal with diagonal 4+4-2*2.5 = 3
      and off-diagonal -1.25.  Threshold 0.25^2 * 3 * 3 = 0.5625 < 1.5625:
      strong.  (At eps it would be 2.25: every node a singleton.)  Pass 1:
      root 0 takes {0,1}; node 2 sees aggregated 1; root 3 takes {3,2}.
    Level 2: A_2 = [[3.5, -1.25], [-1.25, 3.5]] holds 2 unknowns, at most
      coarse_enough = 2: the coarsest level."""
    H = amg.build_hierarchy(chain8(-1.25),
                            amg.AmgParams(eps_strong=0.5, coarse_enough=2, smooth_P=False,
                                          relax="jacobi"))
    assert H.nlevels == 3
    assert H.levels[0].agg.tolist() == [0, 0, 1, 1, 2, 2, 3, 3]
    assert H.levels[1].agg.tolist() == [0, 0, 1, 1]
    np.testing.assert_array_equal(H.levels[1].A.dense(),
                                  [[3, -1.25, 0, 0], [-1.25, 3, -1.25, 0],
                                   [0, -1.25, 3, -1.25], [0, 0, -1.25, 3]])
    np.testing.assert_array_equal(H.A_coarse.dense(), [[3.5, -1.25], [-1.25, 3.5]])
    np.testing.assert_allclose(H.Ainv_coarse, np.linalg.inv([[3.5, -1.25], [-1.25, 3.5]]),
                               rtol=1e-15)


def test_level_schedule_stop_rules():
    """The three ways coarsening ends, on the same chain.
    coarse_enough = 1: level 2 (2 unknowns) coarsens once more, eps_2 =
      0.125: threshold 0.015625 * 3.5^2 < 1.5625, one aggregate, A_3 = [4.5].
    max_levels = 3 stops after two coarsenings although 2 > coarse_enough.
    weak = -0.7: level 1's couplings (0.49 <= 0.5625) are all weak, every
      node is a singleton, aggregation does not shrink the level: stop."""
    A = chain8(-1.25)
    H4 = amg.build_hierarchy(A, amg.AmgParams(eps_strong=0.5, coarse_enough=1, smooth_P=False,
                                              relax="jacobi"))
    assert H4.nlevels == 4
    assert H4.levels[2].agg.tolist() == [0, 0]
    np.testing.assert_array_equal(H4.A_coarse.dense(), [[4.5]])
    H3 = amg.build_hierarchy(A, amg.AmgParams(eps_strong=0.5, coarse_enough=1, max_levels=3,
                                              smooth_P=False, relax="jacobi"))
    assert H3.nlevels == 3 and H3.A_coarse.n_brows == 2
    H2 = amg.build_hierarchy(chain8(-0.7),
                             amg.AmgParams(eps_strong=0.5, coarse_enough=1, smooth_P=False,
                                           relax="jacobi"))
    assert H2.nlevels == 2 and H2.A_coarse.n_brows == 4
    assert H2.levels[0].agg.tolist() == [0, 0, 1, 1, 2, 2, 3, 3]


def _velocity_block(N):
    """The velocity block A_uu of the C3 recipe (3 x 3 blocks) and the
    scalar S with A_uu = S (x) I_3 (u, v, w share every coefficient)."""
    from oracle import schur
    s = si.make_system("c3", N=N)
    A = schur.split(bsr.from_arrays(s.indptr, s.indices, s.data, 4), 3).A
    S = bsr.Bsr(A.indptr.copy(), A.indices.copy(), A.data[:, :1, :1].copy(), A.n_bcols)
    return A, S


def _is_identity_multiple(data):
    B = data.shape[1]
    off = data.copy()
    for a in range(B):
        off[:, a, a] = 0.0
    diag = np.stack([data[:, a, a] for a in range(B)], 1)
    return not off.any() and np.array_equal(diag, np.repeat(diag[:, :1], B, 1))


@pytest.mark.parametrize("relax", ["spai0", "jacobi"])
def test_plain_aggregation_of_identity_blocks_is_kron_of_scalar(relax):
    """Block SA on A = S (x) I_3 with plain aggregation equals the scalar
    setup on S, Kronecker I_3, at every level: the same aggregates, A_l, P_l,
    R_l and smoother blocks, and the coarse inverse.  This ties the block
    code paths (block strength, block SPAI0 / Jacobi inverses, block
    Galerkin products) to the scalar ones, and it is the structure the
    library's S (x) I_B layout stores."""
    A, S = _velocity_block(6)
    assert np.abs(A.dense() - np.kron(S.dense(), np.eye(3))).max() == 0.0
    prm = amg.AmgParams(coarse_enough=30, relax=relax, smooth_P=False)
    Hb, Hs = amg.build_hierarchy(A, prm), amg.build_hierarchy(S, prm)
    assert len(Hb.levels) == len(Hs.levels) >= 2
    I3 = np.eye(3)
    for Lb, Ls in zip(Hb.levels, Hs.levels):
        np.testing.assert_array_equal(Lb.agg, Ls.agg)
        for Xb, Xs in ((Lb.A, Ls.A), (Lb.P, Ls.P), (Lb.R, Ls.R)):
            ref = np.kron(Xs.dense(), I3)
            assert np.abs(Xb.dense() - ref).max() <= 1e-14 * np.abs(ref).max()
        mref = np.einsum("i,ab->iab", Ls.M[:, 0, 0], I3)
        assert np.abs(Lb.M - mref).max() <= 1e-14 * np.abs(mref).max()
    ref = np.kron(Hs.Ainv_coarse, I3)
    assert np.abs(Hb.Ainv_coarse - ref).max() <= 1e-12 * np.abs(ref).max()


def test_smoothed_aggregation_keeps_identity_blocks():
    """With prolongator smoothing (its damping comes from a power iteration,
    so the scalar and block setups differ in omega), every stored block of
    every level -- A_l, P_l, R_l, the SPAI0 blocks -- is still exactly a
    multiple of I_3, bit for bit, and level 0 aggregates as the scalar S."""
    A, S = _velocity_block(7)
    prm = amg.AmgParams(coarse_enough=40)
    Hb = amg.build_hierarchy(A, prm)
    assert len(Hb.levels) >= 2
    for L in Hb.levels:
        for X in (L.A, L.P, L.R):
            assert _is_identity_multiple(X.data)
        assert _is_identity_multiple(L.M)
    agg_s, _ = amg.aggregate(S, prm.eps_strong)
    np.testing.assert_array_equal(Hb.levels[0].agg, agg_s)
