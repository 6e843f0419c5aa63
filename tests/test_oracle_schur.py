"""Oracle pins: Schur pressure correction, Eq. SchurPC / Eq. SchurApprox."""
import numpy as np
import pytest
import scipy.sparse as sp

import stokes_inputs as si
from oracle import amg, bsr, krylov, schur


def _K(N, seed=11):
    mu = np.exp(0.7 * np.random.default_rng(seed).standard_normal(N ** 3))
    ip, ix, d = si.assemble_bsr(N, mu)
    return bsr.from_arrays(ip, ix, d, 4)


def _perm(N):
    """Permutation from interleaved [u v w p] to [U; P] ordering."""
    n = N ** 3
    vel = np.array([4 * i + c for i in range(n) for c in range(3)])
    pre = np.array([4 * i + 3 for i in range(n)])
    return vel, pre


def test_split_reassembles_K():
    N = 3
    K = _K(N)
    S = schur.split(K)
    Kd = K.dense()
    vel, pre = _perm(N)
    np.testing.assert_array_equal(S.A.dense(), Kd[np.ix_(vel, vel)])
    np.testing.assert_array_equal(S.G.dense(), Kd[np.ix_(vel, pre)])
    np.testing.assert_array_equal(S.D.dense(), Kd[np.ix_(pre, vel)])
    np.testing.assert_array_equal(S.C.dense(), Kd[np.ix_(pre, pre)])


def test_s_hat_formula_dense():
    N = 3
    S = schur.split(_K(N))
    A, G, D, C = (S.A.dense(), S.G.dense(), S.D.dense(), S.C.dense())
    ref = C - np.diag(np.diag(D @ np.diag(1.0 / np.diag(A)) @ G))
    np.testing.assert_allclose(schur.s_hat(S).dense(), ref, rtol=1e-14, atol=1e-14)
    # on this system D = -G^T, so S_hat = C + diag(G^T diag(A)^-1 G) > C on the diagonal
    assert np.all(np.diag(schur.s_hat(S).dense()) > np.diag(C))


def _exact_schur(Kb):
    """Schur PC whose inner solves are exact: dense A^-1 and S^-1."""
    S = schur.split(Kb)
    A, G, D, C = (S.A.dense(), S.G.dense(), S.D.dense(), S.C.dense())
    Ai = np.linalg.inv(A)
    Si = np.linalg.inv(C - D @ Ai @ G)
    nv = 3

    def apply(r):
        rr = r.reshape(-1, nv + 1)
        ru = rr[:, :nv].reshape(-1)
        rp = rr[:, nv]
        p = Si @ (rp - D @ (Ai @ ru))
        u = Ai @ (ru - G @ p)
        z = np.empty_like(rr)
        z[:, :nv] = u.reshape(-1, nv)
        z[:, nv] = p
        return z.reshape(-1)
    return apply


def test_exact_inner_solves_give_K_inverse():
    """With exact inner solves Eq. SchurPC is K^-1: GMRES takes 1 iteration."""
    N = 3
    Kb = _K(N)
    Kd = Kb.dense()
    P = _exact_schur(Kb)
    b = np.random.default_rng(0).standard_normal(Kd.shape[0])
    np.testing.assert_allclose(P(b), np.linalg.solve(Kd, b), rtol=1e-9, atol=1e-12)
    x, info = krylov.gmres(lambda v: Kd @ v, P, b, m=30, tol=1e-10)
    assert info.converged and info.iters == 1


def test_schur_apply_matches_dense_composition_and_transpose():
    N = 3
    Kb = _K(N)
    pc = schur.build(Kb, 3, amg.AmgParams(coarse_enough=30), amg.AmgParams(coarse_enough=10))
    assert len(pc.HA.levels) >= 1 and len(pc.HS.levels) >= 1
    S = pc.split
    VA = amg.vcycle_dense(pc.HA)
    VS = amg.vcycle_dense(pc.HS)
    G, D = S.G.dense(), S.D.dense()
    # dense operator in [U; P] ordering, from the three steps of Eq. SchurPC
    Buu = VA + VA @ G @ VS @ D @ VA
    Bup = -VA @ G @ VS
    Bpu = -VS @ D @ VA
    Bpp = VS
    Bd = np.block([[Buu, Bup], [Bpu, Bpp]])
    vel, pre = _perm(N)
    order = np.concatenate([vel, pre])
    n = len(order)
    Bi = np.zeros((n, n))
    cols = np.array([pc.apply(e) for e in np.eye(n)]).T
    np.testing.assert_allclose(cols[np.ix_(order, order)], Bd, atol=1e-11 * np.abs(Bd).max())
    colsT = np.array([pc.apply(e, transpose=True) for e in np.eye(n)]).T
    np.testing.assert_allclose(colsT, cols.T, atol=1e-11 * np.abs(cols).max())


def _exact_lower(Kb):
    """LOWER ordering with exact inner solves: u = A^-1 r_u, p = S^-1 (r_p - D u)."""
    S = schur.split(Kb)
    A, G, D, C = (S.A.dense(), S.G.dense(), S.D.dense(), S.C.dense())
    Ai = np.linalg.inv(A)
    Si = np.linalg.inv(C - D @ Ai @ G)

    def apply(r):
        rr = r.reshape(-1, 4)
        ru = rr[:, :3].reshape(-1)
        u = Ai @ ru
        p = Si @ (rr[:, 3] - D @ u)
        z = np.empty_like(rr)
        z[:, :3] = u.reshape(-1, 3)
        z[:, 3] = p
        return z.reshape(-1)
    return apply


def test_lower_with_exact_inner_solves_two_gmres_iterations():
    """With the exact Schur complement the block-triangular preconditioner
    gives K B with minimal polynomial (z - 1)^2: GMRES needs <= 2 steps."""
    N = 3
    Kb = _K(N)
    Kd = Kb.dense()
    P = _exact_lower(Kb)
    b = np.random.default_rng(1).standard_normal(Kd.shape[0])
    KB = np.array([Kd @ P(e) for e in np.eye(Kd.shape[0])]).T
    E = KB - np.eye(Kd.shape[0])
    assert np.abs(E @ E).max() <= 1e-8 * np.abs(KB).max()
    x, info = krylov.gmres(lambda v: Kd @ v, P, b, m=30, tol=1e-10)
    assert info.converged and info.iters <= 2


@pytest.mark.parametrize("order", ["full", "lower"])
@pytest.mark.parametrize("pressure", ["amg", "spai0"])
def test_schur_variants_dense_composition_and_transpose(order, pressure):
    N = 3
    Kb = _K(N)
    pc = schur.build(Kb, 3, amg.AmgParams(coarse_enough=30), amg.AmgParams(coarse_enough=10),
                     order=order, pressure=pressure)
    S = pc.split
    VA = amg.vcycle_dense(pc.HA)
    if pressure == "amg":
        VS = amg.vcycle_dense(pc.HS)
    else:
        VS = np.diag(pc.M_S.reshape(-1))
        # one SPAI0 application: m_i = s_ii / sum_j s_ij^2 on S_hat
        Sd = pc.S_hat.dense()
        np.testing.assert_allclose(np.diag(VS), np.diag(Sd) / (Sd ** 2).sum(axis=1), rtol=1e-14)
    G, D = S.G.dense(), S.D.dense()
    if order == "full":
        Bd = np.block([[VA + VA @ G @ VS @ D @ VA, -VA @ G @ VS], [-VS @ D @ VA, VS]])
    else:
        Bd = np.block([[VA, np.zeros((VA.shape[0], VS.shape[0]))], [-VS @ D @ VA, VS]])
    vel, pre = _perm(N)
    order_idx = np.concatenate([vel, pre])
    n = len(order_idx)
    cols = np.array([pc.apply(e) for e in np.eye(n)]).T
    np.testing.assert_allclose(cols[np.ix_(order_idx, order_idx)], Bd, atol=1e-11 * np.abs(Bd).max())
    colsT = np.array([pc.apply(e, transpose=True) for e in np.eye(n)]).T
    np.testing.assert_allclose(colsT, cols.T, atol=1e-11 * np.abs(cols).max())
