"""Oracle pins: Schur pressure correction, Eq. SchurPC / Eq. SchurApprox."""
import numpy as np
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
