"""Oracle pins: adjoint solve and sampled outer-product gradient (CPU only)."""
import numpy as np

import stokes_inputs as si
from oracle import adjoint, amg, bsr, krylov


def test_sampled_outer_matches_brute_force():
    rng = np.random.default_rng(0)
    # 3-row BSR with 4x4 blocks, irregular pattern
    K = bsr.Bsr(np.array([0, 2, 3, 5]), np.array([0, 2, 1, 0, 2]), rng.standard_normal((5, 4, 4)), 3)
    lam = rng.standard_normal(12)
    x = rng.standard_normal(12)
    np.testing.assert_array_equal(adjoint.sampled_outer(K, lam, x), adjoint.sampled_outer_brute(K, lam, x))


def _loss_setup(N):
    s = si.make_system("c2", N=N)
    K = bsr.from_arrays(s.indptr, s.indices, s.data, 4)
    xt = si.gaussian_vector(K.shape[0], 4001)
    return s, K, xt


def _solve(K, b, H, tol, transpose=False):
    Ks = K.scipy().T if transpose else K.scipy()
    x, info = krylov.bicgstab(lambda v: Ks @ v, lambda v: amg.vcycle(H, v, 0, transpose), b,
                              tol=tol, maxiter=2000)
    assert info.converged
    return x


def test_adjoint_gradient_matches_dense_inverse():
    """L = 1/2 ||x - x_t||^2, x = K^-1 b: dL/db = K^-T (x - x_t) and
    dL/dK = -lambda x^T restricted to the pattern (dense inverse, N = 4)."""
    s, K, xt = _loss_setup(4)
    Kd = K.dense()
    H = amg.build_hierarchy(K, amg.AmgParams(coarse_enough=30, relax="jacobi"))
    x = _solve(K, s.b, H, 1e-12)
    lam = _solve(K, x - xt, H, 1e-12, transpose=True)
    xd = np.linalg.solve(Kd, s.b)
    lamd = np.linalg.solve(Kd.T, xd - xt)
    np.testing.assert_allclose(lam, lamd, rtol=1e-8, atol=1e-8 * np.abs(lamd).max())
    G = adjoint.sampled_outer(K, lam, x)
    full = -np.outer(lamd, xd)
    rows = K.block_rows()
    for k in range(K.nnzb):
        i, j = rows[k], K.indices[k]
        ref = full[4 * i:4 * i + 4, 4 * j:4 * j + 4]
        np.testing.assert_allclose(G[k], ref, rtol=1e-7, atol=1e-7 * np.abs(full).max())


def test_adjoint_gradient_central_differences():
    """FP64 central differences (h = 1e-6) of the loss, evaluated with dense
    LU solves so that the difference carries no iteration noise, against
    the gradient from the iterative adjoint solve (to 1e-13)."""
    s, K, xt = _loss_setup(3)
    H = amg.build_hierarchy(K, amg.AmgParams(coarse_enough=30, relax="jacobi"))

    def dloss(Kp, bp, Km, bm):
        """L(+) - L(-) for L = 1/2 ||x - x_t||^2, written as
        1/2 (x+ - x-) . (x+ + x- - 2 x_t) to avoid cancellation."""
        xp = np.linalg.solve(Kp.dense(), bp)
        xm = np.linalg.solve(Km.dense(), bm)
        return 0.5 * np.dot(xp - xm, xp + xm - 2.0 * xt)

    x = _solve(K, s.b, H, 1e-13)
    lam = _solve(K, x - xt, H, 1e-13, transpose=True)
    G = adjoint.sampled_outer(K, lam, x)
    rng = np.random.Generator(np.random.PCG64(4002))
    h = 1e-6
    for _ in range(8):
        k = int(rng.integers(K.nnzb))
        a, c = int(rng.integers(4)), int(rng.integers(4))
        Kp = bsr.Bsr(K.indptr, K.indices, K.data.copy(), K.n_bcols)
        Km = bsr.Bsr(K.indptr, K.indices, K.data.copy(), K.n_bcols)
        step = h * max(1.0, abs(K.data[k, a, c]))
        Kp.data[k, a, c] += step
        Km.data[k, a, c] -= step
        fd = dloss(Kp, s.b, Km, s.b) / (2 * step)
        assert abs(fd - G[k, a, c]) <= 1e-5 * max(abs(fd), 1e-3 * np.abs(G).max())
    for idx in rng.integers(K.shape[0], size=4):
        e = np.zeros(K.shape[0])
        e[idx] = h
        fd = dloss(K, s.b + e, K, s.b - e) / (2 * h)
        assert abs(fd - lam[idx]) <= 1e-5 * max(abs(fd), 1e-3 * np.abs(lam).max())
