"""Oracle pins: BiCGStab and GMRES(m) (CPU only)."""
import numpy as np
import scipy.sparse as sp

from oracle import krylov


def _spd_tridiag(n, seed=0):
    rng = np.random.default_rng(seed)
    d = 4.0 + rng.random(n)
    e = -1.0 + 0.2 * rng.random(n - 1)
    return sp.diags([e, d, e], [-1, 0, 1]).tocsr()


def test_gmres_full_space_converges_within_n():
    n = 50
    A = _spd_tridiag(n)
    b = np.random.default_rng(1).standard_normal(n)
    x, info = krylov.gmres(lambda v: A @ v, lambda v: v, b, m=n, tol=1e-12, maxiter=n)
    assert info.converged and info.iters <= n
    np.testing.assert_allclose(A @ x, b, atol=1e-10 * np.linalg.norm(b))
    # the Arnoldi residual estimate decreases monotonically (minimal residual)
    h = np.array(info.history)
    assert np.all(np.diff(h) <= 1e-14)


def test_bicgstab_converges_identity_precond():
    n = 50
    A = _spd_tridiag(n, 2)
    b = np.random.default_rng(3).standard_normal(n)
    x, info = krylov.bicgstab(lambda v: A @ v, lambda v: v, b, tol=1e-12)
    assert info.converged
    np.testing.assert_allclose(A @ x, b, atol=1e-11 * np.linalg.norm(b))


def test_exact_preconditioner_one_iteration():
    rng = np.random.default_rng(4)
    n = 30
    A = rng.standard_normal((n, n)) + n * np.eye(n)
    Ai = np.linalg.inv(A)
    b = rng.standard_normal(n)
    x, info = krylov.gmres(lambda v: A @ v, lambda v: Ai @ v, b, m=30, tol=1e-10)
    assert info.converged and info.iters == 1
    x2, info2 = krylov.bicgstab(lambda v: A @ v, lambda v: Ai @ v, b, tol=1e-10)
    assert info2.converged and info2.iters == 1
    np.testing.assert_allclose(x, np.linalg.solve(A, b), rtol=1e-9)


def test_restart_and_warm_start():
    n = 60
    A = _spd_tridiag(n, 5)
    b = np.random.default_rng(6).standard_normal(n)
    x, info = krylov.gmres(lambda v: A @ v, lambda v: v, b, m=5, tol=1e-10, maxiter=500)
    assert info.converged and info.iters > 5
    # a converged start returns immediately
    x2, info2 = krylov.gmres(lambda v: A @ v, lambda v: v, b, x0=x, m=5, tol=1e-8)
    assert info2.iters == 0 and info2.converged
    x3, info3 = krylov.bicgstab(lambda v: A @ v, lambda v: v, b, x0=x, tol=1e-8)
    assert info3.iters == 0 and info3.converged


def test_zero_rhs_and_maxiter():
    A = _spd_tridiag(10)
    x, info = krylov.bicgstab(lambda v: A @ v, lambda v: v, np.zeros(10))
    assert info.converged and info.iters == 0 and not x.any()
    b = np.ones(10)
    x, info = krylov.bicgstab(lambda v: A @ v, lambda v: v, b, tol=1e-30, maxiter=1)
    assert not info.converged and info.iters == 1


def test_bicgstab_residual_replacement_keeps_true_residual():
    n = 80
    A = _spd_tridiag(n, 7) + sp.diags([0.3 * np.ones(n - 1)], [1])
    b = np.random.default_rng(8).standard_normal(n)
    x, info = krylov.bicgstab(lambda v: A @ v, lambda v: v, b, tol=1e-10, replace_every=3)
    assert info.converged and info.replacements >= 1
    assert np.linalg.norm(b - A @ x) / np.linalg.norm(b) <= 1e-10


def test_splitmix64_published_first_output():
    """SplitMix64 seeded with 0: the first output is 0xE220A8397B1DCDAF."""
    z = krylov.splitmix64(np.array([0], dtype=np.uint64), 0)
    assert int(z[0]) == 0xE220A8397B1DCDAF


def test_idr_shadow_space_orthonormal_and_deterministic():
    P = krylov.idr_shadow_space(1000, 5)
    np.testing.assert_allclose(P @ P.T, np.eye(5), atol=1e-13)
    np.testing.assert_array_equal(P, krylov.idr_shadow_space(1000, 5))
    assert not np.allclose(P, krylov.idr_shadow_space(1000, 5, seed=1))


def test_idrs_exact_preconditioner_one_iteration():
    rng = np.random.default_rng(12)
    n = 40
    A = rng.standard_normal((n, n)) + n * np.eye(n)
    Ai = np.linalg.inv(A)
    b = rng.standard_normal(n)
    x, info = krylov.idrs(lambda v: A @ v, lambda v: Ai @ v, b, s=5, tol=1e-10)
    assert info.converged and info.iters == 1
    np.testing.assert_allclose(x, np.linalg.solve(A, b), rtol=1e-9)


def test_idrs_converges_nonsymmetric_identity_precond():
    n = 80
    A = _spd_tridiag(n, 9) + sp.diags([0.4 * np.ones(n - 1)], [1])
    b = np.random.default_rng(10).standard_normal(n)
    for s in (1, 2, 5):
        x, info = krylov.idrs(lambda v: A @ v, lambda v: v, b, s=s, tol=1e-10, maxiter=2000)
        assert info.converged, s
        assert np.linalg.norm(b - A @ x) / np.linalg.norm(b) <= 1e-10
        # IDR(s) terminates within n + n/s matvecs in exact arithmetic
        assert info.iters <= 2 * n


def test_idrs_residual_stays_orthogonal_to_shadow_space():
    """After the s inner steps of the first cycle the residual is orthogonal
    to the shadow space (the defining property of the IDR step)."""
    n = 60
    A = _spd_tridiag(n, 13) + sp.diags([0.2 * np.ones(n - 1)], [-1])
    b = np.random.default_rng(14).standard_normal(n)
    s = 4
    P = krylov.idr_shadow_space(n, s)
    _, info = krylov.idrs(lambda v: A @ v, lambda v: v, b, s=s, tol=1e-30, maxiter=s, P=P)
    # rerun the same s steps and capture r
    x, info = krylov.idrs(lambda v: A @ v, lambda v: v, b, s=s, tol=1e-30, maxiter=s, P=P)
    r = b - A @ x
    assert np.abs(P @ r).max() <= 1e-10 * np.linalg.norm(b)
