"""Pins for the synthetic finite-difference Stokes systems (CPU only).

The discretisation is the stand-in for the paper's Section 3 systems
(Eq. StokesPDE on the unit cube); these checks pin it to closed forms.
"""
import numpy as np
import pytest
import scipy.sparse as sp

import stokes_inputs as si


def _K(N, mu=None):
    mu = np.ones(N ** 3) if mu is None else mu
    ip, ix, d = si.assemble_bsr(N, mu)
    return sp.bsr_matrix((d, ix, ip), shape=(4 * N ** 3, 4 * N ** 3)).tocsr()


def _coords(N):
    h = 1.0 / (N + 1)
    m = np.arange(N ** 3)
    return (m % N + 1) * h, ((m // N) % N + 1) * h, (m // (N * N) + 1) * h, h


def test_sizes_match_configs():
    # 7 blocks per interior row: N^3 + 6 N^2 (N-1) stored blocks
    for N in (3, 8, 64):
        ip, _, _ = si.assemble_bsr(N, np.ones(N ** 3))
        assert ip[-1] == N ** 3 + 6 * N * N * (N - 1)
    s = si.make_system("c1")
    assert s.indptr[-1] == 154624 and s.n == 16384


def test_quadratic_fields_are_differenced_exactly():
    """Central differences are exact for quadratics: on rows whose stencil
    avoids the ghost layer, K x equals the continuous operator
    (-Lap u + grad p, div u - 0.1 h^2 Lap p) with mu = 1."""
    N = 6
    x, y, z, h = _coords(N)
    u = np.stack([x * x + y * z, y * y + x * z, z * z + x * y, x * y * z + x * x], axis=1)
    r = (_K(N) @ u.reshape(-1)).reshape(-1, 4)
    ex = np.stack([
        -2.0 + (y * z + 2 * x),      # -Lap(x^2 + yz) + dp/dx
        -2.0 + x * z,                # -Lap(y^2 + xz) + dp/dy
        -2.0 + x * y,                # -Lap(z^2 + xy) + dp/dz
        2 * x + 2 * y + 2 * z - 0.1 * h * h * 2.0,
    ], axis=1)
    m = np.arange(N ** 3)
    i, j, k = m % N, (m // N) % N, m // (N * N)
    inner = (i > 0) & (i < N - 1) & (j > 0) & (j < N - 1) & (k > 0) & (k < N - 1)
    assert inner.sum() == (N - 2) ** 3
    np.testing.assert_allclose(r[inner], ex[inner], rtol=0, atol=1e-9)


def test_variable_viscosity_linear_field():
    """u = (x, 0, 0), p = 0 with per-node mu: the x-momentum row equals
    (mu_f(-x) - mu_f(+x)) / h with harmonic face means (ghost face: node mu)."""
    N = 5
    rng = np.random.default_rng(7)
    mu = np.exp(rng.standard_normal(N ** 3))
    x, y, z, h = _coords(N)
    v = np.zeros((N ** 3, 4))
    v[:, 0] = x
    r = (_K(N, mu) @ v.reshape(-1)).reshape(-1, 4)
    m = np.arange(N ** 3)
    i = m % N
    for node in range(N ** 3):
        def face(nb_ok, nb):
            return 2 * mu[node] * mu[nb] / (mu[node] + mu[nb]) if nb_ok else mu[node]
        fm = face(i[node] > 0, node - 1)
        fp = face(i[node] < N - 1, node + 1)
        # ghost neighbours hold 0 (Dirichlet), interior ones hold x -/+ h
        um = x[node] - h if i[node] > 0 else 0.0
        up = x[node] + h if i[node] < N - 1 else 0.0
        ny = 6 - 2  # y and z faces: neighbours equal or ghost 0
        expect = fm * (x[node] - um) / h ** 2 + fp * (x[node] - up) / h ** 2
        # y/z faces: interior neighbours share x, ghost neighbours are 0
        jj, kk = (node // N) % N, node // (N * N)
        for ok, nb in ((jj > 0, node - N), (jj < N - 1, node + N),
                       (kk > 0, node - N * N), (kk < N - 1, node + N * N)):
            f = face(ok, nb)
            expect += f * (x[node] - (x[node] if ok else 0.0)) / h ** 2
        assert ny == 4
        assert abs(r[node, 0] - expect) <= 1e-9 * max(1.0, abs(expect))
        # continuity row sees du/dx by central differences
        cont = ((up if i[node] < N - 1 else 0.0) - (um if i[node] > 0 else 0.0)) / (2 * h)
        assert abs(r[node, 3] - cont) <= 1e-9 * max(1.0, abs(cont))
        assert r[node, 1] == 0.0 and r[node, 2] == 0.0


def test_symmetric_part_and_definiteness():
    """K = [A G; -G^T C]: sym(K) has no velocity-pressure coupling and every
    eigenvalue of K has positive real part (dense, N = 3)."""
    N = 3
    mu = np.exp(0.5 * np.random.default_rng(3).standard_normal(N ** 3))
    K = _K(N, mu).toarray()
    S = 0.5 * (K + K.T)
    vel = np.arange(4 * N ** 3) % 4 != 3
    assert np.abs(S[np.ix_(vel, ~vel)]).max() == 0.0
    assert np.linalg.eigvalsh(S[np.ix_(vel, vel)]).min() > 0
    assert np.linalg.eigvalsh(S[np.ix_(~vel, ~vel)]).min() > 0
    assert np.linalg.eigvals(K).real.min() > 0
    # velocity blocks are symmetric, couplings antisymmetric
    np.testing.assert_array_equal(K[np.ix_(vel, vel)], K[np.ix_(vel, vel)].T)
    np.testing.assert_array_equal(K[np.ix_(vel, ~vel)], -K[np.ix_(~vel, vel)].T)


def test_seeded_inputs_are_reproducible():
    a = si.make_system("c2", N=6)
    b = si.make_system("c2", N=6)
    np.testing.assert_array_equal(a.data, b.data)
    np.testing.assert_array_equal(a.b, b.b)
    assert np.all(a.b.reshape(-1, 4)[:, 3] == 0.0)
    assert a.mu.std() > 0


def test_manufactured_rhs():
    s = si.make_system("c1", N=5)
    K = sp.csr_matrix((s.data, s.indices, s.indptr), shape=(s.n, s.n))
    np.testing.assert_allclose(K @ s.x_exact, s.b, rtol=0, atol=1e-12 * np.abs(s.b).max())
