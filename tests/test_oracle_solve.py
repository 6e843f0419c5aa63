"""Oracle pins: whole preconditioned solves against dense LU (CPU only)."""
import numpy as np
import pytest

import stokes_inputs as si
from oracle import amg, bsr, krylov, schur


@pytest.mark.parametrize("N", [3, 4, 5])
def test_amg_bicgstab_matches_dense_lu(N):
    s = si.make_system("c2", N=N)
    K = bsr.from_arrays(s.indptr, s.indices, s.data, 4)
    H = amg.build_hierarchy(K, amg.AmgParams(coarse_enough=24, relax="jacobi"))
    assert len(H.levels) >= 1
    Kd = K.dense()
    x, info = krylov.bicgstab(lambda v: Kd @ v, lambda v: amg.vcycle(H, v), s.b, tol=1e-10)
    assert info.converged
    xl = np.linalg.solve(Kd, s.b)
    cond = np.linalg.cond(Kd)
    assert np.linalg.norm(x - xl) / np.linalg.norm(xl) <= cond * 1e-10


@pytest.mark.parametrize("N", [3, 4])
def test_schur_gmres_matches_dense_lu(N):
    s = si.make_system("c3", N=N)
    K = bsr.from_arrays(s.indptr, s.indices, s.data, 4)
    pc = schur.build(K, 3, amg.AmgParams(coarse_enough=20), amg.AmgParams(coarse_enough=8))
    Kd = K.dense()
    x, info = krylov.gmres(lambda v: Kd @ v, pc.apply, s.b, m=30, tol=1e-10)
    assert info.converged
    xl = np.linalg.solve(Kd, s.b)
    assert np.linalg.norm(x - xl) / np.linalg.norm(xl) <= np.linalg.cond(Kd) * 1e-10


def test_scalar_csr_c1_recovers_manufactured_solution():
    """C1 reading: b = K x_m, so the solve recovers x_m to ~cond * tol."""
    s = si.make_system("c1", N=6)
    K = bsr.from_arrays(s.indptr, s.indices, s.data, 1)
    H = amg.build_hierarchy(K, amg.AmgParams(coarse_enough=100))
    assert len(H.levels) >= 1
    Ks = K.scipy()
    x, info = krylov.bicgstab(lambda v: Ks @ v, lambda v: amg.vcycle(H, v), s.b, tol=1e-10)
    assert info.converged
    assert np.linalg.norm(x - s.x_exact) / np.linalg.norm(s.x_exact) < 1e-6
