"""C-ABI checks that need no GPU: exported symbols, the host-side C++
setup (smoothed aggregation, SPAI0/Jacobi, Galerkin products, Schur
split) against the oracle, and input validation."""
import os
import re

import numpy as np
import pytest
import scipy.sparse as sp

import stokes_inputs as si
from oracle import amg, bsr, schur
import paper_2006_06052_gb300 as gb

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module", autouse=True)
def built_library():
    gb.build()
    return gb.load_library()


def test_library_exports_every_declared_symbol(built_library):
    hdr = open(os.path.join(ROOT, "include", "gbstokes.h")).read()
    declared = sorted(set(re.findall(r"\b(gbs_[a-z0-9_]+)\s*\(", hdr)))
    assert declared, "no declarations found"
    assert sorted(gb.EXPORTED) == declared
    for name in declared:
        assert hasattr(built_library, name), name


def _host(s, **kw):
    p = gb.params_default(setup_only=1, **kw)
    return gb.build_hierarchy(s.indptr, s.indices, s.data, s.bdim, p)


def _rel_max(a, b):
    d = (sp.csr_matrix(a) - sp.csr_matrix(b))
    scale = abs(sp.csr_matrix(b)).max()
    return (abs(d).max() if d.nnz else 0.0) / scale


def _cmp_hierarchy(Hc, which, Ho, B, tol=1e-11):
    info = gb.hierarchy_info(Hc, which)
    assert info["nlevels"] == Ho.nlevels
    for l in range(Ho.nlevels):
        ptr, col, val, nbc = gb.export_level(Hc, which, l, 0)
        Ac = bsr.Bsr(ptr.astype(np.int64), col.astype(np.int64), val, nbc)
        Ao = Ho.A(l)
        assert Ac.n_brows == Ao.n_brows
        assert _rel_max(Ac.csr(), Ao.csr()) <= tol, ("A", l)
        if l + 1 == Ho.nlevels:
            Ai = gb.export_level(Hc, which, l, 5)
            np.testing.assert_allclose(Ai, Ho.Ainv_coarse, rtol=0,
                                       atol=1e-9 * np.abs(Ho.Ainv_coarse).max())
            continue
        lev = Ho.levels[l]
        agg = gb.export_level(Hc, which, l, 4)
        np.testing.assert_array_equal(agg, lev.agg)       # integer work: exact
        for part, Mo in ((1, lev.P), (2, lev.R)):
            ptr, col, val, nbc = gb.export_level(Hc, which, l, part)
            Mc = bsr.Bsr(ptr.astype(np.int64), col.astype(np.int64), val, nbc)
            assert Mc.shape == Mo.shape
            assert _rel_max(Mc.csr(), Mo.csr()) <= tol, (part, l)
        M = gb.export_level(Hc, which, l, 3)
        np.testing.assert_allclose(M, lev.M, rtol=0, atol=tol * np.abs(lev.M).max())


@pytest.mark.parametrize("N,relax", [(6, "jacobi"), (9, "jacobi"), (6, "spai0")])
def test_host_setup_block_matches_oracle(N, relax):
    s = si.make_system("c2", N=N)
    prm = amg.AmgParams(coarse_enough=40, relax=relax)
    Ho = amg.build_hierarchy(bsr.from_arrays(s.indptr, s.indices, s.data, 4), prm)
    assert len(Ho.levels) >= 2
    Hc = _host(s, coarse_enough=40, relax=gb.GBS_JACOBI if relax == "jacobi" else gb.GBS_SPAI0)
    _cmp_hierarchy(Hc, 0, Ho, 4)


def test_host_setup_scalar_csr_matches_oracle():
    s = si.make_system("c1", N=7)
    Ho = amg.build_hierarchy(bsr.from_arrays(s.indptr, s.indices, s.data, 1),
                             amg.AmgParams(coarse_enough=60))
    assert len(Ho.levels) >= 2
    Hc = _host(s, coarse_enough=60)
    _cmp_hierarchy(Hc, 0, Ho, 1)


def test_host_setup_schur_matches_oracle():
    s = si.make_system("c3", N=7)
    K = bsr.from_arrays(s.indptr, s.indices, s.data, 4)
    po = amg.AmgParams(coarse_enough=40)
    pc = schur.build(K, 3, po, po)
    Hc = _host(s, precond=gb.GBS_PC_SCHUR, krylov=gb.GBS_GMRES, coarse_enough=40)
    _cmp_hierarchy(Hc, 0, pc.HA, 3)
    _cmp_hierarchy(Hc, 1, pc.HS, 1)
    # level 0 of the pressure hierarchy is S_hat of Eq. SchurApprox
    ptr, col, val, nbc = gb.export_level(Hc, 1, 0, 0)
    Sc = bsr.Bsr(ptr.astype(np.int64), col.astype(np.int64), val, nbc)
    assert _rel_max(Sc.csr(), pc.S_hat.csr()) <= 1e-13


def test_host_setup_is_deterministic():
    s = si.make_system("c2", N=7)
    a, b = _host(s, coarse_enough=40), _host(s, coarse_enough=40)
    for l in range(gb.hierarchy_info(a)["nlevels"]):
        for part in (0,):
            pa, ca, va, _ = gb.export_level(a, 0, l, part)
            pb, cb, vb, _ = gb.export_level(b, 0, l, part)
            np.testing.assert_array_equal(pa, pb)
            np.testing.assert_array_equal(ca, cb)
            np.testing.assert_array_equal(va, vb)


def _expect_invalid(ptr, col, val, bdim, **kw):
    with pytest.raises(gb.GbsError) as e:
        _host(si.StokesSystem("x", 0, bdim, np.asarray(ptr), np.asarray(col), np.asarray(val),
                              None, None, None, ""), **kw)
    assert e.value.status == -1
    return str(e.value)


def test_invalid_inputs_rejected():
    # unsorted columns
    assert "increasing" in _expect_invalid([0, 2, 3], [1, 0, 1], [1.0, 2.0, 3.0], 1)
    # column out of range
    assert "range" in _expect_invalid([0, 1, 2], [0, 5], [1.0, 2.0], 1)
    # non-monotone row_ptr
    _expect_invalid([0, 2, 1], [0, 1], [1.0, 2.0], 1)
    # NaN value
    assert "finite" in _expect_invalid([0, 1, 2], [0, 1], [1.0, np.nan], 1)
    # missing diagonal block
    msg = _expect_invalid([0, 1, 2, 3], [1, 0, 2], [1.0, 1.0, 1.0], 1, coarse_enough=1)
    assert "diagonal" in msg
    # zero row -> SPAI0 Gram matrix singular
    n = 40
    A = sp.diags([-np.ones(n - 1), 2 * np.ones(n), -np.ones(n - 1)], [-1, 0, 1]).tolil()
    A[5, :] = 0.0
    A[5, 5] = 0.0
    A = A.tocsr()
    A.sort_indices()
    msg = _expect_invalid(A.indptr, A.indices, A.data, 1, coarse_enough=4)
    assert "singular" in msg or "diagonal" in msg
    # bad parameters
    s = si.make_system("c2", N=3)
    with pytest.raises(gb.GbsError):
        _host(s, restart=0)
    with pytest.raises(gb.GbsError):
        _host(s, precond=gb.GBS_PC_SCHUR, nvel=2)   # bdim 4 != nvel + 1


def test_setup_only_handle_refuses_device_calls():
    s = si.make_system("c2", N=3)
    H = _host(s)
    info = gb.hierarchy_info(H)
    assert info["bytes"] == 0 and info["nlevels"] >= 1
    # no device form of K exists: the outer SpMV format reads as block
    assert gb.outer_format(H) == ("block", s.data.size)
    # device calls are refused on a host-only handle (no GPU touched)
    assert gb.load_library().gbs_level_apply(H.handle, 0, 0, 0, 16, 16, 32, None) == -1


def test_host_setup_plain_aggregation_matches_oracle():
    """smooth_P = 0: plain (unsmoothed) aggregation, P = P_tent (the
    paper's velocity AMG in its V2-V4 solvers)."""
    s = si.make_system("c3", N=7)
    K = bsr.from_arrays(s.indptr, s.indices, s.data, 4)
    po = amg.AmgParams(coarse_enough=40, smooth_P=False)
    pc = schur.build(K, 3, po, po)
    Hc = _host(s, precond=gb.GBS_PC_SCHUR, krylov=gb.GBS_GMRES, coarse_enough=40, smooth_P=0)
    _cmp_hierarchy(Hc, 0, pc.HA, 3)
    _cmp_hierarchy(Hc, 1, pc.HS, 1)
    ptr, col, val, nbc = gb.export_level(Hc, 0, 0, 1)
    assert np.all(np.diff(ptr) == 1)                       # one block per row
    np.testing.assert_array_equal(val, np.broadcast_to(np.eye(3), val.shape))


@pytest.mark.parametrize("case", ["c3_velocity", "c2_monolithic"])
def test_host_ilut_factors_match_oracle(case):
    """The C++ ILUT of every level (relax = ILUT) equals the oracle's ILUT
    of the same exported level matrix: same drop and fill decisions (FP64,
    same operation order), values to the last bit."""
    from oracle import ilut
    if case == "c3_velocity":
        s = si.make_system("c3", N=7)
        H = _host(s, precond=gb.GBS_PC_SCHUR, krylov=gb.GBS_GMRES, coarse_enough=40,
                  relax=gb.GBS_ILUT)
        which = 0
    else:
        s = si.make_system("c2", N=7)
        H = _host(s, coarse_enough=40, relax=gb.GBS_ILUT)
        which = 0
    info = gb.hierarchy_info(H, which)
    assert info["nlevels"] >= 2
    for l in range(info["nlevels"] - 1):
        ptr, col, val, nbc = gb.export_level(H, which, l, 0)
        B = val.shape[1]
        A = sp.bsr_matrix((val, col, ptr), shape=(len(ptr) - 1) * B * np.array([1, 1])).tocsr()
        A.eliminate_zeros()
        A.sort_indices()
        Lo, do, Uo = ilut.ilut(A, p=2.0, tau=1e-2)
        for part, Mo in ((6, Lo), (7, Uo)):
            cp, cc, cv, n = gb.export_level(H, which, l, part)
            assert n == A.shape[0]
            np.testing.assert_array_equal(cp, Mo.indptr)
            np.testing.assert_array_equal(cc, Mo.indices)
            np.testing.assert_array_equal(cv, Mo.data)
        np.testing.assert_array_equal(gb.export_level(H, which, l, 8), do)


def test_ilut_parameters_validated():
    s = si.make_system("c2", N=3)
    with pytest.raises(gb.GbsError):
        _host(s, relax=gb.GBS_ILUT, ilut_sweeps=17)
    with pytest.raises(gb.GbsError):
        _host(s, relax=gb.GBS_ILUT, ilut_omega=0.0)
    with pytest.raises(gb.GbsError):
        _host(s, precond=gb.GBS_PC_SCHUR, schur_p=1, relax_p=gb.GBS_ILUT)


def test_params_layout_matches_the_header():
    """gbs_params_default fills the ctypes mirror: the trailing fields come
    back with their documented defaults only if every field before them has
    the C layout."""
    p = gb.params_default()
    assert (p.idr_s, p.idr_seed) == (5, 0)
    assert (p.ilut_p, p.ilut_tau, p.ilut_sweeps, p.ilut_omega) == (2.0, 1e-2, 2, 1.0)
    assert (p.gmres_reorth, p.wait_log2, p.iso_blocks) == (0, 31, 1)
    assert (p.relax, p.relax_p, p.level_format, p.schur_p, p.schur_order) == (0, 0, 0, 0, 0)


@pytest.mark.parametrize("smooth_P", [1, 0])
def test_velocity_hierarchy_is_identity_blocks(smooth_P):
    """The library's own setup of the Schur velocity hierarchy (C3 recipe)
    keeps every stored block of A_l, P_l, R_l and the SPAI0 blocks an exact
    multiple of I_3 at every level -- the condition under which the device
    stores those levels as S (x) I_3 (iso_blocks)."""
    s = si.make_system("c3", N=8)
    H = _host(s, precond=gb.GBS_PC_SCHUR, krylov=gb.GBS_GMRES, coarse_enough=60,
              smooth_P=smooth_P)
    nl = gb.hierarchy_info(H, 0)["nlevels"]
    assert nl >= 2
    for l in range(nl - 1):
        blocks = [gb.export_level(H, 0, l, part)[2] for part in (0, 1, 2)]
        blocks.append(gb.export_level(H, 0, l, 3).reshape(-1, 3, 3))
        for v in blocks:
            off = v.copy()
            for a in range(3):
                off[:, a, a] = 0.0
            assert not off.any(), l
            assert np.array_equal(v[:, 1, 1], v[:, 0, 0]) and np.array_equal(v[:, 2, 2], v[:, 0, 0]), l


def test_iso_blocks_parameter_validated():
    """iso_blocks takes 0 (level_format decides every level's layout) or 1
    (levels of identity-multiple blocks stored as S (x) I_B); anything else
    is rejected before any work."""
    s = si.make_system("c3", N=4)
    for v in (0, 1):
        _host(s, precond=gb.GBS_PC_SCHUR, krylov=gb.GBS_GMRES, coarse_enough=40, iso_blocks=v)
    with pytest.raises(gb.GbsError) as e:
        _host(s, precond=gb.GBS_PC_SCHUR, krylov=gb.GBS_GMRES, coarse_enough=40, iso_blocks=2)
    assert e.value.status == -1
