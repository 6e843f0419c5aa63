"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle.

Tolerances (FP64 forms): SpMV elementwise |y - y_ref| <= 1e-13 (|A||x|)_i
(the rounding bound of a dot product of <= 48 terms is ~48 eps); V-cycle
and Schur applications on the same (imported) hierarchy 1e-12 relative in
the max norm; whole solves reach the 1e-8 true relative residual with an
iteration count within +-10% of the oracle's.  Mixed forms (FP32/BF16
hierarchies) are judged by the FP64 true residual and report their error
against the oracle solution.
"""
import math

import numpy as np
import pytest

import stokes_inputs as si
from oracle import adjoint, amg, bsr, krylov, schur
from oracle.precision import round_to

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
import paper_2006_06052_gb300 as gb  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    gb.build()
    return gb.load_library()


def dev(a):
    return torch.as_tensor(np.ascontiguousarray(a, dtype=np.float64), device="cuda")


def host(t):
    torch.cuda.synchronize()
    return t.detach().cpu().numpy()


def rel_inf(a, b):
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


def check_spmv(H, A, x, transpose=False):
    y = host(gb.spmv(H, dev(x), transpose=transpose))
    Asp = A.scipy().T if transpose else A.scipy()
    ref = Asp @ x
    bound = abs(Asp) @ np.abs(x)
    assert np.all(np.abs(y - ref) <= 1e-13 * bound + 1e-300)


# ------------------------------------------------------------------ SpMV
@pytest.mark.parametrize("fmt", ["0", "1", "2", "3"])
@pytest.mark.parametrize("case", ["c1_csr", "c2_bsr4", "vel_bsr3"])
def test_outer_spmv_and_transpose(case, fmt, monkeypatch):
    """K in block form (1), as scalar CSR of its nonzeros (2), in 32-node
    component slices (3), or as chosen automatically (0: slices on these
    stencil systems)."""
    monkeypatch.setenv("GBS_LEVEL_FORMAT", fmt)
    N = 9   # 729 nodes: a ragged tail for every rows-per-warp grouping
    if case == "c1_csr":
        s = si.make_system("c1", N=N)
        A = bsr.from_arrays(s.indptr, s.indices, s.data, 1)
        ip, ix, d, B = s.indptr, s.indices, s.data, 1
    elif case == "c2_bsr4":
        s = si.make_system("c2", N=N)
        A = bsr.from_arrays(s.indptr, s.indices, s.data, 4)
        ip, ix, d, B = s.indptr, s.indices, s.data, 4
    else:
        s = si.make_system("c3", N=N)
        A = schur.split(bsr.from_arrays(s.indptr, s.indices, s.data, 4)).A
        ip, ix, d, B = A.indptr, A.indices, A.data, 3
    H = gb.build_hierarchy(ip, ix, d, B, gb.params_default(relax=gb.GBS_JACOBI))
    x = np.random.default_rng(1).standard_normal(A.shape[0])
    check_spmv(H, A, x)
    check_spmv(H, A, x, transpose=True)


def test_paper_block_example_spmv():
    """The 2x2-block matrix of the paper's Section 4 worked example."""
    from conftest import load_golden
    g = load_golden("paper_block_example.txt")
    A = bsr.Bsr(np.array(g["bsr_ptr"], dtype=np.int64), np.array(g["bsr_col"], dtype=np.int64),
                np.array(g["bsr_val"]).reshape(-1, 2, 2), 3)
    H = gb.build_hierarchy(A.indptr, A.indices, A.data, 2, gb.params_default(enable_adjoint=0))
    for seed in range(3):
        x = np.random.default_rng(seed).standard_normal(6)
        check_spmv(H, A, x)


# ------------------------------------------------------- V-cycle / Schur
def _import(Ho, B, **kw):
    lv = Ho.levels
    As = [(L.A.indptr, L.A.indices, L.A.data) for L in lv] + \
         [(Ho.A_coarse.indptr, Ho.A_coarse.indices, Ho.A_coarse.data)]
    Ps = [(L.P.indptr, L.P.indices, L.P.data, L.P.n_bcols) for L in lv]
    Rs = [(L.R.indptr, L.R.indices, L.R.data, L.R.n_bcols) for L in lv]
    Ms = [L.M for L in lv]
    return gb.import_hierarchy(As, Ps, Rs, Ms, Ho.Ainv_coarse, B, gb.params_default(**kw))


@pytest.mark.parametrize("fmt", ["0", "0u", "1", "2", "3", "3w", "1b", "3o"])
@pytest.mark.parametrize("cfg", [("c2", 9, "jacobi"), ("c2", 10, "spai0"), ("c1", 9, "spai0")])
def test_vcycle_on_imported_oracle_hierarchy(cfg, fmt, monkeypatch):
    """Level formats: 0 automatic (scalar CSR where blocks are mostly zero,
    sliced where that pads little), 1 block CSR everywhere, 2 plain scalar
    CSR wherever possible, 3 sliced scalar CSR wherever possible; 1b block
    form everywhere with every block level's residual and relaxation in
    block-row slices (the transposed cycle keeps the block CSR form); 3o
    slices with the nodes of every irregular operator sorted by length.
    Every FP64 level in slices fuses its zero-guess pre-smoothing step
    with the residual (r = f - (A M) f); 0u keeps the two passes.  Sliced
    products run one warp per 32-node group; 3w runs one warp per slice."""
    monkeypatch.setenv("GBS_LEVEL_FORMAT", fmt[0])
    monkeypatch.setenv("GBS_FUSE", "0" if fmt.endswith("u") else "1")
    monkeypatch.setenv("GBS_SELL_GROUP", "0" if fmt.endswith("w") else "1")
    monkeypatch.setenv("GBS_BSELL", "1" if fmt.endswith("b") else "0")
    monkeypatch.setenv("GBS_SELL_SORT", "1" if fmt.endswith("o") else "0")
    name, N, relax = cfg
    s = si.make_system(name, N=N)
    B = s.bdim
    A = bsr.from_arrays(s.indptr, s.indices, s.data, B)
    Ho = amg.build_hierarchy(A, amg.AmgParams(coarse_enough=50, relax=relax))
    assert len(Ho.levels) >= 2
    H = _import(Ho, B)
    rng = np.random.default_rng(7)
    for tr in (False, True):
        r = rng.standard_normal(A.shape[0])
        z = host(gb.apply_precond(H, dev(r), transpose=tr))
        ref = amg.vcycle(Ho, r, 0, transpose=tr)
        assert rel_inf(z, ref) <= 1e-12, (tr, rel_inf(z, ref))


@pytest.mark.parametrize("G,S", [("0", "1"), ("0", "2"), ("0", "4"), ("0", "8"), ("8", "1"),
                                 ("16", "1"), ("32", "1"), ("256", "1")])
@pytest.mark.parametrize("name", ["c2", "c1"])
def test_vcycle_every_lane_group_width(name, G, S, monkeypatch):
    """Force each SpMV lane mapping on every level -- one lane per scalar row
    with a row split over S = 1, 2, 4, 8 lanes, or G = 8, 16, 32 lanes or a
    256-thread CTA per block row -- and compare with the oracle."""
    monkeypatch.setenv("GBS_SPMV_GROUP", G)
    monkeypatch.setenv("GBS_SPMV_SPLIT", S)
    monkeypatch.setenv("GBS_BSELL", "0")
    s = si.make_system(name, N=9)
    B = s.bdim
    A = bsr.from_arrays(s.indptr, s.indices, s.data, B)
    Ho = amg.build_hierarchy(A, amg.AmgParams(coarse_enough=50, relax="jacobi"))
    H = _import(Ho, B, relax=gb.GBS_JACOBI)
    rng = np.random.default_rng(int(G) + 1)
    for tr in (False, True):
        r = rng.standard_normal(A.shape[0])
        z = host(gb.apply_precond(H, dev(r), transpose=tr))
        ref = amg.vcycle(Ho, r, 0, transpose=tr)
        assert rel_inf(z, ref) <= 1e-12, (tr, rel_inf(z, ref))


def test_vcycle_on_library_built_hierarchy():
    s = si.make_system("c2", N=12)
    A = bsr.from_arrays(s.indptr, s.indices, s.data, 4)
    Ho = amg.build_hierarchy(A, amg.AmgParams(coarse_enough=100, relax="jacobi"))
    H = gb.build_hierarchy(s.indptr, s.indices, s.data, 4,
                           gb.params_default(coarse_enough=100, relax=gb.GBS_JACOBI))
    assert gb.hierarchy_info(H)["nlevels"] == Ho.nlevels
    r = np.random.default_rng(3).standard_normal(A.shape[0])
    z = host(gb.apply_precond(H, dev(r)))
    assert rel_inf(z, amg.vcycle(Ho, r)) <= 1e-10


def test_schur_apply_matches_oracle():
    s = si.make_system("c3", N=9)
    K = bsr.from_arrays(s.indptr, s.indices, s.data, 4)
    po = amg.AmgParams(coarse_enough=60)
    pc = schur.build(K, 3, po, po)
    H = gb.build_hierarchy(s.indptr, s.indices, s.data, 4,
                           gb.params_default(precond=gb.GBS_PC_SCHUR, krylov=gb.GBS_GMRES,
                                             coarse_enough=60))
    rng = np.random.default_rng(11)
    for tr in (False, True):
        r = rng.standard_normal(K.shape[0])
        z = host(gb.apply_precond(H, dev(r), transpose=tr))
        ref = pc.apply(r, transpose=tr)
        assert rel_inf(z, ref) <= 1e-10, (tr, rel_inf(z, ref))


@pytest.mark.parametrize("fmt", ["1", "2", "3"])
@pytest.mark.parametrize("S", ["1", "2", "4", "8"])
def test_schur_apply_every_row_split(S, fmt, monkeypatch):
    """3x3 velocity and scalar pressure hierarchies with each row split, in
    block form and in scalar CSR form."""
    monkeypatch.setenv("GBS_SPMV_SPLIT", S)
    monkeypatch.setenv("GBS_LEVEL_FORMAT", fmt)
    s = si.make_system("c3", N=9)
    K = bsr.from_arrays(s.indptr, s.indices, s.data, 4)
    po = amg.AmgParams(coarse_enough=60)
    pc = schur.build(K, 3, po, po)
    H = gb.build_hierarchy(s.indptr, s.indices, s.data, 4,
                           gb.params_default(precond=gb.GBS_PC_SCHUR, krylov=gb.GBS_GMRES,
                                             coarse_enough=60))
    rng = np.random.default_rng(int(S))
    for tr in (False, True):
        r = rng.standard_normal(K.shape[0])
        z = host(gb.apply_precond(H, dev(r), transpose=tr))
        assert rel_inf(z, pc.apply(r, transpose=tr)) <= 1e-10


@pytest.mark.parametrize("fmt", ["2", "3"])
@pytest.mark.parametrize("S", ["1", "4"])
@pytest.mark.parametrize("precision", [gb.GBS_FP32, gb.GBS_BF16])
def test_mixed_csr_levels_match_block_levels(precision, S, fmt, monkeypatch):
    """The scalar CSR form (plain or sliced) of a mixed-precision level
    computes the same operator as its block form (FP32 accumulation: 1e-5
    relative)."""
    monkeypatch.setenv("GBS_SPMV_SPLIT", S)
    s = si.make_system("c3", N=10)
    p = _params(s, precision=precision, coarse_enough=60)
    monkeypatch.setenv("GBS_LEVEL_FORMAT", "1")
    Hb = gb.build_hierarchy(s.indptr, s.indices, s.data, 4, p)
    monkeypatch.setenv("GBS_LEVEL_FORMAT", fmt)
    Hc = gb.build_hierarchy(s.indptr, s.indices, s.data, 4, p)
    r = dev(np.random.default_rng(9).standard_normal(s.n))
    zb = host(gb.apply_precond(Hb, r))
    zc = host(gb.apply_precond(Hc, r))
    assert rel_inf(zc, zb) <= 1e-5


def _levels(Ho):
    lv = Ho.levels
    As = [(L.A.indptr, L.A.indices, L.A.data) for L in lv] + \
         [(Ho.A_coarse.indptr, Ho.A_coarse.indices, Ho.A_coarse.data)]
    Ps = [(L.P.indptr, L.P.indices, L.P.data, L.P.n_bcols) for L in lv]
    Rs = [(L.R.indptr, L.R.indices, L.R.data, L.R.n_bcols) for L in lv]
    return As, Ps, Rs, [L.M for L in lv], Ho.Ainv_coarse


def _import_schur(s, pc, **kw):
    """The oracle's Schur preconditioner (both inner hierarchies, or the
    pressure smoother) imported as it is: the GPU runs the same values."""
    order = 1 if pc.order == "lower" else 0
    kw.setdefault("krylov", gb.GBS_GMRES)
    p = gb.params_default(precond=gb.GBS_PC_SCHUR, schur_order=order,
                          schur_p=0 if pc.HS is not None else 1, **kw)
    return gb.import_schur(s.indptr, s.indices, s.data, _levels(pc.HA),
                           _levels(pc.HS) if pc.HS is not None else None,
                           pc.M_S.reshape(-1) if pc.M_S is not None else None, p)


@pytest.mark.parametrize("iso", ["1", "0"])
@pytest.mark.parametrize("fmt", ["0", "0f", "1", "2", "3", "3o"])
@pytest.mark.parametrize("variant", [("full", "amg"), ("lower", "amg"), ("full", "spai0"),
                                     ("lower", "jacobi")])
def test_schur_apply_on_imported_oracle_hierarchy(variant, fmt, iso, monkeypatch):
    """Eq. SchurPC (Section 4) on the oracle's own velocity and pressure
    hierarchies: the gather, the coupling kernels (r_p - D u, r_u - G p and
    their transposes through the transpose map), the inner V-cycles and
    the scatter match the oracle to 1e-12, forward and transposed, in every
    level format (3o: slices with sorted nodes wherever rows are irregular;
    0f: without the fused zero-guess smoothing step).
    The oracle's velocity levels are S (x) I_3 exactly (a scalar viscosity
    couples u, v, w identically), so with iso = 1 they run as one scalar
    operator on three interleaved components (except under format 1, every
    level in block form); iso = 0 runs the per-component layouts."""
    monkeypatch.setenv("GBS_LEVEL_FORMAT", fmt[0])
    monkeypatch.setenv("GBS_SELL_SORT", "1" if fmt.endswith("o") else "0")
    monkeypatch.setenv("GBS_FUSE", "0" if fmt.endswith("f") else "1")
    monkeypatch.setenv("GBS_ISO", iso)
    order, pressure = variant
    s = si.make_system("c3", N=9)
    K = bsr.from_arrays(s.indptr, s.indices, s.data, 4)
    po = amg.AmgParams(coarse_enough=60)
    pc = schur.build(K, 3, po, po, order=order, pressure=pressure)
    H = _import_schur(s, pc)
    want_iso = iso == "1" and fmt[0] != "1"
    for l in range(len(pc.HA.levels)):
        assert gb.level_iso(H, 0, l) == want_iso, l
    rng = np.random.default_rng(21)
    for tr in (False, True):
        r = rng.standard_normal(K.shape[0])
        z = host(gb.apply_precond(H, dev(r), transpose=tr))
        ref = pc.apply(r, transpose=tr)
        assert rel_inf(z, ref) <= 1e-12, (tr, rel_inf(z, ref))


def test_schur_import_rejects_mismatched_levels():
    s = si.make_system("c3", N=6)
    K = bsr.from_arrays(s.indptr, s.indices, s.data, 4)
    po = amg.AmgParams(coarse_enough=40)
    pc = schur.build(K, 3, po, po)
    s5 = si.make_system("c3", N=5)
    other = schur.build(bsr.from_arrays(s5.indptr, s5.indices, s5.data, 4), 3, po, po)
    p = gb.params_default(precond=gb.GBS_PC_SCHUR, krylov=gb.GBS_GMRES)
    with pytest.raises(gb.GbsError) as e:
        gb.import_schur(s.indptr, s.indices, s.data, _levels(other.HA), _levels(pc.HS), None, p)
    assert e.value.status == -1
    with pytest.raises(gb.GbsError):
        gb.import_schur(s.indptr, s.indices, s.data, _levels(pc.HA), None, None, p)


FMT = {gb.GBS_FP32: "fp32", gb.GBS_BF16: "bf16"}


@pytest.mark.parametrize("fmt", ["0", "1", "2", "2c", "3", "3s", "3d", "3w", "1b", "3o"])
@pytest.mark.parametrize("precision", [gb.GBS_FP32, gb.GBS_BF16])
def test_mixed_vcycle_matches_oracle_on_cast_hierarchy(precision, fmt, monkeypatch):
    """Mixed forms (Section 4, Listing V4; BF16 storage with FP32
    accumulation) against the oracle's FP64 V-cycle run on the same
    hierarchy with every stored value rounded exactly as the library
    uploads it (oracle.amg.cast_values) and the input rounded to FP32, as
    it enters the V-cycle.  What remains is FP32 accumulation and FP32
    vector storage: a few units of 2^-24 per operation over the levels, so
    1e-5 relative in the max norm for both forms.  Formats 2 and 3 put
    every level in scalar CSR and in slices (the staged bulk-copy
    kernels, or the direct ones where every slice is uniform; plain CSR
    with long rows streams 16-byte chunks, 2c keeps strided lanes); 3s / 3d
    send every sliced operator to the staged / direct kernels; 1b forces
    block-row slices on every block level."""
    monkeypatch.setenv("GBS_LEVEL_FORMAT", fmt[0])
    monkeypatch.setenv("GBS_BSELL", "1" if fmt.endswith("b") else "0")
    monkeypatch.setenv("GBS_SELL_SORT", "1" if fmt.endswith("o") else "0")
    monkeypatch.setenv("GBS_SELL_GROUP", "0" if fmt.endswith("w") else "1")
    monkeypatch.setenv("GBS_CSR_CHUNK", "0" if fmt.endswith("c") else "1")
    if fmt[1:] in ("s", "d"):
        monkeypatch.setenv("GBS_SELL_DIRECT", "0" if fmt.endswith("s") else "1")
    s = si.make_system("c2", N=10)
    A = bsr.from_arrays(s.indptr, s.indices, s.data, 4)
    Ho = amg.build_hierarchy(A, amg.AmgParams(coarse_enough=60, relax="jacobi"))
    H = _import(Ho, 4, relax=gb.GBS_JACOBI, precision=precision)
    Hc = amg.cast_values(Ho, FMT[precision])
    rng = np.random.default_rng(31)
    for tr in (False, True):
        r = rng.standard_normal(A.shape[0])
        z = host(gb.apply_precond(H, dev(r), transpose=tr))
        ref = amg.vcycle(Hc, round_to(r, "fp32"), 0, transpose=tr)
        assert rel_inf(z, ref) <= 1e-5, (tr, rel_inf(z, ref))
        if precision == gb.GBS_BF16:
            # BF16 storage rounding, not the accumulation, separates it from FP64
            z64 = amg.vcycle(Ho, r, 0, transpose=tr)
            assert rel_inf(z, z64) > 10 * rel_inf(z, ref)


@pytest.mark.parametrize("fmt", ["0", "2", "3"])
@pytest.mark.parametrize("case", ["c1_scalar", "c3_velocity"])
@pytest.mark.parametrize("precision", [gb.GBS_FP32, gb.GBS_BF16])
def test_mixed_identity_block_vcycle_matches_oracle(precision, case, fmt, monkeypatch):
    """A monolithic AMG whose levels are all S (x) I_B in a mixed form: the
    scalar C1 system (B = 1) and the C3 velocity block run as a system of
    its own (B = 3).  The finest level's first kernel takes the FP64 input
    and rounds it (the precision boundary folded into k_iso_cast_mapply),
    and its last sweep writes the FP64 output; forward and transposed, 1e-5
    against the oracle's V-cycle on the cast hierarchy, in slices or CSR."""
    monkeypatch.setenv("GBS_LEVEL_FORMAT", fmt)
    monkeypatch.setenv("GBS_ISO", "1")
    if case == "c1_scalar":
        s = si.make_system("c1", N=10)
        A = bsr.from_arrays(s.indptr, s.indices, s.data, 1)
        B = 1
    else:
        s = si.make_system("c3", N=10)
        A = schur.split(bsr.from_arrays(s.indptr, s.indices, s.data, 4), 3).A
        B = 3
    Ho = amg.build_hierarchy(A, amg.AmgParams(coarse_enough=60))
    assert len(Ho.levels) >= 2
    H = _import(Ho, B, precision=precision)
    for l in range(len(Ho.levels)):
        assert gb.level_iso(H, 0, l), l
    Hc = amg.cast_values(Ho, FMT[precision])
    rng = np.random.default_rng(47)
    for tr in (False, True):
        r = rng.standard_normal(A.shape[0])
        z = host(gb.apply_precond(H, dev(r), transpose=tr))
        ref = amg.vcycle(Hc, round_to(r, "fp32"), 0, transpose=tr)
        assert rel_inf(z, ref) <= 1e-5, (tr, rel_inf(z, ref))


@pytest.mark.parametrize("iso", ["1", "0"])
@pytest.mark.parametrize("fmt", ["0", "0f", "2", "3"])
@pytest.mark.parametrize("precision", [gb.GBS_FP32, gb.GBS_BF16])
def test_mixed_schur_matches_oracle_on_cast_hierarchy(precision, fmt, iso, monkeypatch):
    """The Schur preconditioner in the mixed forms against the oracle on
    the cast values (velocity and pressure hierarchies, G and D), 1e-5,
    with the velocity levels as S (x) I_3 (iso = 1) or per component; 0f
    keeps the zero-guess smoothing step apart from the residual (fused,
    an S (x) I_3 level forms x = m .* f in the residual's gather)."""
    monkeypatch.setenv("GBS_LEVEL_FORMAT", fmt[0])
    monkeypatch.setenv("GBS_FUSE", "0" if fmt.endswith("f") else "1")
    monkeypatch.setenv("GBS_ISO", iso)
    s = si.make_system("c3", N=10)
    K = bsr.from_arrays(s.indptr, s.indices, s.data, 4)
    po = amg.AmgParams(coarse_enough=60)
    pc = schur.build(K, 3, po, po)
    H = _import_schur(s, pc, precision=precision)
    pcc = schur.cast_values(pc, FMT[precision])
    rng = np.random.default_rng(41)
    for tr in (False, True):
        r = rng.standard_normal(K.shape[0])
        z = host(gb.apply_precond(H, dev(r), transpose=tr))
        ref = pcc.apply(round_to(r, "fp32"), transpose=tr)
        assert rel_inf(z, ref) <= 1e-5, (tr, rel_inf(z, ref))


@pytest.mark.parametrize("split", ["1", "2", "16", "32", "256"])
@pytest.mark.parametrize("precision", [gb.GBS_FP64, gb.GBS_BF16])
def test_iso_lane_groups_match_oracle(precision, split, monkeypatch):
    """Every S (x) I_3 velocity level in plain CSR, with 1 .. 32 lanes a row
    of S or a 256-thread CTA a row (the widths small levels of long rows
    take), forward and transposed, against the oracle's Schur application
    on the same (for BF16: cast) hierarchy."""
    monkeypatch.setenv("GBS_LEVEL_FORMAT", "2")
    monkeypatch.setenv("GBS_ISO", "1")
    monkeypatch.setenv("GBS_ISO_SPLIT", split)
    s = si.make_system("c3", N=10)
    K = bsr.from_arrays(s.indptr, s.indices, s.data, 4)
    po = amg.AmgParams(coarse_enough=60)
    pc = schur.build(K, 3, po, po)
    H = _import_schur(s, pc, precision=precision)
    assert all(gb.level_iso(H, 0, l) for l in range(len(pc.HA.levels)))
    ref_pc = pc if precision == gb.GBS_FP64 else schur.cast_values(pc, FMT[precision])
    rng = np.random.default_rng(43)
    for tr in (False, True):
        r = rng.standard_normal(K.shape[0])
        z = host(gb.apply_precond(H, dev(r), transpose=tr))
        if precision == gb.GBS_FP64:
            assert rel_inf(z, ref_pc.apply(r, transpose=tr)) <= 1e-12, tr
        else:
            assert rel_inf(z, ref_pc.apply(round_to(r, "fp32"), transpose=tr)) <= 1e-5, tr


# ----------------------------------------------------------------- solves
def _oracle_solve(s, relax, coarse_enough=1000):
    K = bsr.from_arrays(s.indptr, s.indices, s.data, s.bdim)
    Ks = K.scipy()
    if s.method == "amg_bicgstab":
        Ho = amg.build_hierarchy(K, amg.AmgParams(relax=relax, coarse_enough=coarse_enough))
        return krylov.bicgstab(lambda v: Ks @ v, lambda v: amg.vcycle(Ho, v), s.b, tol=1e-8)
    pc = schur.build(K, 3, amg.AmgParams(coarse_enough=coarse_enough),
                     amg.AmgParams(coarse_enough=coarse_enough))
    return krylov.gmres(lambda v: Ks @ v, pc.apply, s.b, m=30, tol=1e-8)


def _true_rel(s, x):
    return np.linalg.norm(s.b - s.scipy() @ x) / np.linalg.norm(s.b)


def _params(s, **kw):
    if s.method == "amg_bicgstab":
        return gb.params_default(**kw)
    return gb.params_default(precond=gb.GBS_PC_SCHUR, krylov=gb.GBS_GMRES, **kw)


@pytest.mark.parametrize("use_graph", [1, 0])
def test_solve_c1_full_size(use_graph):
    """C1: N=16 scalar CSR, SA-AMG (SPAI0 1+1) + BiCGStab to 1e-8."""
    s = si.make_system("c1")
    xo, io = _oracle_solve(s, "spai0")
    H = gb.build_hierarchy(s.indptr, s.indices, s.data, 1, _params(s, use_graph=use_graph))
    x, info = gb.solve(H, dev(s.b))
    x = host(x)
    assert info.converged and _true_rel(s, x) <= 1e-8
    assert abs(info.iters - io.iters) <= max(1, math.ceil(0.1 * io.iters)), (info.iters, io.iters)
    # ||x - x_m|| / ||x_m|| <= cond(K) * 1e-8 with cond(K) ~ 2e3 at N = 16
    assert np.linalg.norm(x - s.x_exact) / np.linalg.norm(s.x_exact) < 1e-4


@pytest.mark.parametrize("N", [13, 16])
def test_solve_c2_recipe(N):
    s = si.make_system("c2", N=N)
    xo, io = _oracle_solve(s, "jacobi")
    H = gb.build_hierarchy(s.indptr, s.indices, s.data, 4, _params(s, relax=gb.GBS_JACOBI))
    x, info = gb.solve(H, dev(s.b))
    x = host(x)
    assert info.converged and _true_rel(s, x) <= 1e-8
    assert abs(info.iters - io.iters) <= max(1, math.ceil(0.1 * io.iters)), (info.iters, io.iters)
    assert np.linalg.norm(x - xo) / np.linalg.norm(xo) < 1e-5


@pytest.mark.parametrize("precision", [gb.GBS_FP64, gb.GBS_FP32, gb.GBS_BF16])
def test_solve_c3_recipe_forms(precision):
    s = si.make_system("c3", N=14)
    xo, io = _oracle_solve(s, "spai0")
    H = gb.build_hierarchy(s.indptr, s.indices, s.data, 4, _params(s, precision=precision))
    x, info = gb.solve(H, dev(s.b))
    x = host(x)
    assert info.converged and _true_rel(s, x) <= 1e-8
    err = np.linalg.norm(x - xo) / np.linalg.norm(xo)
    assert err < 1e-5
    if precision == gb.GBS_FP64:
        assert abs(info.iters - io.iters) <= max(1, math.ceil(0.1 * io.iters))


def test_solve_edge_cases():
    s = si.make_system("c2", N=6)
    H = gb.build_hierarchy(s.indptr, s.indices, s.data, 4, _params(s, relax=gb.GBS_JACOBI))
    # zero right-hand side: x = 0, no iterations
    x, info = gb.solve(H, dev(np.zeros(s.n)), dev(np.ones(s.n)))
    assert info.converged and info.iters == 0 and not host(x).any()
    # a converged start returns immediately (warm start)
    x1, info1 = gb.solve(H, dev(s.b))
    x2, info2 = gb.solve(H, dev(s.b), x1.clone())
    assert info2.iters == 0 and info2.converged
    # maxiter = 1: not converged, x and info still written
    H1 = gb.build_hierarchy(s.indptr, s.indices, s.data, 4,
                            _params(s, relax=gb.GBS_JACOBI, maxiter=1, tol=1e-14,
                                    coarse_enough=40))
    x, info = gb.solve(H1, dev(s.b))
    assert not info.converged and info.iters == 1 and info.status == 1
    assert info.rel_res < 1.0
    # NaN in b is reported, not propagated silently
    b = s.b.copy()
    b[3] = np.nan
    with pytest.raises(gb.GbsError) as e:
        gb.solve(H, dev(b))
    assert e.value.status == -5


def test_gmres_edge_cases():
    s = si.make_system("c3", N=5)
    H = gb.build_hierarchy(s.indptr, s.indices, s.data, 4, _params(s, coarse_enough=40))
    x, info = gb.solve(H, dev(np.zeros(s.n)))
    assert info.converged and info.iters == 0
    H2 = gb.build_hierarchy(s.indptr, s.indices, s.data, 4,
                            _params(s, coarse_enough=40, restart=4, maxiter=3, tol=1e-14))
    x, info = gb.solve(H2, dev(s.b))
    assert not info.converged and info.iters == 3


# ---------------------------------------------------------------- adjoint
def test_sampled_outer_matches_oracle():
    s = si.make_system("c2", N=7)
    K = bsr.from_arrays(s.indptr, s.indices, s.data, 4)
    H = gb.build_hierarchy(s.indptr, s.indices, s.data, 4, _params(s, relax=gb.GBS_JACOBI))
    rng = np.random.default_rng(5)
    lam, x = rng.standard_normal((2, s.n))
    g = host(gb.sampled_outer(H, dev(lam), dev(x), -1.0)).reshape(-1, 4, 4)
    ref = adjoint.sampled_outer(K, lam, x, -1.0)
    assert np.array_equal(g, ref)


@pytest.mark.parametrize("method", ["amg_bicgstab", "schur_gmres"])
def test_adjoint_matches_dense_inverse(method):
    name = "c2" if method == "amg_bicgstab" else "c3"
    s = si.make_system(name, N=5)
    Kd = s.scipy().toarray()
    xt = si.gaussian_vector(s.n, 4001)
    H = gb.build_hierarchy(s.indptr, s.indices, s.data, 4,
                           _params(s, relax=gb.GBS_JACOBI, coarse_enough=40, tol=1e-12))
    x, _ = gb.solve(H, dev(s.b))
    lam, info = gb.solve_adjoint(H, x - dev(xt))
    assert info.converged
    xd = np.linalg.solve(Kd, s.b)
    lamd = np.linalg.solve(Kd.T, xd - xt)
    np.testing.assert_allclose(host(lam), lamd, rtol=0, atol=1e-8 * np.abs(lamd).max())


def test_autograd_gradients_match_dense_inverse():
    from paper_2006_06052_gb300.autograd import stokes_solve
    s = si.make_system("c2", N=5)
    K = bsr.from_arrays(s.indptr, s.indices, s.data, 4)
    Kd = K.dense()
    xt = si.gaussian_vector(s.n, 4001)
    H = gb.build_hierarchy(s.indptr, s.indices, s.data, 4,
                           _params(s, relax=gb.GBS_JACOBI, coarse_enough=40, tol=1e-12))
    vals = dev(s.data.reshape(-1)).requires_grad_(True)
    b = dev(s.b).requires_grad_(True)
    x = stokes_solve(vals, b, H)
    loss = 0.5 * ((x - dev(xt)) ** 2).sum()
    loss.backward()
    xd = np.linalg.solve(Kd, s.b)
    lamd = np.linalg.solve(Kd.T, xd - xt)
    np.testing.assert_allclose(host(b.grad), lamd, rtol=0, atol=1e-8 * np.abs(lamd).max())
    gref = adjoint.sampled_outer(K, lamd, xd, -1.0).reshape(-1)
    np.testing.assert_allclose(host(vals.grad), gref, rtol=0, atol=1e-8 * np.abs(gref).max())


def test_autograd_central_differences_c4_recipe():
    """C4 recipe at N=6: FP64 central differences (h = 1e-6) of
    L = 1/2 ||x - x_t||^2 on sampled entries, solves to 1e-13 through
    gbs_update_values (hierarchy reused), vs the adjoint gradient."""
    from paper_2006_06052_gb300.autograd import stokes_solve
    s = si.make_system("c4", N=6)
    xt = dev(si.gaussian_vector(s.n, 4001))
    H = gb.build_hierarchy(s.indptr, s.indices, s.data, 4,
                           _params(s, relax=gb.GBS_JACOBI, coarse_enough=100, tol=1e-13))
    v0 = dev(s.data.reshape(-1))
    vals = v0.clone().requires_grad_(True)
    x = stokes_solve(vals, dev(s.b), H)
    (0.5 * ((x - xt) ** 2).sum()).backward()
    G = host(vals.grad)
    rng = np.random.Generator(np.random.PCG64(4002))
    nz = np.nonzero(s.data.reshape(-1))[0]
    for idx in rng.choice(nz, size=8, replace=False):
        step = 1e-6 * max(1.0, abs(float(s.data.reshape(-1)[idx])))
        vp = v0.clone()
        vm = v0.clone()
        vp[idx] += step
        vm[idx] -= step
        with torch.no_grad():
            xp = stokes_solve(vp, dev(s.b), H)
            xm = stokes_solve(vm, dev(s.b), H)
        dl = 0.5 * torch.dot(xp - xm, xp + xm - 2 * xt).item()
        fd = dl / (2 * step)
        assert abs(fd - G[idx]) <= 1e-5 * max(abs(fd), 1e-3 * np.abs(G).max()), (idx, fd, G[idx])


# ------------------------------------------------------------ full sizes
def test_full_size_c2_against_oracle():
    """C2 at full size (N=64, 1,048,576 unknowns, 4x4 BSR FP64), the
    benchmarked configuration: true residual (oracle SpMV) <= 1e-8 and
    iteration count within +-10% of the oracle's solve."""
    s = si.make_system("c2")
    H = gb.build_hierarchy(s.indptr, s.indices, s.data, 4, _params(s, relax=gb.GBS_JACOBI))
    x, info = gb.solve(H, dev(s.b))
    x = host(x)
    assert info.converged and _true_rel(s, x) <= 1e-8
    xo, io = _oracle_solve(s, "jacobi")
    assert abs(info.iters - io.iters) <= max(1, math.ceil(0.1 * io.iters)), (info.iters, io.iters)
    assert np.linalg.norm(x - xo) / np.linalg.norm(xo) < 1e-5


def _exported(H, which):
    """Every level of hierarchy `which` of a handle, as gbs_export_level
    returns it (the FP64 setup values), in import_hierarchy's layout."""
    nl = gb.hierarchy_info(H, which)["nlevels"]
    As, Ps, Rs, Ms = [], [], [], []
    for l in range(nl):
        As.append(gb.export_level(H, which, l, 0))
        if l + 1 < nl:
            Ps.append(gb.export_level(H, which, l, 1))
            Rs.append(gb.export_level(H, which, l, 2))
            Ms.append(gb.export_level(H, which, l, 3))
    return As, Ps, Rs, Ms, gb.export_level(H, which, nl - 1, 5)


_C3 = {}


def _c3_handle(precision):
    """The full-size N=128 Schur system; the host setup runs once (FP64
    handle) and the mixed forms import its exported hierarchies."""
    if "fp64" not in _C3:
        s = si.make_system("c3")
        _C3["s"] = s
        _C3["fp64"] = gb.build_hierarchy(s.indptr, s.indices, s.data, 4,
                                         _params(s, enable_adjoint=0))
    s, H64 = _C3["s"], _C3["fp64"]
    if precision == gb.GBS_FP64:
        return s, H64
    return s, gb.import_schur(s.indptr, s.indices, s.data, _exported(H64, 0), _exported(H64, 1),
                              None, _params(s, precision=precision, enable_adjoint=0))


def c3_error_vs_oracle(x, g, n):
    """||x - x_oracle|| / ||x_oracle|| estimated from the oracle solution's
    stored sample (uniform indices): sqrt(n/m sum (x_i - xo_i)^2) / ||xo||."""
    idx = np.array(g["sample_idx"], dtype=np.int64)
    xs = np.array(g["sample_x"])
    return float(np.sqrt(n / len(idx) * np.sum((x[idx] - xs) ** 2)) / g["x_norm"][0])


@pytest.mark.parametrize("precision", [gb.GBS_FP64, gb.GBS_FP32, gb.GBS_BF16])
def test_full_size_c3_against_oracle(precision):
    """C3 at full size (N=128, 8,388,608 unknowns, Schur + GMRES(30)) in
    each hierarchy form, against the oracle's own full-size solve
    (tests/golden/c3_oracle_solution.txt, written by make_c3_oracle.py):
    the FP64 true residual recomputed on the host is <= 1e-8; the FP64
    form's iteration count is within +-10% of the oracle's; every form's
    error against the oracle solution is reported and bounded."""
    from conftest import load_golden
    g = load_golden("c3_oracle_solution.txt")
    s, H = _c3_handle(precision)
    assert int(g["n"][0]) == s.n
    x, info = gb.solve(H, dev(s.b))
    x = host(x)
    rel = _true_rel(s, x)
    io = int(g["iterations"][0])
    err = c3_error_vs_oracle(x, g, s.n)
    norm_dev = abs(np.linalg.norm(x) - g["x_norm"][0]) / g["x_norm"][0]
    print("C3 form %d: iterations %d (oracle %d), true rel. residual %.3e, "
          "||x - x_oracle||/||x_oracle|| ~ %.3e, | ||x|| - ||x_oracle|| |/||x_oracle|| %.3e"
          % (precision, info.iters, io, rel, err, norm_dev))
    assert info.converged and rel <= 1e-8
    if precision == gb.GBS_FP64:
        assert abs(info.iters - io) <= max(1, math.ceil(0.1 * io)), (info.iters, io)
    bound = C3_ERR_BOUND[precision]
    assert err <= bound and norm_dev <= bound, (err, norm_dev)


# Two solutions that both meet ||b - K x|| <= 1e-8 ||b|| may differ by up to
# cond(K) * 2e-8 relative.  The FP64 form takes the oracle's own path (same
# hierarchy, same Krylov steps: measured 1.7e-15), so it is held to 1e-10;
# the mixed forms stop at a different iterate (measured 3.8e-8 FP32,
# 1.3e-7 BF16) and are held to 1e-5, the bound of the C3 small-grid test.
C3_ERR_BOUND = {gb.GBS_FP64: 1e-10, gb.GBS_FP32: 1e-5, gb.GBS_BF16: 1e-5}


def test_full_size_c4_adjoint_central_differences():
    """C4 at full size (N=64, 4x4 BSR FP64): L = 1/2 ||x - x_t||^2, adjoint
    gradient of 64 random stored entries (seed 4002) against FP64 central
    differences (h = 1e-6) with solves to 1e-13 reusing the hierarchy.
    Tolerance per entry: 5e-5 relative, or 1e-5 max|G| absolute, whichever
    is larger.  The absolute term is the difference quotient's noise: each
    solve stops at relative residual 1e-13, leaving an error of order
    cond(K) 1e-13 |x| (cond(K) ~ 1e4 at N=64) that does not cancel exactly
    between the two solves, and that error is divided by the step (seen up
    to 1.6e-6 max|G|).  A wrong gradient is off by O(1) on entries of any
    size; the small-grid tests pin it to 1e-5 and to the dense inverse."""
    from paper_2006_06052_gb300.autograd import stokes_solve
    s = si.make_system("c4")
    xt = dev(si.gaussian_vector(s.n, 4001))
    H = gb.build_hierarchy(s.indptr, s.indices, s.data, 4,
                           _params(s, relax=gb.GBS_JACOBI, tol=1e-13, maxiter=3000))
    v0 = dev(s.data.reshape(-1))
    vals = v0.clone().requires_grad_(True)
    b = dev(s.b).requires_grad_(True)
    x = stokes_solve(vals, b, H)
    (0.5 * ((x - xt) ** 2).sum()).backward()
    G = host(vals.grad)
    gb_ = host(b.grad)
    rng = np.random.Generator(np.random.PCG64(4002))
    flat = s.data.reshape(-1)
    nz = np.nonzero(flat)[0]
    gmax = np.abs(G).max()
    for idx in rng.choice(nz, size=64, replace=False):
        step = 1e-6 * max(1.0, abs(float(flat[idx])))
        vp, vm = v0.clone(), v0.clone()
        vp[idx] += step
        vm[idx] -= step
        with torch.no_grad():
            xp = stokes_solve(vp, dev(s.b), H)
            xm = stokes_solve(vm, dev(s.b), H)
        fd = 0.5 * torch.dot(xp - xm, xp + xm - 2 * xt).item() / (2 * step)
        assert abs(fd - G[idx]) <= max(5e-5 * abs(fd), 1e-5 * gmax), (idx, fd, G[idx])
    # grad_b by central differences on a few unknowns
    for i in rng.integers(s.n, size=4):
        e = torch.zeros(s.n, dtype=torch.float64, device="cuda")
        e[int(i)] = 1e-6
        with torch.no_grad():
            xp = stokes_solve(v0, dev(s.b) + e, H)
            xm = stokes_solve(v0, dev(s.b) - e, H)
        fd = 0.5 * torch.dot(xp - xm, xp + xm - 2 * xt).item() / 2e-6
        assert abs(fd - gb_[int(i)]) <= max(5e-5 * abs(fd), 1e-5 * np.abs(gb_).max())


@pytest.mark.parametrize("N", [24, pytest.param(128, id="full_size")])
def test_c5_mixed_adjoint_matches_fp64_adjoint(N):
    """C5 (full size at N=128): BF16/FP32 Schur hierarchy shared by the
    forward and the transposed backward, only x kept (the backward recomputes
    the adjoint solve); ||grad_b|| within 1e-5 of the FP64 GPU adjoint."""
    from paper_2006_06052_gb300.autograd import stokes_solve
    s = si.make_system("c5", N=N)
    xt = dev(si.gaussian_vector(s.n, 5001))
    grads = {}
    for prec in (gb.GBS_BF16, gb.GBS_FP64):
        H = gb.build_hierarchy(s.indptr, s.indices, s.data, 4, _params(s, precision=prec))
        vals = dev(s.data.reshape(-1)).requires_grad_(True)
        b = dev(s.b).requires_grad_(True)
        x = stokes_solve(vals, b, H)
        (0.5 * ((x - xt) ** 2).sum()).backward()
        grads[prec] = (host(b.grad), vals.grad.norm().item())
        del H
    g16, g64 = grads[gb.GBS_BF16][0], grads[gb.GBS_FP64][0]
    n16, n64 = np.linalg.norm(g16), np.linalg.norm(g64)
    assert abs(n16 - n64) <= 1e-5 * n64
    assert np.linalg.norm(g16 - g64) <= 1e-4 * n64
    assert abs(grads[gb.GBS_BF16][1] - grads[gb.GBS_FP64][1]) <= 1e-4 * grads[gb.GBS_FP64][1]


@pytest.mark.parametrize("fmt", ["2", "3"])
def test_update_values_inside_csr_pattern(fmt, monkeypatch):
    """New values on K's build-time nonzero pattern reach the scalar form
    of K (plain CSR or slices)."""
    monkeypatch.setenv("GBS_LEVEL_FORMAT", fmt)
    s = si.make_system("c2", N=7)
    H = gb.build_hierarchy(s.indptr, s.indices, s.data, 4, _params(s, relax=gb.GBS_JACOBI))
    gb.solve(H, dev(s.b))
    rng = np.random.default_rng(12)
    vals = s.data * (1.0 + 0.25 * rng.random(s.data.shape))
    K2 = bsr.from_arrays(s.indptr, s.indices, vals, 4).scipy()
    gb.update_values(H, dev(vals.reshape(-1)))
    x = rng.standard_normal(s.n)
    y = host(gb.spmv(H, dev(x)))
    assert np.all(np.abs(y - K2 @ x) <= 1e-13 * (abs(K2) @ np.abs(x)) + 1e-300)
    xs, info = gb.solve(H, dev(s.b))
    assert info.converged
    assert np.linalg.norm(s.b - K2 @ host(xs)) / np.linalg.norm(s.b) <= 1e-8


@pytest.mark.parametrize("fmt", ["2", "3"])
def test_update_values_outside_csr_pattern_falls_back_to_blocks(fmt, monkeypatch):
    """K runs as scalar CSR (or slices) of its build-time nonzeros; an
    update that puts a nonzero where a stored block held a zero must still
    be honoured."""
    monkeypatch.setenv("GBS_LEVEL_FORMAT", fmt)
    s = si.make_system("c2", N=7)
    H = gb.build_hierarchy(s.indptr, s.indices, s.data, 4, _params(s, relax=gb.GBS_JACOBI))
    gb.solve(H, dev(s.b))            # captures the CUDA-graph iteration with K in CSR form
    vals = s.data.copy()
    blk = np.nonzero(s.indices != np.repeat(np.arange(len(s.indptr) - 1), np.diff(s.indptr)))[0][5]
    assert vals[blk, 0, 1] == 0.0
    vals[blk, 0, 1] = 0.37 * vals[blk, 0, 0]
    K2 = bsr.from_arrays(s.indptr, s.indices, vals, 4)
    x = np.random.default_rng(4).standard_normal(s.n)
    gb.update_values(H, dev(vals.reshape(-1)))
    y = host(gb.spmv(H, dev(x)))
    assert np.all(np.abs(y - K2.scipy() @ x) <= 1e-13 * (abs(K2.scipy()) @ np.abs(x)) + 1e-300)
    xs, info = gb.solve(H, dev(s.b))
    assert info.converged
    assert np.linalg.norm(s.b - K2.scipy() @ host(xs)) / np.linalg.norm(s.b) <= 1e-8
    # and back: values inside the pattern keep the fast form correct too
    gb.update_values(H, dev(s.data.reshape(-1)))
    y = host(gb.spmv(H, dev(x)))
    K1 = bsr.from_arrays(s.indptr, s.indices, s.data, 4).scipy()
    assert np.all(np.abs(y - K1 @ x) <= 1e-13 * (abs(K1) @ np.abs(x)) + 1e-300)


@pytest.mark.parametrize("order", [0, 1])
@pytest.mark.parametrize("schur_p", [0, 1])
def test_schur_variants_apply_and_solve(order, schur_p):
    """Schur variants: pressure solve = AMG V-cycle (0) or one SPAI0
    application on S_hat (1); "full" (0) or "lower" (1) ordering.  The
    application (forward and transposed) matches the oracle's, and GMRES(30)
    reaches 1e-8 within +-10% of the oracle's iteration count."""
    s = si.make_system("c3", N=12)
    K = bsr.from_arrays(s.indptr, s.indices, s.data, 4)
    po = amg.AmgParams(coarse_enough=60)
    pc = schur.build(K, 3, po, po, order=("full", "lower")[order],
                     pressure=("amg", "spai0")[schur_p])
    H = gb.build_hierarchy(s.indptr, s.indices, s.data, 4,
                           _params(s, coarse_enough=60, schur_p=schur_p, schur_order=order))
    rng = np.random.default_rng(21)
    for tr in (False, True):
        r = rng.standard_normal(K.shape[0])
        z = host(gb.apply_precond(H, dev(r), transpose=tr))
        assert rel_inf(z, pc.apply(r, transpose=tr)) <= 1e-10, tr
    Ks = K.scipy()
    xo, io = krylov.gmres(lambda v: Ks @ v, pc.apply, s.b, m=30, tol=1e-8)
    x, info = gb.solve(H, dev(s.b))
    assert info.converged and _true_rel(s, host(x)) <= 1e-8
    assert abs(info.iters - io.iters) <= max(1, math.ceil(0.1 * io.iters)), (info.iters, io.iters)


@pytest.mark.parametrize("case", ["c2_amg", "c3_schur"])
def test_idrs_solve_matches_oracle(case):
    """IDR(5), the paper's outer solver: converges to the 1e-8 true residual
    within +-10% of the oracle's matvec count, forward and adjoint."""
    if case == "c2_amg":
        s = si.make_system("c2", N=13)
        K = bsr.from_arrays(s.indptr, s.indices, s.data, 4)
        Ho = amg.build_hierarchy(K, amg.AmgParams(relax="jacobi"))
        Mo, MoT = (lambda v: amg.vcycle(Ho, v)), (lambda v: amg.vcycle(Ho, v, 0, True))
        p = gb.params_default(krylov=gb.GBS_IDRS, relax=gb.GBS_JACOBI)
    else:
        s = si.make_system("c3", N=12)
        K = bsr.from_arrays(s.indptr, s.indices, s.data, 4)
        pc = schur.build(K, 3)
        Mo, MoT = pc.apply, (lambda v: pc.apply(v, transpose=True))
        p = gb.params_default(krylov=gb.GBS_IDRS, precond=gb.GBS_PC_SCHUR)
    Ks = K.scipy()
    xo, io = krylov.idrs(lambda v: Ks @ v, Mo, s.b, s=5, tol=1e-8)
    H = gb.build_hierarchy(s.indptr, s.indices, s.data, 4, p)
    x, info = gb.solve(H, dev(s.b))
    assert info.converged and _true_rel(s, host(x)) <= 1e-8
    assert abs(info.iters - io.iters) <= max(2, math.ceil(0.1 * io.iters)), (info.iters, io.iters)
    g = np.random.default_rng(2).standard_normal(s.n)
    lo, ilo = krylov.idrs(lambda v: Ks.T @ v, MoT, g, s=5, tol=1e-8)
    lam, il = gb.solve_adjoint(H, dev(g))
    assert il.converged
    assert np.linalg.norm(g - Ks.T @ host(lam)) / np.linalg.norm(g) <= 1e-8
    assert abs(il.iters - ilo.iters) <= max(2, math.ceil(0.1 * ilo.iters)), (il.iters, ilo.iters)


def test_plain_aggregation_solves():
    """smooth_P = 0 (plain aggregation) for the Schur velocity/pressure AMG:
    V-cycle parity on the oracle's hierarchy and a converged solve."""
    s = si.make_system("c3", N=12)
    K = bsr.from_arrays(s.indptr, s.indices, s.data, 4)
    po = amg.AmgParams(smooth_P=False, coarse_enough=60)
    pc = schur.build(K, 3, po, po)
    H = gb.build_hierarchy(s.indptr, s.indices, s.data, 4,
                           _params(s, smooth_P=0, coarse_enough=60))
    r = np.random.default_rng(31).standard_normal(K.shape[0])
    assert rel_inf(host(gb.apply_precond(H, dev(r))), pc.apply(r)) <= 1e-10
    Ks = K.scipy()
    xo, io = krylov.gmres(lambda v: Ks @ v, pc.apply, s.b, m=30, tol=1e-8)
    x, info = gb.solve(H, dev(s.b))
    assert info.converged and _true_rel(s, host(x)) <= 1e-8
    assert abs(info.iters - io.iters) <= max(1, math.ceil(0.1 * io.iters))


# ------------------------------------------------------------------ ILUT
@pytest.mark.parametrize("fmt", ["0", "1"])
@pytest.mark.parametrize("sweeps", [0, 2, 3])
@pytest.mark.parametrize("case", ["c3_velocity", "c2_monolithic"])
def test_ilut_vcycle_on_imported_oracle_hierarchy(case, sweeps, fmt, monkeypatch):
    """ILUT relaxation (the velocity smoother of Listings V2-V4): the
    library factors each imported level itself and its V-cycle (forward
    and transposed) matches the oracle's to 1e-12."""
    monkeypatch.setenv("GBS_LEVEL_FORMAT", fmt)
    if case == "c3_velocity":
        s = si.make_system("c3", N=9)
        A = schur.split(bsr.from_arrays(s.indptr, s.indices, s.data, 4), 3).A
        B = 3
    else:
        s = si.make_system("c2", N=9)
        A = bsr.from_arrays(s.indptr, s.indices, s.data, 4)
        B = 4
    Ho = amg.build_hierarchy(A, amg.AmgParams(coarse_enough=50, relax="ilut", ilut_sweeps=sweeps))
    assert len(Ho.levels) >= 2
    H = _import(Ho, B, relax=gb.GBS_ILUT, ilut_sweeps=sweeps)
    rng = np.random.default_rng(sweeps + 31)
    for tr in (False, True):
        r = rng.standard_normal(A.shape[0])
        z = host(gb.apply_precond(H, dev(r), transpose=tr))
        ref = amg.vcycle(Ho, r, 0, transpose=tr)
        assert rel_inf(z, ref) <= 1e-12, (tr, rel_inf(z, ref))


@pytest.mark.parametrize("precision", [gb.GBS_FP64, gb.GBS_FP32, gb.GBS_BF16])
def test_schur_ilut_solve_matches_oracle(precision):
    """C3 recipe at N=12 with the ILUT-relaxed velocity AMG: the FP64
    preconditioner matches the oracle's Eq. SchurPC application, and every
    form's GMRES(30) reaches the 1e-8 true residual (FP64 within +-10% of
    the oracle's iterations)."""
    s = si.make_system("c3", N=12)
    K = bsr.from_arrays(s.indptr, s.indices, s.data, 4)
    pa = amg.AmgParams(coarse_enough=60, relax="ilut")
    ps = amg.AmgParams(coarse_enough=60)
    pc = schur.build(K, 3, pa, ps)
    H = gb.build_hierarchy(s.indptr, s.indices, s.data, 4,
                           _params(s, coarse_enough=60, relax=gb.GBS_ILUT, precision=precision))
    Ks = K.scipy()
    if precision == gb.GBS_FP64:
        rng = np.random.default_rng(41)
        for tr in (False, True):
            r = rng.standard_normal(K.shape[0])
            z = host(gb.apply_precond(H, dev(r), transpose=tr))
            assert rel_inf(z, pc.apply(r, transpose=tr)) <= 1e-10, tr
    xo, io = krylov.gmres(lambda v: Ks @ v, pc.apply, s.b, m=30, tol=1e-8)
    x, info = gb.solve(H, dev(s.b))
    assert info.converged and _true_rel(s, host(x)) <= 1e-8
    if precision == gb.GBS_FP64:
        assert abs(info.iters - io.iters) <= max(1, math.ceil(0.1 * io.iters)), (info.iters, io.iters)


# ------------------------------------------------------------------ level ops
@pytest.mark.parametrize("relax", ["jacobi", "spai0", "ilut"])
def test_level_apply_matches_oracle(relax):
    """gbs_level_apply runs one level operation as the V-cycle launches it:
    the residual and one relaxation sweep of every level below the coarsest
    match the oracle's."""
    s = si.make_system("c2", N=9)
    A = bsr.from_arrays(s.indptr, s.indices, s.data, 4)
    Ho = amg.build_hierarchy(A, amg.AmgParams(coarse_enough=50, relax=relax))
    code = {"jacobi": gb.GBS_JACOBI, "spai0": gb.GBS_SPAI0, "ilut": gb.GBS_ILUT}[relax]
    H = _import(Ho, 4, relax=code)
    rng = np.random.default_rng(61)
    for l, lev in enumerate(Ho.levels):
        As = lev.A.scipy()
        n = As.shape[0]
        x, f = rng.standard_normal(n), rng.standard_normal(n)
        r = host(gb.level_apply(H, 0, l, 0, dev(x), dev(f)))
        assert rel_inf(r, f - As @ x) <= 1e-13, ("resid", l)
        y = host(gb.level_apply(H, 0, l, 1, dev(x), dev(f)))
        assert rel_inf(y, x + amg.smooth(lev, f - As @ x)) <= 1e-12, ("sweep", l)
    with pytest.raises(gb.GbsError):
        gb.level_apply(H, 0, len(Ho.levels), 0, dev(np.zeros(4)), dev(np.zeros(4)))


def test_schur_ilut_pressure_amg_matches_oracle():
    """ILUT relaxation in the pressure AMG on S_hat (relax_p = ILUT) as well
    as in the velocity AMG: the application (forward and transposed)
    matches the oracle's, and GMRES(30) converges."""
    s = si.make_system("c3", N=10)
    K = bsr.from_arrays(s.indptr, s.indices, s.data, 4)
    po = amg.AmgParams(coarse_enough=60, relax="ilut")
    pc = schur.build(K, 3, po, po)
    H = gb.build_hierarchy(s.indptr, s.indices, s.data, 4,
                           _params(s, coarse_enough=60, relax=gb.GBS_ILUT, relax_p=gb.GBS_ILUT))
    rng = np.random.default_rng(71)
    for tr in (False, True):
        r = rng.standard_normal(K.shape[0])
        z = host(gb.apply_precond(H, dev(r), transpose=tr))
        assert rel_inf(z, pc.apply(r, transpose=tr)) <= 1e-10, tr
    x, info = gb.solve(H, dev(s.b))
    assert info.converged and _true_rel(s, host(x)) <= 1e-8


def test_pipeline_wait_timeout_is_reported(monkeypatch):
    """The staged FP32 kernels (every level in slices, bulk copies on an
    mbarrier) with each pipeline wait bounded at 2^0 SM clocks: the first
    wait gives up before its copy lands, the warp records the timeout in
    the solve's scalar block after waiting (full bound) for every copy it
    has in flight, and the solve returns GBS_ERR_CUDA.  Nothing hangs and
    nothing faults; a fresh handle with the default bound then solves.
    A wait that finds its copy already landed succeeds whatever the bound,
    so L2 is flushed first: the first copies then come from DRAM and take
    far longer than the wait allows."""
    monkeypatch.setenv("GBS_LEVEL_FORMAT", "3")
    monkeypatch.setenv("GBS_SELL_DIRECT", "0")
    s = si.make_system("c2", N=10)
    H = gb.build_hierarchy(s.indptr, s.indices, s.data, 4,
                           _params(s, relax=gb.GBS_JACOBI, precision=gb.GBS_FP32, wait_log2=0))
    b = dev(s.b)
    flush = torch.zeros(32 << 20, dtype=torch.float64, device="cuda")   # 256 MB > L2
    flush += 1.0
    torch.cuda.synchronize()
    del flush
    with pytest.raises(gb.GbsError) as e:
        gb.solve(H, b)
    assert e.value.status == -2 and "timed out" in str(e.value)
    H2 = gb.build_hierarchy(s.indptr, s.indices, s.data, 4,
                            _params(s, relax=gb.GBS_JACOBI, precision=gb.GBS_FP32))
    x, info = gb.solve(H2, dev(s.b))
    assert info.converged and _true_rel(s, host(x)) <= 1e-8
