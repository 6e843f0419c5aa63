"""Oracle pins: rounding to the mixed forms' storage formats (CPU only).

round_to() is checked against two library conversions it must equal --
numpy's FP64 -> float32 cast and torch's float32 -> bfloat16 cast (both
round to nearest, ties to even) -- and against hand-computed ties,
subnormals and the overflow bound.  cast_values() is checked to round
every stored value of a hierarchy and nothing else.
"""
import numpy as np
import pytest

import stokes_inputs as si
from oracle import amg, bsr, schur
from oracle.precision import round_to


def test_fp32_equals_numpy_cast_over_the_whole_range():
    rng = np.random.default_rng(0)
    v = rng.standard_normal(200000) * np.exp2(rng.uniform(-160, 125, 200000))
    np.testing.assert_array_equal(round_to(v, "fp32"), v.astype(np.float32).astype(np.float64))


def test_bf16_equals_torch_cast_of_float32_values():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(1)
    f = (rng.standard_normal(200000) * np.exp2(rng.integers(-140, 120, 200000))).astype(np.float32)
    ref = torch.from_numpy(f).to(torch.bfloat16).to(torch.float64).numpy()
    np.testing.assert_array_equal(round_to(f.astype(np.float64), "bf16"), ref)


def test_hand_computed_ties_and_subnormals():
    # bf16 keeps 7 mantissa bits: the spacing at 1 is 2^-7
    assert round_to(1 + 2.0 ** -8, "bf16") == 1.0                    # tie -> even (1.0)
    assert round_to(1 + 3 * 2.0 ** -8, "bf16") == 1 + 2.0 ** -6      # tie -> even (mantissa 2)
    assert round_to(1 + 2.0 ** -8 + 2.0 ** -30, "bf16") == 1 + 2.0 ** -7
    assert round_to(-(1 + 2.0 ** -8 + 2.0 ** -30), "bf16") == -(1 + 2.0 ** -7)
    # below 2^-126 the spacing stays 2^-133 (bf16) / 2^-149 (fp32)
    assert round_to(1.5 * 2.0 ** -133, "bf16") == 2.0 ** -132         # 1.5 ulp -> 2 ulp (even)
    assert round_to(2.0 ** -135, "bf16") == 0.0                       # a quarter ulp
    assert round_to(2.0 ** -149 * 0.5, "fp32") == 0.0                 # tie -> even (0)
    assert round_to(2.0 ** -149 * 0.75, "fp32") == 2.0 ** -149
    assert round_to(0.0, "bf16") == 0.0
    # fp32 at 1: spacing 2^-23
    assert round_to(1 + 2.0 ** -24, "fp32") == 1.0
    assert round_to(1 + 3 * 2.0 ** -24, "fp32") == 1 + 2.0 ** -22


def test_overflow_raises():
    with pytest.raises(ValueError):
        round_to(3.5e38, "fp32")
    with pytest.raises(ValueError):
        round_to(np.inf, "bf16")


def test_cast_values_rounds_every_stored_value():
    s = si.make_system("c2", N=6)
    K = bsr.from_arrays(s.indptr, s.indices, s.data, 4)
    H = amg.build_hierarchy(K, amg.AmgParams(relax="jacobi", coarse_enough=60))
    for fmt in ("fp32", "bf16"):
        Hc = amg.cast_values(H, fmt)
        assert Hc.nlevels == H.nlevels
        for a, b in zip(H.levels, Hc.levels):
            for X, Y in ((a.A, b.A), (a.P, b.P), (a.R, b.R)):
                assert np.array_equal(X.indptr, Y.indptr) and np.array_equal(X.indices, Y.indices)
                np.testing.assert_array_equal(Y.data, round_to(X.data, fmt))
            np.testing.assert_array_equal(b.M, round_to(a.M, fmt))
        np.testing.assert_array_equal(Hc.Ainv_coarse, round_to(H.Ainv_coarse, "fp32"))
        # the rounding is real: some value moved, none moved by more than half a spacing
        A0, A0c = H.levels[0].A.data, Hc.levels[0].A.data
        assert np.any(A0 != A0c)
        rel = np.abs(A0c - A0)[A0 != 0] / np.abs(A0[A0 != 0])
        assert rel.max() <= 2.0 ** -(24 if fmt == "fp32" else 8)


def test_schur_cast_values_rounds_couplings():
    s = si.make_system("c3", N=5)
    K = bsr.from_arrays(s.indptr, s.indices, s.data, 4)
    po = amg.AmgParams(coarse_enough=40)
    pc = schur.build(K, 3, po, po)
    pcc = schur.cast_values(pc, "bf16")
    np.testing.assert_array_equal(pcc.split.G.data, round_to(pc.split.G.data, "bf16"))
    np.testing.assert_array_equal(pcc.split.D.data, round_to(pc.split.D.data, "bf16"))
    np.testing.assert_array_equal(pcc.HA.levels[0].A.data,
                                  round_to(pc.HA.levels[0].A.data, "bf16"))
    np.testing.assert_array_equal(pcc.HS.levels[0].M, round_to(pc.HS.levels[0].M, "bf16"))
