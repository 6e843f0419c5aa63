"""Rounding to the storage formats of the mixed-precision forms (FP64 oracle).

TEST INFRASTRUCTURE ONLY (see the package docstring).

Section 4 of the paper keeps the outer Krylov iteration in double precision
and stores the nested preconditioner in single precision (Listing V4); the
BF16 form extends that to 16-bit storage.  The oracle does not emulate
reduced-precision arithmetic.  It models the one step of those forms that
has a plain definition: every stored value of the hierarchy (A_l, P_l, R_l,
M_l, the Schur couplings) and the vector entering the preconditioner are
rounded from FP64 to the storage format, round-to-nearest with ties to
even.  Applying the FP64 V-cycle to the rounded values then isolates the
only remaining difference from the GPU path: its FP32 accumulation.

Both formats share float32's exponent range (normal numbers down to
2^-126, subnormals below); they differ in the explicit mantissa bits:
23 for FP32, 7 for BF16.  A value is rounded once, straight from FP64.
"""
from __future__ import annotations

import numpy as np

MANTISSA_BITS = {"fp32": 23, "bf16": 7}
EMIN = -126                      # exponent of the smallest normal number
MAX_FINITE = {"fp32": (2.0 - 2.0 ** -23) * 2.0 ** 127,
              "bf16": (2.0 - 2.0 ** -7) * 2.0 ** 127}


def round_to(v, fmt: str) -> np.ndarray:
    """Round FP64 values to the nearest value of `fmt` ("fp32" or "bf16"),
    ties to even, returned as FP64.

    The representable numbers near |v| are the multiples of
    ulp = 2^(max(e, EMIN) - p), e the exponent of v's leading bit and p
    the mantissa bits (below 2^EMIN the spacing stays 2^(EMIN - p): the
    subnormals).  v / ulp is exact (a power-of-two scaling), so rounding
    it to an integer with ties to even and scaling back is the rounding
    itself.  Values beyond the format's largest finite number raise."""
    p = MANTISSA_BITS[fmt]
    v = np.asarray(v, dtype=np.float64)
    if np.any(~np.isfinite(v)):
        raise ValueError("round_to: non-finite input")
    a = np.abs(v)
    _, e2 = np.frexp(np.where(a > 0, a, 1.0))   # a = m 2^e2, m in [0.5, 1)
    lead = np.maximum(e2 - 1, EMIN)
    ulp = np.ldexp(1.0, lead - p)
    out = np.round(v / ulp) * ulp                # np.round: ties to even
    if np.any(np.abs(out) > MAX_FINITE[fmt]):
        raise ValueError("round_to: value beyond the largest finite %s" % fmt)
    return np.where(a > 0, out, v)
