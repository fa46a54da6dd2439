"""Pins of the oracle's FP64 -> FP8-e4m3 / BF16 / FP16 / FP32 rounding.

The method computes the sketch "in precision u_p" (Alg. 1); the oracle
emulates u_p by one RNE rounding from FP64.  Pinned against the format
definitions (exhaustive decode of every bit pattern, written here from the
OCP FP8 and IEEE 754 layouts), and against numpy / torch casts as
independent library references.
"""
import numpy as np
import pytest
import torch

import oracle as O


def decode(bits, ebits, mbits, bias, fn_nan_only_allones=False):
    """Value of a sign/exponent/mantissa bit pattern (IEEE-style layout)."""
    s = -1.0 if (bits >> (ebits + mbits)) & 1 else 1.0
    e = (bits >> mbits) & ((1 << ebits) - 1)
    f = bits & ((1 << mbits) - 1)
    if fn_nan_only_allones:
        if e == (1 << ebits) - 1 and f == (1 << mbits) - 1:
            return np.nan
    elif e == (1 << ebits) - 1:
        return s * np.inf if f == 0 else np.nan
    if e == 0:
        return s * f * 2.0 ** (1 - bias - mbits)
    return s * (1.0 + f / 2.0 ** mbits) * 2.0 ** (e - bias)


FORMATS = {
    O.FP8_E4M3: dict(ebits=4, mbits=3, bias=7, fn_nan_only_allones=True),
    O.BF16: dict(ebits=8, mbits=7, bias=127),
    O.FP16: dict(ebits=5, mbits=10, bias=15),
}


def finite_values(prec):
    fmt = FORMATS[prec]
    nb = 1 + fmt["ebits"] + fmt["mbits"]
    vals = np.array([decode(b, **fmt) for b in range(1 << nb)])
    vals = vals[np.isfinite(vals)]
    return np.unique(vals)


@pytest.mark.parametrize("prec", [O.FP8_E4M3, O.BF16, O.FP16])
def test_every_finite_value_is_fixed_point(prec):
    v = finite_values(prec)
    np.testing.assert_array_equal(O.round_to(v, prec), v)


@pytest.mark.parametrize("prec", [O.FP8_E4M3, O.BF16, O.FP16])
def test_midpoints_round_to_even_and_neighbours_to_nearest(prec):
    v = finite_values(prec)
    pos = v[v >= 0]
    lo, hi = pos[:-1], pos[1:]
    mid = (lo + hi) / 2  # exact in FP64 for these short formats
    fmt = FORMATS[prec]
    nb = 1 + fmt["ebits"] + fmt["mbits"]
    # "even" = the neighbour whose last mantissa bit is 0
    enc = {}
    for b in range(1 << (nb - 1)):
        d = decode(b, **fmt)
        if np.isfinite(d):
            enc.setdefault(d, b)
    even = np.array([lo_ if (enc[lo_] & 1) == 0 else hi_ for lo_, hi_ in zip(lo, hi)])
    np.testing.assert_array_equal(O.round_to(mid, prec), even)
    eps = (hi - lo) * 1e-6
    np.testing.assert_array_equal(O.round_to(mid - eps, prec), lo)
    np.testing.assert_array_equal(O.round_to(mid + eps, prec), hi)
    np.testing.assert_array_equal(O.round_to(-(mid + eps), prec), -hi)


def test_fp8_saturates_and_bf16_fp16_overflow():
    assert O.round_to([1e6], O.FP8_E4M3)[0] == 448.0
    assert O.round_to([-500.0], O.FP8_E4M3)[0] == -448.0
    assert O.round_to([464.0], O.FP8_E4M3)[0] == 448.0
    assert O.round_to([2.0 ** -10], O.FP8_E4M3)[0] == 0.0  # half the smallest subnormal ties to 0
    assert O.round_to([1.5 * 2.0 ** -10], O.FP8_E4M3)[0] == 2.0 ** -9
    assert np.isinf(O.round_to([65520.0], O.FP16)[0])
    assert O.round_to([65519.0], O.FP16)[0] == 65504.0
    assert np.isinf(O.round_to([3.5e38], O.BF16)[0])


def test_no_double_rounding_through_fp32():
    # 1 + 2^-8 + 2^-30 lies just above the BF16 midpoint between 1 and 1 + 2^-7.
    # Rounded directly it goes up; through FP32 the 2^-30 is lost and the tie goes to even (1.0).
    x = 1.0 + 2.0 ** -8 + 2.0 ** -30
    assert O.round_to([x], O.BF16)[0] == 1.0 + 2.0 ** -7
    via32 = float(torch.tensor(float(np.float32(x))).to(torch.bfloat16).float())
    assert via32 == 1.0


def test_fp32_and_fp16_match_numpy_casts():
    rng = np.random.default_rng(1)
    x = rng.standard_normal(20000) * np.exp2(rng.integers(-160, 140, 20000))
    np.testing.assert_array_equal(O.round_to(x, O.FP32), x.astype(np.float32).astype(np.float64))
    y = rng.standard_normal(20000) * np.exp2(rng.integers(-28, 18, 20000))
    np.testing.assert_array_equal(O.round_to(y, O.FP16), y.astype(np.float16).astype(np.float64))


def test_bf16_fp8_match_torch_from_fp32():
    rng = np.random.default_rng(2)
    x = (rng.standard_normal(20000) * np.exp2(rng.integers(-130, 120, 20000))).astype(np.float32)
    ref = torch.from_numpy(x).to(torch.bfloat16).to(torch.float64).numpy()
    np.testing.assert_array_equal(O.round_to(x.astype(np.float64), O.BF16), ref)
    y = (rng.standard_normal(20000) * np.exp2(rng.integers(-12, 8, 20000))).astype(np.float32)
    y = np.clip(y, -448, 448)
    ref8 = torch.from_numpy(y).to(torch.float8_e4m3fn).to(torch.float64).numpy()
    np.testing.assert_array_equal(O.round_to(y.astype(np.float64), O.FP8_E4M3), ref8)
