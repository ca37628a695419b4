"""Pins of the CPU model of the 16-bit matrix copies (tests/_round16.py) against
library conversions: numpy's binary16 cast and torch's float32 -> bfloat16 cast,
both round to nearest with ties to even."""
import numpy as np
import pytest

from _round16 import round_sig, pow2_row_scale, stored_rows, _col_round


def _values(rng, n):
    mag = 10.0 ** rng.uniform(-9, -0.01, n)
    return mag * rng.choice([-1.0, 1.0], n)


def test_fp16_matches_numpy_cast():
    rng = np.random.default_rng(0)
    x = _values(rng, 20000)
    # exact ties between neighbouring binary16 values, normal and subnormal
    h = np.float16(rng.uniform(-0.9, 0.9, 2000)).astype(np.float64)
    ulp = np.spacing(np.abs(np.float16(h))).astype(np.float64)
    ties = h + 0.5 * ulp * np.sign(h)
    sub = (rng.integers(1, 1000, 500) + 0.5) * 2.0 ** -24
    for v in (x, ties, sub, -sub):
        assert np.array_equal(round_sig(v, "fp16"), v.astype(np.float16).astype(np.float64))


def test_bf16_matches_torch_cast():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(1)
    x = _values(rng, 20000).astype(np.float32)
    # float32 values halfway between two bfloat16 values
    b = torch.tensor(rng.uniform(-0.9, 0.9, 2000), dtype=torch.float32).to(torch.bfloat16)
    bits = b.view(torch.int16).to(torch.int32) << 16
    ties = (bits | 0x8000).to(torch.int32).view(torch.float32).numpy()
    for v in (x, ties):
        ref = torch.tensor(v).to(torch.bfloat16).to(torch.float64).numpy()
        assert np.array_equal(round_sig(v.astype(np.float64), "bf16"), ref)


def test_row_scales_are_powers_of_two():
    rng = np.random.default_rng(2)
    M = rng.standard_normal((40, 24)) * 10.0 ** rng.uniform(-8, 8, (40, 1))
    M[3] = 0.0
    s = pow2_row_scale(M)
    m, e = np.frexp(s)
    assert np.all(m == 0.5)
    r = np.abs(M).max(axis=1) / s
    assert np.all((r[np.arange(40) != 3] >= 0.5) & (r[np.arange(40) != 3] < 1.0)) and s[3] == 1.0
    for fmt, bits in (("fp16", 11), ("bf16", 8)):
        Ms = stored_rows(M, fmt)
        # error at most half a unit of the row's leading binade (normal range of the scaled rows)
        assert np.all(np.abs(Ms - M) <= 0.5 * 2.0 ** -bits * s[:, None] * (1 + 1e-12))


def test_column_rounding():
    rng = np.random.default_rng(3)
    v = rng.standard_normal(50) * 1e5
    for fmt, bits in (("fp16", 11), ("bf16", 8)):
        q = _col_round(v, fmt)
        s = pow2_row_scale(v[None, :])[0]
        assert np.all(np.abs(q - v) <= 0.5 * 2.0 ** -bits * s * (1 + 1e-12))
        assert np.array_equal(_col_round(q, fmt), q)     # idempotent
    assert np.array_equal(_col_round(np.zeros(4), "fp16"), np.zeros(4))
