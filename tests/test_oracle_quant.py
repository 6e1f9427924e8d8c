"""Pins of the oracle's own BF16 / FP8-E4M3 encoders against PyTorch's casts
(library routines, round-to-nearest-even) and of the power-of-two scale."""
import numpy as np
import pytest
import torch

import oracle


def edge_values():
    rng = np.random.default_rng(0)
    v = np.concatenate([
        rng.uniform(0, 1, 20000), rng.uniform(0, 448, 20000), 10.0 ** rng.uniform(-12, 2, 20000),
        [0.0, 1.0, 448.0, 2.0 ** -9, 2.0 ** -6, 240.0, 1.0 + 2 ** -8, 1.0 + 3 * 2 ** -8],
    ]).astype(np.float32)
    # exact midpoints between neighbouring E4M3 codes and between neighbouring
    # bfloat16 values near 1: round-half-to-even decides these
    e4 = torch.arange(0, 127, dtype=torch.uint8).view(torch.float8_e4m3fn).float().numpy().astype(np.float64)
    mids = ((e4[1:] + e4[:-1]) / 2).astype(np.float32)
    bmid = (1.0 + (np.arange(64) + 0.5) * 2.0 ** -7).astype(np.float32)
    v = np.concatenate([v, mids, bmid])
    return np.concatenate([v, -v[:1000], -mids])


def test_bf16_matches_torch():
    v = edge_values()
    mine = oracle.bf16_codes(v)
    ref = torch.from_numpy(v).to(torch.bfloat16).view(torch.int16).numpy().view(np.uint16)
    np.testing.assert_array_equal(mine, ref)


def test_e4m3_matches_torch():
    v = edge_values()
    v = v[np.abs(v) <= 448]
    mine = oracle.e4m3_codes(v.astype(np.float64))
    ref = torch.from_numpy(v).to(torch.float8_e4m3fn).view(torch.uint8).numpy()
    np.testing.assert_array_equal(mine, ref)
    np.testing.assert_array_equal(oracle.e4m3_values(mine), torch.from_numpy(ref).view(torch.float8_e4m3fn).float().numpy())


@pytest.mark.parametrize("m", [1e-9, 0.3, 1.0, 448.0, 449.0, 896.0, 1e6])
def test_pow2_scale(m):
    s = float(oracle.e4m3_scale(np.array([m]))[0])
    assert 448.0 * s >= m > 224.0 * s
    assert np.log2(s) == np.round(np.log2(s))


def test_quantized_fp8_relative_error():
    rng = np.random.default_rng(1)
    blt = rng.integers(0, 50, 5000).astype(np.int32)
    val = rng.uniform(0.01, 1, 5000).astype(np.float32)
    dq, s = oracle.quantize_ddc(50, blt, val, "fp8")
    # E4M3 keeps 3 mantissa bits: relative error <= 2^-4 for normal codes
    assert np.all(np.abs(dq - val) <= 2.0 ** -4 * np.abs(val) + 2.0 ** -9 * s[blt])
    dq, _ = oracle.quantize_ddc(50, blt, val, "bf16")
    # bfloat16 keeps 8 significant bits: relative error <= 2^-8
    assert np.all(np.abs(dq - val) <= 2.0 ** -8 * np.abs(val))
