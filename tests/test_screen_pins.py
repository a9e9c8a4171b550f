"""Pins for the screened-precision reference (oracle/screen.py) against independent library casts."""
import numpy as np
import pytest
import torch

import oracle
import synth
from oracle import screen


def test_bf16_round_matches_torch_cast():
    rng = np.random.default_rng(0)
    x = np.concatenate([rng.standard_normal(20000).astype(np.float32) * 10,
                        np.float32([0.0, -0.0, 1.0, 1.00390625, 1.01171875, 3.0e-39, 65504.0])])
    ref = torch.from_numpy(x).to(torch.bfloat16).to(torch.float32).numpy()
    assert np.array_equal(screen.bf16_round(x), ref)


def test_e4m3_round_matches_torch_cast_in_range():
    rng = np.random.default_rng(1)
    y = np.concatenate([rng.uniform(-448, 448, 20000), rng.uniform(-0.02, 0.02, 5000),
                        [0.0, 448.0, -448.0, 2.0 ** -9, 2.0 ** -10, 3 * 2.0 ** -10, 2.0 ** -6,
                         1.0625, 1.1875, 240.0, 248.0, 432.0, 440.0]]).astype(np.float32)
    ref = torch.from_numpy(y).to(torch.float8_e4m3fn).to(torch.float64).numpy()
    np.testing.assert_array_equal(screen.e4m3_round(y), ref)


def test_e4m3_saturates():
    y = np.float32([449.0, 463.9, 464.0, 1e6, -500.0])
    np.testing.assert_array_equal(screen.e4m3_round(y), [448, 448, 448, 448, -448])


def test_fp8_quantize_row_scale():
    X = np.float32([[1.0, -2.0, 0.5], [0.0, 0.0, 0.0], [3.0, 3.0, -3.0]])
    scale, codes = screen.fp8_quantize(X)
    assert scale[1] == 1.0 and np.all(codes[1] == 0)
    assert scale[0] == np.float32(2.0) / np.float32(448.0)
    assert codes[0, 1] == -448.0 and codes[2, 2] == -448.0
    assert np.all(np.abs(codes) <= 448)


def test_screened_search_with_full_shortlist_is_exact_search():
    # R >= every candidate count: the exact rerank sees all candidates, so the result is the
    # plain float64 search whatever the screen's precision.
    X, Q = synth.mixture(2000, 24, 20, "B", seed=3)
    F = oracle.build_forest(X, 4, 30, seed=1)
    ids, d = oracle.search(F, X, Q, 5)
    for prec in ("bf16", "fp8"):
        si, sd, _ = screen.screened_search(F, X, Q, 5, 10_000, prec)
        assert np.array_equal(si, ids)
        np.testing.assert_allclose(sd, d, rtol=1e-12)
