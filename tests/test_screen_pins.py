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


# Two points where the screen's rounding reverses the exact order (query at the origin), worked by
# hand.  bf16 (8 significant bits): x1 = (1.0045, 0) rounds to (1.0078125, 0), screened 1.015686
# against exact 1.009020; x2 = (1, 0.1) rounds to (1, 0.10009766), screened 1.010020 against exact
# 1.01.  So the exact nearest is x1 but the screen ranks x2 first.  fp8 (row scale a / 448, codes
# e4m3(x 448 / a)): x1 = (1, 0.06) has codes (448, 26) since 26.88 rounds to 26 (e4m3 steps of 2
# in [16, 32)), dequantized (1, 0.0580357), screened 1.003368 against exact 1.0036; x2 =
# (1.0017, 0) has codes (448, 0), screened and exact 1.003403.  So the exact nearest is x2 but the
# screen ranks x1 first.  With a shortlist of one the screened search must return the point the
# screen ranks first, reported with its exact distance; with a shortlist of two, the exact nearest.
SCREEN_FLIPS = {
    "bf16": (np.float32([[1.0045, 0.0], [1.0, 0.1]]), 1, 0),
    "fp8": (np.float32([[1.0, 0.06], [1.0017, 0.0]]), 0, 1),
}


@pytest.mark.parametrize("prec", ["bf16", "fp8"])
def test_screen_rounding_reorders_a_hand_worked_pair(prec):
    X, screen_first, exact_first = SCREEN_FLIPS[prec]
    Q = np.zeros((1, 2), np.float32)
    F = oracle.build_forest(X, 1, 2, t=2, seed=0)  # one leaf: both points are candidates
    exact = (X.astype(np.float64) ** 2).sum(axis=1)
    ids, d, shortlist = screen.screened_search(F, X, Q, 1, 1, prec)
    assert ids[0, 0] == screen_first and d[0, 0] == exact[screen_first]
    assert shortlist[0][0].tolist() == [screen_first]
    ids2, d2, _ = screen.screened_search(F, X, Q, 1, 2, prec)
    assert ids2[0, 0] == exact_first and d2[0, 0] == exact[exact_first]
    screened = (screen.dequantized_rows(X, np.arange(2), prec) ** 2).sum(axis=1)
    expect = {"bf16": [1.0156860351, 1.0100195408], "fp8": [1.0033682, 1.0034030]}[prec]
    np.testing.assert_allclose(screened, expect, rtol=2e-7)
