"""The screened comparison rule (parity.assert_screened_close) on the CPU: it must accept every answer
a screen within its rounding bound can give, and reject answers no such screen gives.  The GPU is
replaced by rows made from the oracle's own float64 screen (Sec. 3 "Distance computation"):
  - scores moved anywhere inside the bound, their shortlist and exact top-k: accepted;
  - the k worst candidates of the query, at their exact distances and in order: rejected;
  - the nearest candidate dropped when the shortlist must hold it: rejected;
  - with the GPU's own scores given, a row that is not the top-k of the shortlist they make: rejected.
"""
import numpy as np
import pytest

import oracle
import synth
from oracle import screen
from parity import assert_screened_close, screen_bounds, screened_sets


@pytest.fixture(scope="module")
def setup():
    X, Q = synth.mixture(3000, 24, 40, "B", seed=3, qseed=4)
    F = oracle.build_forest(X, 6, 40, seed=5)
    offs, ids = oracle.candidates(F, oracle.descend(F, Q))
    return X, Q, F, offs, ids


def perturbed_answer(X, Q, offs, ids, k, R, precision, form, rng, bounds=screen_bounds):
    """What a screen whose scores lie within the bound of screen_bounds may return."""
    m = len(offs) - 1
    gi = np.full((m, k), -1, dtype=np.int64)
    gd = np.full((m, k), np.inf, dtype=np.float32)
    for i in range(m):
        c = ids[offs[i]:offs[i + 1]].astype(np.int64)
        sd, eps = bounds(X, Q[i], c, precision, form)
        g = sd + eps * rng.uniform(-1, 1, size=len(c))
        sl = np.lexsort((c, g))[:R]
        ed = ((X[c[sl]].astype(np.float64) - Q[i].astype(np.float64)) ** 2).sum(axis=1)
        top = np.lexsort((c[sl], ed))[:k]
        gi[i, :len(top)] = c[sl][top]
        gd[i, :len(top)] = ed[top]
    return gi, gd


@pytest.mark.parametrize("precision,form", [("bf16", "norm"), ("fp8", "norm"), ("bf16", "direct"), ("fp8", "direct")])
def test_accepts_any_screen_within_the_bound(setup, precision, form, monkeypatch):
    """Scores anywhere within the bound give answers the rule accepts.  At the true bound this data
    has no score close enough to the shortlist boundary to change a row, so the bound is also
    widened (in the rule and in the scores alike) until a good share of the rows differ from the
    oracle's, which exercises the rule's checks of differing rows."""
    import parity
    X, Q, F, offs, ids = setup
    k, R = 4, 8
    oi, od, _ = screen.screened_search(F, X, Q, k, R, precision, offs, ids)
    true_bounds = parity.screen_bounds
    for widen in [1.0] + [10.0 ** j for j in range(1, 8)]:
        monkeypatch.setattr(parity, "screen_bounds",
                            lambda *a, w=widen: (true_bounds(*a)[0], w * true_bounds(*a)[1]))
        rng = np.random.default_rng(0)
        differ = 0
        for trial in range(3):
            gi, gd = perturbed_answer(X, Q, offs, ids, k, R, precision, form, rng, bounds=parity.screen_bounds)
            differ = max(differ, int((gi != oi).any(axis=1).sum()))
            parity.assert_screened_close(X, Q, gi, gd, oi, od, offs, ids, precision, R, form, max_frac=1.0)
        if differ >= len(oi) // 10:
            return
    pytest.fail("no widening of the bound changed a tenth of the rows")


def test_rejects_the_k_worst_candidates(setup):
    X, Q, F, offs, ids = setup
    k, R = 4, 8
    oi, od, _ = screen.screened_search(F, X, Q, k, R, "bf16", offs, ids)
    gi, gd = oi.copy(), od.astype(np.float32).copy()
    c = ids[offs[0]:offs[1]].astype(np.int64)
    ed = ((X[c].astype(np.float64) - Q[0].astype(np.float64)) ** 2).sum(axis=1)
    worst = np.lexsort((c, ed))[-k:]
    gi[0], gd[0] = c[worst], ed[worst]
    with pytest.raises(AssertionError, match="cannot be on a shortlist"):
        assert_screened_close(X, Q, gi, gd, oi, od, offs, ids, "bf16", R, "norm")


def test_rejects_a_missing_required_candidate(setup):
    X, Q, F, offs, ids = setup
    k, R = 4, 8
    oi, od, shortlists = screen.screened_search(F, X, Q, k, R, "bf16", offs, ids)
    for i in range(len(offs) - 1):
        c = ids[offs[i]:offs[i + 1]].astype(np.int64)
        if len(c) <= R + k:
            continue
        sd, eps = screen_bounds(X, Q[i], c, "bf16", "norm")
        may, must = screened_sets(sd, eps, R)
        p0 = np.searchsorted(c, oi[i, 0])
        if not must[p0]:
            continue
        # the nearest dropped, the next shortlisted point (by exact distance) appended
        sl = shortlists[i][0]
        ed = ((X[sl].astype(np.float64) - Q[i].astype(np.float64)) ** 2).sum(axis=1)
        order = np.lexsort((sl, ed))
        gi, gd = oi.copy(), od.astype(np.float32).copy()
        gi[i], gd[i] = sl[order[1:k + 1]], ed[order[1:k + 1]]
        with pytest.raises(AssertionError, match="left out"):
            assert_screened_close(X, Q, gi, gd, oi, od, offs, ids, "bf16", R, "norm")
        return
    pytest.fail("no query whose nearest candidate the shortlist must hold")


def test_rejects_a_row_that_is_not_the_top_k_of_the_gpu_shortlist(setup):
    X, Q, F, offs, ids = setup
    k, R = 4, 8
    oi, od, _ = screen.screened_search(F, X, Q, k, R, "bf16", offs, ids)
    m = len(offs) - 1
    width = int(np.diff(offs).max())
    gs = np.full((m, width), np.nan, dtype=np.float32)
    ge = np.full((m, width), np.nan, dtype=np.float32)
    for i in range(m):
        c = ids[offs[i]:offs[i + 1]]
        gs[i, :len(c)] = ((screen.dequantized_rows(X, c, "bf16") - Q[i].astype(np.float64)) ** 2).sum(axis=1)
        ge[i, :len(c)] = ((X[c].astype(np.float64) - Q[i].astype(np.float64)) ** 2).sum(axis=1)
    # the oracle's own answer, with float32 distances, is the top-k of these scores' shortlist
    gi = oi.copy()
    gd = np.where(oi >= 0, od, np.inf).astype(np.float32)
    for i in range(m):
        c = ids[offs[i]:offs[i + 1]]
        gd[i, :len(c[:k])] = ge[i, np.searchsorted(c, oi[i, :min(k, len(c))])]
    assert_screened_close(X, Q, gi, gd, oi, od, offs, ids, "bf16", R, "direct", gpu_scores=(gs, ge))
    # swap in a candidate from outside the shortlist at its exact distance: the exact check fails
    c = ids[offs[0]:offs[1]]
    sl = np.lexsort((c, gs[0, :len(c)]))[:R]
    outside = np.setdiff1d(np.arange(len(c)), sl)
    j = outside[np.argmin(ge[0, outside])]
    gi[0, -1], gd[0, -1] = c[j], max(ge[0, j], gd[0, -2])
    with pytest.raises(AssertionError):
        assert_screened_close(X, Q, gi, gd, oi, od, offs, ids, "bf16", R, "direct", gpu_scores=(gs, ge))
