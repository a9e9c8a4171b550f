"""Reference for the screened precisions -- TEST INFRASTRUCTURE (see oracle/__init__.py).

Sec. 3 ("Distance computation") makes the distance evaluation the cost of a search; the screened
precisions rank the candidates with a low-precision copy of the points and rescore a shortlist
exactly.  This module restates, in float64 numpy, what that computes:

* bfloat16: round-to-nearest-even of the float32 value to 8 significant bits (IEEE rounding of
  the upper 16 bits of the float32 pattern).
* FP8-E4M3 (OCP 8-bit floating point, E4M3: bias 7, 3 mantissa bits, largest finite 448, no
  infinities): per row a = max_j |x_j|, inv = float32(448 / a), scale = float32(a / 448); each
  value y = float32(x_j * inv) is rounded to nearest-even on the E4M3 grid and saturated to +-448.
  A zero row keeps codes 0 and scale 1.
* screened distance: sum_j (q_j - deq_j)^2 in float64 with deq = bf16 value or scale * e4m3 value;
  the R smallest by (screened distance, id) are rescored with the exact float64 distance and the k
  smallest by (distance, id) returned.
"""
from __future__ import annotations

import numpy as np

import oracle


def bf16_round(x: np.ndarray) -> np.ndarray:
    """float32 -> nearest bfloat16 (ties to even), returned as float32 values."""
    u = np.ascontiguousarray(x, dtype=np.float32).view(np.uint32).astype(np.uint64)
    lsb = (u >> 16) & 1
    u = (u + 0x7FFF + lsb) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32)


def e4m3_round(y: np.ndarray) -> np.ndarray:
    """float32 values -> nearest E4M3 value (ties to even, saturating at +-448), as float64."""
    y = np.asarray(y, dtype=np.float64)
    a = np.abs(y)
    e = np.floor(np.log2(np.where(a > 0, a, 1.0)))
    e = np.where(np.exp2(e) > a, e - 1, e)        # guard log2 rounding at powers of two
    e = np.where(np.exp2(e + 1) <= a, e + 1, e)
    e = np.maximum(e, -6.0)                       # below 2^-6 the grid is the subnormal step 2^-9
    step = np.exp2(e - 3.0)
    r = np.round(a / step) * step                 # numpy rounds halves to even
    r = np.minimum(r, 448.0)
    return np.sign(y) * r


def fp8_quantize(X: np.ndarray):
    """Per-row scales and dequantized E4M3 codes (as float64 code values, before the scale)."""
    X = np.ascontiguousarray(X, dtype=np.float32)
    a = np.abs(X).max(axis=1)
    pos = a > 0
    inv = np.zeros_like(a)
    inv[pos] = np.float32(448.0) / a[pos]
    scale = np.ones_like(a)
    scale[pos] = a[pos] / np.float32(448.0)
    Y = (X * inv[:, None]).astype(np.float32)
    return scale.astype(np.float32), e4m3_round(Y)


def dequantized_rows(X: np.ndarray, rows: np.ndarray, precision: str) -> np.ndarray:
    """float64 values the screen of `precision` sees for the given rows of X."""
    Xr = np.ascontiguousarray(X[rows], dtype=np.float32)
    if precision == "bf16":
        return bf16_round(Xr).astype(np.float64)
    if precision == "fp8":
        scale, codes = fp8_quantize(Xr)
        return codes * scale.astype(np.float64)[:, None]
    if precision == "fp32":
        return Xr.astype(np.float64)
    raise ValueError(precision)


def screened_search(F, X, Q, k, R, precision: str, offs=None, cand=None):
    """Candidates of the forest, screened ranking, shortlist of R, exact rerank, top-k."""
    X = np.asarray(X)
    Q = np.ascontiguousarray(Q, dtype=np.float32)
    if offs is None:
        offs, cand = oracle.candidates(F, oracle.descend(F, Q))
    m = Q.shape[0]
    ids = np.full((m, k), -1, dtype=np.int64)
    dd = np.full((m, k), np.inf)
    shortlist = []
    for i in range(m):
        c = cand[offs[i]:offs[i + 1]].astype(np.int64)
        q = Q[i].astype(np.float64)
        sd = ((dequantized_rows(X, c, precision) - q) ** 2).sum(axis=1)
        order = np.lexsort((c, sd))[:R]
        sl = c[order]
        shortlist.append((sl, sd[order]))
        ed = ((X[sl].astype(np.float64) - q) ** 2).sum(axis=1)
        o2 = np.lexsort((sl, ed))[:k]
        ids[i, :len(o2)] = sl[o2]
        dd[i, :len(o2)] = ed[o2]
    return ids, dd, shortlist
