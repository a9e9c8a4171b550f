"""Seeded synthetic inputs shaped like the paper's workloads.

The paper evaluates on GIST (10^6 x 960, and its 10^5 subset), SIFT, MNIST and on synthetic
manifolds (Sec. 4 "Datasets"). None of those files exist here, so Gaussian mixtures of the same
shapes stand in for them.  This module only draws numbers: it contains none of the search
method's arithmetic, and both the CUDA path's tests and the CPU oracle's tests take their inputs
from it.

Laws (every one float32, row-major):

* ``"A"``  K=20 centers c_k ~ N(0, 4 I_d); component uniform; x = c_k + N(0, I_d).
* ``"B"``  K=100 centers c_k ~ N(0, 4 I_d); x = c_k + sigma * z with sigma_j = 1/sqrt(1 + j/32)
           (GIST-like anisotropy); then every dimension is shifted by minus its minimum over the
           dataset so that the data are non-negative.  Queries get the same shift.
* ``"C"``  as B with K=50 and sigma_j = 1/sqrt(1 + j/256) (the d = 10,000 law).

Queries are independent draws from the same mixture (same centers).  Generation is split into
fixed blocks of rows, each with its own seeded ``numpy.random.Generator``; blocks run on a thread
pool, so the output does not depend on the number of threads.
"""
from __future__ import annotations

import os
from concurrent.futures import ThreadPoolExecutor
from dataclasses import dataclass

import numpy as np

__all__ = ["Law", "LAWS", "mixture", "manifold", "quantize_u8", "BLOCK_ROWS"]

BLOCK_ROWS = 16384


@dataclass(frozen=True)
class Law:
    name: str
    K: int             # number of mixture components
    center_std: float  # centers ~ N(0, center_std^2 I)
    decay: float       # sigma_j = 1/sqrt(1 + j/decay); 0 means sigma_j = 1
    shift: bool        # shift every dimension to a minimum of zero

    def sigma(self, d: int) -> np.ndarray:
        j = np.arange(d, dtype=np.float64)
        if self.decay == 0:
            return np.ones(d, dtype=np.float32)
        return (1.0 / np.sqrt(1.0 + j / self.decay)).astype(np.float32)


LAWS = {
    "A": Law("A", K=20, center_std=2.0, decay=0.0, shift=False),
    "B": Law("B", K=100, center_std=2.0, decay=32.0, shift=True),
    "C": Law("C", K=50, center_std=2.0, decay=256.0, shift=True),
}


def _centers(law: Law, d: int, seed: int) -> np.ndarray:
    rng = np.random.default_rng([seed, 0xC0])
    return (rng.standard_normal((law.K, d)) * law.center_std).astype(np.float32)


def _fill(out: np.ndarray, centers: np.ndarray, sigma: np.ndarray, seed: int, stream: int,
          threads: int) -> None:
    rows = out.shape[0]
    nblk = (rows + BLOCK_ROWS - 1) // BLOCK_ROWS

    def work(b: int) -> None:
        lo, hi = b * BLOCK_ROWS, min(rows, (b + 1) * BLOCK_ROWS)
        rng = np.random.default_rng([seed, stream, b])
        lab = rng.integers(0, centers.shape[0], size=hi - lo)
        z = rng.standard_normal((hi - lo, out.shape[1]), dtype=np.float32)
        z *= sigma
        z += centers[lab]
        out[lo:hi] = z

    if nblk <= 1 or threads <= 1:
        for b in range(nblk):
            work(b)
    else:
        with ThreadPoolExecutor(max_workers=threads) as ex:
            list(ex.map(work, range(nblk)))


def mixture(n: int, d: int, m: int, law: str = "A", seed: int = 0, qseed: int = 1,
            threads: int | None = None) -> tuple[np.ndarray, np.ndarray]:
    """Return (X [n, d], Q [m, d]) float32 drawn from mixture ``law``.

    ``seed`` fixes the centers and the data points, ``qseed`` the queries.
    """
    L = LAWS[law]
    if threads is None:
        threads = min(32, os.cpu_count() or 1)
    C = _centers(L, d, seed)
    sig = L.sigma(d)
    X = np.empty((n, d), dtype=np.float32)
    Q = np.empty((m, d), dtype=np.float32)
    _fill(X, C, sig, seed, 1, threads)
    _fill(Q, C, sig, qseed, 2, threads)
    if L.shift and n > 0:
        mn = X.min(axis=0)
        X -= mn
        Q -= mn
    return X, Q


def _frame(k: int, d: int, seed: int) -> np.ndarray:
    """A seeded random orthonormal k x d frame (rows orthonormal), k <= d."""
    rng = np.random.default_rng([seed, 0xF0])
    G = rng.standard_normal((d, k))
    Qm, R = np.linalg.qr(G)
    return (Qm * np.sign(np.diag(R))).T  # k x d


def _manifold_points(kind: str, count: int, rng) -> np.ndarray:
    if kind == "klein":
        # the Klein bottle's embedding in R^4 with radii 2 and 1:
        # ((2 + cos v) cos u, (2 + cos v) sin u, sin v cos(u/2), sin v sin(u/2)), u, v uniform
        u = rng.uniform(0, 2 * np.pi, count)
        v = rng.uniform(0, 2 * np.pi, count)
        return np.stack([(2 + np.cos(v)) * np.cos(u), (2 + np.cos(v)) * np.sin(u),
                         np.sin(v) * np.cos(u / 2), np.sin(v) * np.sin(u / 2)], axis=1)
    if kind == "sphere":
        # uniform on the unit 2-sphere
        g = rng.standard_normal((count, 3))
        return g / np.linalg.norm(g, axis=1, keepdims=True)
    raise ValueError(kind)


def manifold(n: int, d: int, m: int, kind: str = "klein", noise: float | None = None, seed: int = 0,
             qseed: int = 1) -> tuple[np.ndarray, np.ndarray]:
    """Noisy low-dimensional manifold in R^d (the paper's Klein-bottle and sphere sets, Sec. 4).

    Points are drawn uniformly in the manifold's parameters, mapped into R^d by a seeded random
    orthonormal frame, and every coordinate gets N(0, noise^2) (0.05 for the Klein bottle, 0.1 for
    the sphere, as in the paper).  Queries are independent draws from the same law.
    """
    if noise is None:
        noise = 0.05 if kind == "klein" else 0.1
    dim = 4 if kind == "klein" else 3
    Fr = _frame(dim, d, seed)
    out = []
    for cnt, sd in ((n, [seed, 11]), (m, [qseed, 12])):
        rng = np.random.default_rng(sd)
        P = _manifold_points(kind, cnt, rng) @ Fr
        P += rng.standard_normal(P.shape) * noise
        out.append(P.astype(np.float32))
    return out[0], out[1]


def quantize_u8(A: np.ndarray, scale: float = 8.0) -> np.ndarray:
    """Round to integer-valued floats in [0, 255] (SIFT-like byte data: many exact ties)."""
    return np.clip(np.rint(A * scale), 0, 255).astype(np.float32)
