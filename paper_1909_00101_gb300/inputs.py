"""Seeded synthetic GSVD input pairs (F, G) with known generalized singular values.

This module holds none of the Hari-Zimmermann method's arithmetic: it only
builds test and benchmark inputs.  Both the oracle-side tests and the CUDA
library's tests and benchmark draw their inputs from here.

Construction (the paper's datasets are not available; these stand in for
them with the shapes of the benchmark configurations):

1. sigma_i log-spaced in [lo, hi], then a seeded permutation so that the
   input is not presorted;
2. Sigma_F = sigma / sqrt(1 + sigma^2), Sigma_G = 1 / sqrt(1 + sigma^2), so
   Sigma_F^2 + Sigma_G^2 = I and Sigma_G^{-1} Sigma_F = sigma;
3. U0 (mF x n) and V0 (mG x n) with orthonormal (unitary) columns, Haar
   distributed: QR of a Gaussian matrix with the sign/phase of R's diagonal
   moved into Q (Mezzadri 2007);
4. X = Q1 diag(d) Q2 with Q1, Q2 Haar and d log-spaced in [1, cond];
5. F = U0 Sigma_F X, G = V0 Sigma_G X, so that F X^{-1} = U0 Sigma_F and
   G X^{-1} = V0 Sigma_G: the exact GSVD of (F, G) has Z = X^{-1} up to
   column order and unit scalars.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np


def _haar(rng: np.random.Generator, m: int, n: int, cplx: bool) -> np.ndarray:
    a = rng.standard_normal((m, n))
    if cplx:
        a = (a + 1j * rng.standard_normal((m, n))) / np.sqrt(2.0)
    q, r = np.linalg.qr(a)
    d = np.diagonal(r)
    ph = d / np.abs(d)
    return q * ph[None, :]


@dataclass
class Pair:
    F: np.ndarray          # mF x n, Fortran order
    G: np.ndarray          # mG x n, Fortran order
    sigma: np.ndarray      # generated generalized singular values, sorted descending
    cond_x: float
    seed: int


def make_pair(mf: int, mg: int, n: int, *, lo: float = 1e-2, hi: float = 1e2,
              cond: float = 1e2, cplx: bool = False, seed: int = 0) -> Pair:
    """One seeded pair; real float64 or complex128, column-major."""
    if n < 1 or mf < n or mg < n:
        raise ValueError("need mF, mG >= n >= 1")
    rng = np.random.default_rng(seed)
    sig = np.logspace(np.log10(lo), np.log10(hi), n) if n > 1 else np.array([np.sqrt(lo * hi)])
    sig = sig[rng.permutation(n)]
    sf = sig / np.sqrt(1.0 + sig * sig)
    sg = 1.0 / np.sqrt(1.0 + sig * sig)
    u0 = _haar(rng, mf, n, cplx)
    v0 = _haar(rng, mg, n, cplx)
    q1 = _haar(rng, n, n, cplx)
    q2 = _haar(rng, n, n, cplx)
    d = np.logspace(0.0, np.log10(cond), n) if n > 1 else np.ones(1)
    x = (q1 * d[None, :]) @ q2
    F = np.asfortranarray((u0 * sf[None, :]) @ x)
    G = np.asfortranarray((v0 * sg[None, :]) @ x)
    return Pair(F=F, G=G, sigma=np.sort(sig)[::-1].copy(), cond_x=float(cond), seed=seed)


def make_graded_pair(mf: int, mg: int, n: int, kappa_b_exp: float, *, seed: int = 0) -> tuple:
    """A pair in the manner of the GSVD-versus-GEVD experiment of App. G:
    A = F^T F with cond(A) = 10 (F = U0 diag(f) Q with f log-spaced in
    [1, sqrt(10)]) and G = V0 C diag(d) with C well conditioned (cond 2) and
    d log-spaced in [10^(-kappa_b_exp / 2), 1] in a seeded order, so that
    cond(B) = cond(G^T G) is about 10^kappa_b_exp through the column scaling
    of G alone.  Real float64, column-major; the reference sigma of the
    rounded pair is to be computed, not generated."""
    rng = np.random.default_rng(seed)
    f = np.logspace(0.0, 0.5, n)
    F = (_haar(rng, mf, n, False) * f[None, :]) @ _haar(rng, n, n, False)
    c = np.logspace(0.0, np.log10(2.0), n)
    C = (_haar(rng, n, n, False) * c[None, :]) @ _haar(rng, n, n, False)
    d = np.logspace(0.0, -kappa_b_exp / 2.0, n)[rng.permutation(n)]
    G = (_haar(rng, mg, n, False) @ C) * d[None, :]
    return np.asfortranarray(F), np.asfortranarray(G)


def batch_shapes(count: int, *, n_lo: int = 16, n_hi: int = 256, seed: int = 0):
    """Shapes (mF, mG, n) of a batch: n log-uniform in [n_lo, n_hi], mF, mG uniform in [n, 2n]."""
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(count):
        n = int(round(np.exp(rng.uniform(np.log(n_lo), np.log(n_hi)))))
        n = min(max(n, n_lo), n_hi)
        mf = int(rng.integers(n, 2 * n + 1))
        mg = int(rng.integers(n, 2 * n + 1))
        out.append((mf, mg, n))
    return out


# The benchmark configurations (shapes and value ranges), named by what they are.
POINTWISE_64x32 = dict(mf=64, mg=48, n=32, lo=1e-2, hi=1e2, cond=1e2, cplx=False, seed=0)
BLOCKED_REAL_4096x2048 = dict(mf=4096, mg=4096, n=2048, lo=1e-4, hi=1e4, cond=1e3, cplx=False, seed=0)
BLOCKED_CPLX_3072x1024 = dict(mf=3072, mg=2048, n=1024, lo=1e-3, hi=1e3, cond=1e3, cplx=True, seed=0)
