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
   distributed: Gram-Schmidt of a Gaussian matrix, which leaves R with a
   positive diagonal (Mezzadri 2007);
4. X = Q1 diag(d) Q2 with Q1, Q2 Haar and d log-spaced in [1, cond];
5. F = U0 Sigma_F X, G = V0 Sigma_G X, so that F X^{-1} = U0 Sigma_F and
   G X^{-1} = V0 Sigma_G: the exact GSVD of (F, G) has Z = X^{-1} up to
   column order and unit scalars.

Every number is computed by ``inputs_gen.c`` with a fixed sequence of
correctly rounded IEEE operations (its own random streams, ln and exp; no
BLAS, LAPACK or libm transcendental; no fused multiply-add), so a pair is
the same bytes on x86-64 and AArch64.  ``sha256(pair)`` names a pair by its
bytes; reference values computed once on one machine are keyed by it.
"""
from __future__ import annotations

import ctypes
import hashlib
import os
import subprocess
import threading
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "inputs_gen.c")
_LIB_PATH = os.path.join(_HERE, "_build", "libinputs_gen.so")
_lock = threading.Lock()
_lib = None

# stream ids of one pair's random draws
_S_PERM, _S_U0, _S_V0, _S_Q1, _S_Q2, _S_SHAPES, _S_GRADE = 0, 1, 2, 3, 4, 5, 6


def build(force: bool = False) -> str:
    """Compile inputs_gen.c (with OpenMP where the compiler has it)."""
    os.makedirs(os.path.dirname(_LIB_PATH), exist_ok=True)
    if not force and os.path.exists(_LIB_PATH) and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC):
        return _LIB_PATH
    tmp = _LIB_PATH + ".tmp%d" % os.getpid()
    base = ["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared", "-std=gnu11", "-Wall"]
    try:
        subprocess.check_call(base + ["-fopenmp", _SRC, "-o", tmp, "-lm"], stderr=subprocess.DEVNULL)
    except subprocess.CalledProcessError:
        subprocess.check_call(base + [_SRC, "-o", tmp, "-lm"])
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            # threads that wait at a barrier sleep instead of spinning (the
            # generator may share the cores with other work)
            os.environ.setdefault("OMP_WAIT_POLICY", "passive")
            lib = ctypes.CDLL(build())
            dp = ctypes.POINTER(ctypes.c_double)
            i64, u64, i32 = ctypes.c_int64, ctypes.c_uint64, ctypes.c_int32
            lib.ig_log.argtypes = [ctypes.c_double]
            lib.ig_log.restype = ctypes.c_double
            lib.ig_exp.argtypes = [ctypes.c_double]
            lib.ig_exp.restype = ctypes.c_double
            lib.ig_uniform.argtypes = [u64, u64, i64, dp]
            lib.ig_gauss.argtypes = [u64, u64, i64, dp]
            lib.ig_permutation.argtypes = [u64, u64, i64, ctypes.POINTER(i64)]
            lib.ig_logspace.argtypes = [ctypes.c_double, ctypes.c_double, i64, dp]
            lib.ig_orthonormalize.argtypes = [i64, i64, dp, i32, i32]
            lib.ig_orthonormalize.restype = ctypes.c_int
            lib.ig_scale_cols.argtypes = [i64, i64, dp, i64, dp, i32]
            lib.ig_gemm.argtypes = [i64, i64, i64, dp, i64, dp, i64, dp, i64, i32, i32]
            _lib = lib
    return _lib


def _p(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _threads(work: float = 1e12) -> int:
    """Threads for a job of about `work` multiply-adds: one below 2^24 (the
    parallel regions would cost more than they save), else every core.  The
    results do not depend on the thread count."""
    if work < 2.0 ** 24:
        return 1
    try:
        return max(1, len(os.sched_getaffinity(0)))
    except AttributeError:
        return os.cpu_count() or 1


def uniform(seed: int, stream: int, count: int) -> np.ndarray:
    out = np.empty(count)
    _load().ig_uniform(seed, stream, count, _p(out))
    return out


def logspace(lo: float, hi: float, n: int) -> np.ndarray:
    """n values log-spaced in [lo, hi] (n >= 2), platform-independent."""
    out = np.empty(n)
    _load().ig_logspace(float(lo), float(hi), n, _p(out))
    return out


def permutation(seed: int, stream: int, n: int) -> np.ndarray:
    out = np.empty(n, dtype=np.int64)
    _load().ig_permutation(seed, stream, n, out.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)))
    return out


def haar(seed: int, stream: int, m: int, n: int, cplx: bool = False) -> np.ndarray:
    """m x n with orthonormal (unitary) columns, Haar distributed, column-major."""
    lib = _load()
    g = np.empty(m * n * (2 if cplx else 1))
    lib.ig_gauss(seed, stream, g.size, _p(g))
    st = lib.ig_orthonormalize(m, n, _p(g), 1 if cplx else 0, _threads(2.0 * m * n * n))
    if st != 0:
        raise RuntimeError("Gram-Schmidt of a Gaussian matrix failed (%d)" % st)
    return _as_matrix(g, m, n, cplx)


def _as_matrix(buf: np.ndarray, m: int, n: int, cplx: bool) -> np.ndarray:
    if cplx:
        return buf.view(np.complex128).reshape((n, m)).T
    return buf.reshape((n, m)).T


def _buf(a: np.ndarray) -> np.ndarray:
    """The column-major float64 buffer of a (a view when a is Fortran-ordered)."""
    a = np.asfortranarray(a)
    return a.reshape(-1, order="F").view(np.float64)


def scale_cols(a: np.ndarray, s: np.ndarray) -> np.ndarray:
    """a * s[None, :] (a fresh column-major matrix)."""
    m, n = a.shape
    cplx = np.iscomplexobj(a)
    b = np.array(a, order="F", copy=True)
    bb = _buf(b)
    s = np.ascontiguousarray(s, dtype=np.float64)
    _load().ig_scale_cols(m, n, _p(bb), m, _p(s), 1 if cplx else 0)
    return b


def matmul(a: np.ndarray, b: np.ndarray) -> np.ndarray:
    """a @ b with every entry summed in increasing k (platform-independent)."""
    m, k = a.shape
    k2, n = b.shape
    assert k == k2
    cplx = np.iscomplexobj(a) or np.iscomplexobj(b)
    dt = np.complex128 if cplx else np.float64
    a = np.asfortranarray(a, dtype=dt)
    b = np.asfortranarray(b, dtype=dt)
    c = np.empty((m, n), dtype=dt, order="F")
    _load().ig_gemm(m, n, k, _p(_buf(a)), m, _p(_buf(b)), k, _p(_buf(c)), m, 1 if cplx else 0,
                    _threads(float(m) * n * k))
    return c


def sha256(F: np.ndarray, G: np.ndarray) -> str:
    """Hex SHA-256 of the column-major bytes of F followed by those of G."""
    h = hashlib.sha256()
    h.update(np.asfortranarray(F).tobytes(order="F"))
    h.update(np.asfortranarray(G).tobytes(order="F"))
    return h.hexdigest()


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
    sig = logspace(lo, hi, n) if n > 1 else np.array([np.sqrt(lo * hi)])
    sig = sig[permutation(seed, _S_PERM, n)]
    den = np.sqrt(1.0 + sig * sig)
    sf = sig / den
    sg = 1.0 / den
    u0 = haar(seed, _S_U0, mf, n, cplx)
    v0 = haar(seed, _S_V0, mg, n, cplx)
    q1 = haar(seed, _S_Q1, n, n, cplx)
    q2 = haar(seed, _S_Q2, n, n, cplx)
    d = logspace(1.0, cond, n) if n > 1 else np.ones(1)
    x = matmul(scale_cols(q1, d), q2)
    F = matmul(scale_cols(u0, sf), x)
    G = matmul(scale_cols(v0, sg), x)
    return Pair(F=F, G=G, sigma=np.sort(sig)[::-1].copy(), cond_x=float(cond), seed=seed)


def make_graded_pair(mf: int, mg: int, n: int, kappa_b_exp: float, *, seed: int = 0) -> tuple:
    """A pair in the manner of the GSVD-versus-GEVD experiment of App. G:
    A = F^T F with cond(A) = 10 (F = U0 diag(f) Q with f log-spaced in
    [1, sqrt(10)]) and G = V0 C diag(d) with C well conditioned (cond 2) and
    d log-spaced in [10^(-kappa_b_exp / 2), 1] in a seeded order, so that
    cond(B) = cond(G^T G) is about 10^kappa_b_exp through the column scaling
    of G alone.  Real float64, column-major; the reference sigma of the
    rounded pair is to be computed, not generated."""
    f = logspace(1.0, np.sqrt(10.0), n)
    F = matmul(scale_cols(haar(seed, _S_U0, mf, n), f), haar(seed, _S_Q1, n, n))
    c = logspace(1.0, 2.0, n)
    C = matmul(scale_cols(haar(seed, _S_Q2, n, n), c), haar(seed, _S_GRADE, n, n))
    lib = _load()
    d = logspace(1.0, lib.ig_exp(-kappa_b_exp / 2.0 * lib.ig_log(10.0)), n)[permutation(seed, _S_PERM, n)]
    G = scale_cols(matmul(haar(seed, _S_V0, mg, n), C), d)
    return F, G


def batch_shapes(count: int, *, n_lo: int = 16, n_hi: int = 256, seed: int = 0):
    """Shapes (mF, mG, n) of a batch: n log-uniform in [n_lo, n_hi], mF, mG uniform in [n, 2n]."""
    lib = _load()
    u = uniform(seed, _S_SHAPES, 3 * count)
    a, b = lib.ig_log(float(n_lo)), lib.ig_log(float(n_hi))
    out = []
    for k in range(count):
        n = int(round(lib.ig_exp(a + (b - a) * float(u[3 * k]))))
        n = min(max(n, n_lo), n_hi)
        mf = n + min(int(u[3 * k + 1] * (n + 1)), n)
        mg = n + min(int(u[3 * k + 2] * (n + 1)), n)
        out.append((mf, mg, n))
    return out


# The benchmark configurations (shapes and value ranges), named by what they are.
POINTWISE_64x32 = dict(mf=64, mg=48, n=32, lo=1e-2, hi=1e2, cond=1e2, cplx=False, seed=0)
BLOCKED_REAL_4096x2048 = dict(mf=4096, mg=4096, n=2048, lo=1e-4, hi=1e4, cond=1e3, cplx=False, seed=0)
BLOCKED_CPLX_3072x1024 = dict(mf=3072, mg=2048, n=1024, lo=1e-3, hi=1e3, cond=1e3, cplx=True, seed=0)
