"""The oracle -- TEST INFRASTRUCTURE ONLY.

A plain, slow CPU implementation of the one-sided implicit Hari-Zimmermann
GSVD (Novakovic & Singer, arXiv 1909.00101): pointwise, sequential
row-cyclic, any variant of Table "Variants" (Sec. 2.6; variant 0 by
default) with per-step sorting, in double precision (``*_d``) and in long
double (``*_ld``, reference values of the rounded inputs).
The arithmetic lives in ``hz_oracle.c``; this module only compiles it,
marshals NumPy arrays through ctypes and returns the results.

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline
leg may import this package.  It shares no code with the CUDA library.

Every function here is pinned by ``tests/test_oracle_pins.py`` (closed
forms, the worked example of Appendix G, brute force on tiny inputs,
generated pairs with known generalized singular values, invariants).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "hz_oracle.c")
_LIB_PATH = os.path.join(_HERE, "_build", "libhz_oracle.so")
_lock = threading.Lock()
_lib = None

STATUS = {0: "OK", -1: "EINVAL", -3: "ENOCONV", -4: "ENOTPD"}


class _Opts(ctypes.Structure):
    _fields_ = [("max_sweeps", ctypes.c_int32), ("sort", ctypes.c_int32),
                ("criterion", ctypes.c_int32), ("max_pivots", ctypes.c_int32),
                ("enhanced", ctypes.c_int32), ("dscale", ctypes.c_int32)]


class _Stats(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int32), ("sweeps", ctypes.c_int32),
                ("transf_all", ctypes.c_int64), ("transf_big", ctypes.c_int64),
                ("presorted", ctypes.c_int32), ("pad", ctypes.c_int32)]


def build(force: bool = False, src: str = _SRC, lib_path: str = _LIB_PATH) -> str:
    """Compile hz_oracle.c twice (double and long double) into one .so."""
    out_dir = os.path.dirname(lib_path)
    os.makedirs(out_dir, exist_ok=True)
    if not force and os.path.exists(lib_path) and os.path.getmtime(lib_path) >= os.path.getmtime(src):
        return lib_path
    flags = ["-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-std=c11", "-Wall"]
    o_d = os.path.join(out_dir, "hz_oracle_d.%d.o" % os.getpid())
    o_ld = os.path.join(out_dir, "hz_oracle_ld.%d.o" % os.getpid())
    subprocess.check_call(["gcc", *flags, "-c", src, "-o", o_d])
    subprocess.check_call(["gcc", *flags, "-DHZO_EXTENDED", "-c", src, "-o", o_ld])
    tmp = lib_path + ".tmp%d" % os.getpid()
    subprocess.check_call(["gcc", "-shared", "-o", tmp, o_d, o_ld, "-lm"])
    os.replace(tmp, lib_path)
    os.remove(o_d)
    os.remove(o_ld)
    return lib_path


def _load(lib_path: str | None = None):
    """Load (building if needed) the oracle library; another path loads a separate copy."""
    global _lib
    with _lock:
        if lib_path is not None:
            return _bind(ctypes.CDLL(lib_path))
        if _lib is None:
            _lib = _bind(ctypes.CDLL(build()))
    return _lib


def _bind(lib):
    dp = ctypes.POINTER(ctypes.c_double)
    for suf in ("d", "ld"):
        for kind in ("real", "cplx"):
            fn = getattr(lib, "hzo_gsvd_%s_%s" % (kind, suf))
            fn.restype = ctypes.c_int
            fn.argtypes = [ctypes.c_int64] * 3 + [dp, ctypes.c_int64, dp, ctypes.c_int64,
                                                  dp, ctypes.c_int64, dp, dp, dp,
                                                  ctypes.POINTER(_Opts), ctypes.POINTER(_Stats)]
        fr = getattr(lib, "hzo_pivot_real_%s" % suf)
        fr.restype = ctypes.c_int
        fr.argtypes = [ctypes.c_double] * 4 + [ctypes.c_int32, dp, ctypes.POINTER(ctypes.c_int32)]
        fc = getattr(lib, "hzo_pivot_cplx_%s" % suf)
        fc.restype = ctypes.c_int
        fc.argtypes = [ctypes.c_double, ctypes.c_double, dp, dp, ctypes.c_int32, dp,
                       ctypes.POINTER(ctypes.c_int32)]
        fr = getattr(lib, "hzo_pivot_real_dscaled_%s" % suf)
        fr.restype = ctypes.c_int
        fr.argtypes = [ctypes.c_double] * 6 + [ctypes.c_int32, dp, ctypes.POINTER(ctypes.c_int32)]
        fc = getattr(lib, "hzo_pivot_cplx_dscaled_%s" % suf)
        fc.restype = ctypes.c_int
        fc.argtypes = [ctypes.c_double, ctypes.c_double, dp, ctypes.c_double, ctypes.c_double, dp,
                       ctypes.c_int32, dp, ctypes.POINTER(ctypes.c_int32)]
        fd = getattr(lib, "hzo_dot_real_%s" % suf)
        fd.restype = ctypes.c_double
        fd.argtypes = [dp, dp, ctypes.c_int64, ctypes.c_int32]
        fn = getattr(lib, "hzo_nrm2sq_cplx_%s" % suf)
        fn.restype = ctypes.c_double
        fn.argtypes = [dp, ctypes.c_int64, ctypes.c_int32]
    return lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def gsvd(F, G, *, max_sweeps: int = 100, sort: bool = True, criterion: int = 1,
         extended: bool = False, max_pivots: int = 0, variant: int | None = None, lib=None) -> dict:
    """GSVD of (F, G) by the oracle.

    F (mF x n) and G (mG x n) are real float64 or complex128 arrays.  Returns
    a dict with U, V, Z, sigma_f, sigma_g, sigma (sorted descending), status
    (0 = OK), sweeps, transf_all, transf_big and presorted (the final sort
    found the columns in order).  ``extended`` runs the long double
    instantiation (80-bit on x86-64, 128-bit on AArch64).  ``variant`` (0-7,
    Table "Variants" of Sec. 2.6) sets the enhanced dot products (+1), the
    D-hat rescaling (+2) and criterion C2 (+4), overriding ``criterion``.
    """
    enhanced = dscale = 0
    if variant is not None:
        if not 0 <= variant <= 7:
            raise ValueError("variant must be 0..7")
        enhanced, dscale, criterion = variant & 1, (variant >> 1) & 1, 2 if variant & 4 else 1
    F = np.asarray(F)
    G = np.asarray(G)
    cplx = np.iscomplexobj(F) or np.iscomplexobj(G)
    dt = np.complex128 if cplx else np.float64
    Fw = np.array(F, dtype=dt, order="F", copy=True)
    Gw = np.array(G, dtype=dt, order="F", copy=True)
    mf, n = Fw.shape
    mg, n2 = Gw.shape
    if n2 != n:
        raise ValueError("F and G must have the same number of columns")
    Zw = np.zeros((n, n), dtype=dt, order="F")
    sf = np.zeros(n)
    sg = np.zeros(n)
    sig = np.zeros(n)
    opts = _Opts(max_sweeps, 1 if sort else 0, criterion, max_pivots, enhanced, dscale)
    st = _Stats()
    lib = lib or _load()
    fn = getattr(lib, "hzo_gsvd_%s_%s" % ("cplx" if cplx else "real", "ld" if extended else "d"))
    fn(mf, mg, n, _ptr(Fw), max(mf, 1), _ptr(Gw), max(mg, 1), _ptr(Zw), max(n, 1),
       _ptr(sf), _ptr(sg), _ptr(sig), ctypes.byref(opts), ctypes.byref(st))
    return dict(U=Fw, V=Gw, Z=Zw, sigma_f=sf, sigma_g=sg, sigma=sig, status=st.status,
                sweeps=st.sweeps, transf_all=st.transf_all, transf_big=st.transf_big,
                presorted=bool(st.presorted))


def pivot_real(a11, a22, a12, x, *, criterion: int = 1, extended: bool = False, lib=None):
    """The real 2x2 transformation of Sec. 2.1.2: returns (Zhat 2x2, small, status)."""
    lib = lib or _load()
    z = np.zeros(4)
    sm = ctypes.c_int32(0)
    fn = getattr(lib, "hzo_pivot_real_%s" % ("ld" if extended else "d"))
    st = fn(float(a11), float(a22), float(a12), float(x), criterion, _ptr(z), ctypes.byref(sm))
    return z.reshape(2, 2), bool(sm.value), st


def pivot_cplx(a11, a22, a12, b12, *, criterion: int = 1, extended: bool = False, lib=None):
    """The complex 2x2 transformation of Sec. 2.1.1: returns (Zhat 2x2, small, status)."""
    lib = lib or _load()
    a = np.array([complex(a12).real, complex(a12).imag])
    b = np.array([complex(b12).real, complex(b12).imag])
    z = np.zeros(8)
    sm = ctypes.c_int32(0)
    fn = getattr(lib, "hzo_pivot_cplx_%s" % ("ld" if extended else "d"))
    st = fn(float(a11), float(a22), _ptr(a), _ptr(b), criterion, _ptr(z), ctypes.byref(sm))
    return z.view(np.complex128).reshape(2, 2), bool(sm.value), st


def pivot_real_dscaled(a11, a22, a12, b11, b22, b12, *, criterion: int = 1, extended: bool = False, lib=None):
    """The real 2x2 transformation of the D-hat variants (Sec. 2.1): Z-hat' of
    D A D, D B D and Z-hat = D Z-hat'; returns (Zhat 2x2, small, status)."""
    lib = lib or _load()
    z = np.zeros(4)
    sm = ctypes.c_int32(0)
    fn = getattr(lib, "hzo_pivot_real_dscaled_%s" % ("ld" if extended else "d"))
    st = fn(float(a11), float(a22), float(a12), float(b11), float(b22), float(b12), criterion, _ptr(z),
            ctypes.byref(sm))
    return z.reshape(2, 2), bool(sm.value), st


def pivot_cplx_dscaled(a11, a22, a12, b11, b22, b12, *, criterion: int = 1, extended: bool = False, lib=None):
    """The complex 2x2 transformation of the D-hat variants: (Zhat 2x2, small, status)."""
    lib = lib or _load()
    a = np.array([complex(a12).real, complex(a12).imag])
    b = np.array([complex(b12).real, complex(b12).imag])
    z = np.zeros(8)
    sm = ctypes.c_int32(0)
    fn = getattr(lib, "hzo_pivot_cplx_dscaled_%s" % ("ld" if extended else "d"))
    st = fn(float(a11), float(a22), _ptr(a), float(b11), float(b22), _ptr(b), criterion, _ptr(z),
            ctypes.byref(sm))
    return z.view(np.complex128).reshape(2, 2), bool(sm.value), st


def dot_real(a, b, *, enhanced: bool = False, extended: bool = False, lib=None) -> float:
    """a^T b of two real vectors, ordinary (sequential) or enhanced (App. A)."""
    lib = lib or _load()
    a = np.ascontiguousarray(a, dtype=np.float64)
    b = np.ascontiguousarray(b, dtype=np.float64)
    fn = getattr(lib, "hzo_dot_real_%s" % ("ld" if extended else "d"))
    return fn(_ptr(a), _ptr(b), a.size, 1 if enhanced else 0)


def nrm2sq_cplx(a, *, enhanced: bool = False, extended: bool = False, lib=None) -> float:
    """||a||^2 of a complex vector, ordinary or enhanced (App. A, the simpler procedure)."""
    lib = lib or _load()
    a = np.ascontiguousarray(a, dtype=np.complex128)
    fn = getattr(lib, "hzo_nrm2sq_cplx_%s" % ("ld" if extended else "d"))
    return fn(_ptr(a.view(np.float64)), a.size, 1 if enhanced else 0)
