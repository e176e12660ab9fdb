"""GB300 implicit Hari-Zimmermann GSVD engine: thin Python binding of the C ABI.

Every step of the solve runs in the CUDA library ``_build/libgsvd_gb300.so``
(declared in ``include/gsvd.h``); this module only marshals arguments.  There
is no CPU fallback: if the library is missing, importing the binding's entry
points raises.

    import torch, paper_1909_00101_gb300 as hz
    F = torch.randn(64, 32, dtype=torch.float64, device="cuda")   # any strides ok
    G = torch.randn(48, 32, dtype=torch.float64, device="cuda")
    r = hz.solve(F, G)            # r.U, r.V, r.Z, r.sigma_f, r.sigma_g, r.sigma, r.info

Matrices are used column-major (a tensor whose stride(0) == 1); other
layouts are copied.  Paper: Novakovic & Singer, arXiv 1909.00101.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libgsvd_gb300.so")

OK, EAGAIN, EINVAL, ENOMEM, ENOCONV, ENOTPD, EOVERFLOW, ETIMEOUT, ECUDA, ETOOBIG = 0, 1, -1, -2, -3, -4, -5, -6, -7, -8
R64, C128 = 0, 1
PREC = {"fp64": 0, "mixed": 1}
PATH = {"auto": 0, "pointwise": 1, "blocked": 2}
ORDER = {"round_robin": 0, "row_cyclic": 1}


class Config(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int32), ("block_w", ctypes.c_int32), ("max_sweeps", ctypes.c_int32),
                ("inner_max_sweeps", ctypes.c_int32), ("criterion", ctypes.c_int32), ("sort", ctypes.c_int32),
                ("path", ctypes.c_int32), ("order", ctypes.c_int32), ("fp32_max_sweeps", ctypes.c_int32),
                ("timeout_ms", ctypes.c_int32), ("hbm_budget_bytes", ctypes.c_uint64),
                ("max_inflight", ctypes.c_int32), ("profile", ctypes.c_int32),
                ("inner_max_sweeps_fp32", ctypes.c_int32), ("shorten", ctypes.c_int32),
                ("fp32_params", ctypes.c_int32), ("fp64_gemm", ctypes.c_int32),
                ("fp32_stop_permille", ctypes.c_int32), ("variant", ctypes.c_int32)]


class Problem(ctypes.Structure):
    _fields_ = [("dtype", ctypes.c_int32), ("reserved", ctypes.c_int32), ("m_f", ctypes.c_int64),
                ("m_g", ctypes.c_int64), ("n", ctypes.c_int64), ("F", ctypes.c_void_p), ("ldf", ctypes.c_int64),
                ("G", ctypes.c_void_p), ("ldg", ctypes.c_int64), ("Z", ctypes.c_void_p), ("ldz", ctypes.c_int64),
                ("sigma_f", ctypes.c_void_p), ("sigma_g", ctypes.c_void_p), ("sigma", ctypes.c_void_p),
                ("X", ctypes.c_void_p), ("ldx", ctypes.c_int64)]


class Info(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int32), ("sweeps_fp32", ctypes.c_int32), ("sweeps_fp64", ctypes.c_int32),
                ("path", ctypes.c_int32), ("transf_all", ctypes.c_uint64), ("transf_big", ctypes.c_uint64),
                ("t_total_us", ctypes.c_double), ("t_fp32_us", ctypes.c_double), ("t_refine_us", ctypes.c_double),
                ("block_w", ctypes.c_int32), ("chol_skipped", ctypes.c_int32),
                ("visits", ctypes.c_uint64), ("visits_applied", ctypes.c_uint64),
                ("t_kernel_us", ctypes.c_double * 6), ("n_kernel", ctypes.c_int32 * 6),
                ("visits_fp32", ctypes.c_uint64), ("visits_applied_fp32", ctypes.c_uint64),
                ("shortened", ctypes.c_int32), ("shorten_skipped", ctypes.c_int32), ("t_qr_us", ctypes.c_double),
                ("qr_launches", ctypes.c_int32), ("reserved2", ctypes.c_int32)]

    def as_dict(self) -> dict:
        d = {}
        for k, _ in self._fields_:
            v = getattr(self, k)
            d[k] = list(v) if k in ("t_kernel_us", "n_kernel") else v
        return d


ENTRY_POINTS = ("gsvd_config_default", "gsvd_create", "gsvd_destroy", "gsvd_solve", "gsvd_solve_batched",
                "gsvd_submit", "gsvd_poll", "gsvd_workspace_bytes", "gsvd_strerror", "gsvd_solve_small_noalloc")
NOALLOC_MAX_PROBLEMS = 4096

_lib = None


def load_library(path: str = LIB_PATH):
    """Load the CUDA library (raises if it has not been built)."""
    global _lib
    if _lib is not None and path == LIB_PATH:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError("GSVD CUDA library not built (%s); run __graft_entry__.build()" % path)
    lib = ctypes.CDLL(path)
    P = ctypes.POINTER
    lib.gsvd_config_default.argtypes = [P(Config)]
    lib.gsvd_config_default.restype = None
    lib.gsvd_create.argtypes = [P(ctypes.c_void_p), P(Config), ctypes.c_void_p]
    lib.gsvd_destroy.argtypes = [ctypes.c_void_p]
    lib.gsvd_solve.argtypes = [ctypes.c_void_p, P(Problem), P(Info)]
    lib.gsvd_solve_batched.argtypes = [ctypes.c_void_p, P(Problem), ctypes.c_int32, P(Info)]
    lib.gsvd_submit.argtypes = [ctypes.c_void_p, P(Problem), P(ctypes.c_uint64)]
    lib.gsvd_poll.argtypes = [ctypes.c_void_p, ctypes.c_uint64, P(Info)]
    lib.gsvd_workspace_bytes.argtypes = [P(Config), ctypes.c_int32, ctypes.c_int64, ctypes.c_int64, ctypes.c_int64]
    lib.gsvd_workspace_bytes.restype = ctypes.c_uint64
    lib.gsvd_strerror.argtypes = [ctypes.c_int]
    lib.gsvd_strerror.restype = ctypes.c_char_p
    lib.gsvd_solve_small_noalloc.argtypes = [P(Problem), ctypes.c_int32, P(Config), ctypes.c_void_p, P(Info)]
    lib.gsvd_solve_small_noalloc.restype = ctypes.c_int
    for name in ("gsvd_create", "gsvd_destroy", "gsvd_solve", "gsvd_solve_batched", "gsvd_submit", "gsvd_poll"):
        getattr(lib, name).restype = ctypes.c_int
    if path == LIB_PATH:
        _lib = lib
    return lib


def strerror(status: int) -> str:
    return load_library().gsvd_strerror(status).decode()


def make_config(precision="fp64", block_w=0, max_sweeps=30, inner_max_sweeps=30, criterion=1, sort=True,
                path="auto", order="round_robin", fp32_max_sweeps=30, hbm_budget_bytes=60 << 30,
                max_inflight=16, profile=False, inner_max_sweeps_fp32=1, shorten=1,
                fp32_params=1, fp64_gemm=1, fp32_stop_permille=50, variant=0, timeout_ms=0) -> Config:
    c = Config()
    load_library().gsvd_config_default(ctypes.byref(c))
    c.precision = PREC[precision]
    c.block_w = block_w
    c.max_sweeps = max_sweeps
    c.inner_max_sweeps = inner_max_sweeps
    c.criterion = criterion
    c.sort = 1 if sort else 0
    c.path = PATH[path]
    c.order = ORDER[order]
    c.fp32_max_sweeps = fp32_max_sweeps
    c.hbm_budget_bytes = hbm_budget_bytes
    c.max_inflight = max_inflight
    c.profile = 1 if profile else 0
    c.inner_max_sweeps_fp32 = inner_max_sweeps_fp32
    c.shorten = shorten
    c.fp32_params = fp32_params
    c.fp64_gemm = fp64_gemm
    c.fp32_stop_permille = fp32_stop_permille
    c.variant = variant
    c.timeout_ms = timeout_ms
    return c


@dataclass
class Result:
    U: object
    V: object
    Z: object
    sigma_f: object
    sigma_g: object
    sigma: object
    info: dict = field(default_factory=dict)
    X: object = None  # right vectors X = Z^-1 when requested

    @property
    def status(self) -> int:
        return self.info.get("status", 0)


def _colmajor(t, dev):
    """A column-major view (stride(0) == 1) of t; copies when t is not one."""
    if dev:
        if t.dim() == 2 and t.stride(0) == 1 and t.stride(1) >= max(1, t.shape[0]):
            return t
        return t.t().contiguous().t()
    if t.flags.f_contiguous:
        return t
    return np.asfortranarray(t)


def _ld(t, dev):
    """Leading dimension (elements) of a column-major matrix; a single column has
    no meaningful column stride, so its ld is its row count."""
    m, n = t.shape
    if n <= 1:
        return max(1, m)
    return t.stride(1) if dev else t.strides[1] // t.itemsize


def _problem(F, G, Z, sf, sg, sig, dev) -> Problem:
    p = Problem()
    cplx = (F.is_complex() if dev else np.iscomplexobj(F))
    p.dtype = C128 if cplx else R64
    p.m_f, p.n = F.shape
    p.m_g = G.shape[0]
    p.ldf, p.ldg, p.ldz = _ld(F, dev), _ld(G, dev), _ld(Z, dev)
    if dev:
        p.F, p.G, p.Z = F.data_ptr(), G.data_ptr(), Z.data_ptr()
        p.sigma_f, p.sigma_g, p.sigma = sf.data_ptr(), sg.data_ptr(), sig.data_ptr()
    else:
        p.F, p.G, p.Z = F.ctypes.data, G.ctypes.data, Z.ctypes.data
        p.sigma_f, p.sigma_g, p.sigma = sf.ctypes.data, sg.ctypes.data, sig.ctypes.data
    return p


def _prepare(F, G, inplace):
    """Output buffers for one problem: (F, G) become U, V; Z and vectors allocated."""
    dev = not isinstance(F, np.ndarray)
    if dev:
        import torch
        cplx = F.is_complex() or G.is_complex()
        dt = torch.complex128 if cplx else torch.float64
        if F.dtype != dt:
            F = F.to(dt)
        if G.dtype != dt:
            G = G.to(dt)
        Fc = _colmajor(F, True) if inplace else F.t().contiguous().t().clone(memory_format=torch.preserve_format)
        Gc = _colmajor(G, True) if inplace else G.t().contiguous().t().clone(memory_format=torch.preserve_format)
        if Fc.stride(0) != 1:
            Fc = Fc.t().contiguous().t()
        if Gc.stride(0) != 1:
            Gc = Gc.t().contiguous().t()
        n = Fc.shape[1]
        Z = torch.empty((n, n), dtype=dt, device=Fc.device).t()
        sf = torch.empty(n, dtype=torch.float64, device=Fc.device)
        sg = torch.empty_like(sf)
        sig = torch.empty_like(sf)
    else:
        cplx = np.iscomplexobj(F) or np.iscomplexobj(G)
        dt = np.complex128 if cplx else np.float64
        Fc = np.array(F, dtype=dt, order="F", copy=not inplace)
        Gc = np.array(G, dtype=dt, order="F", copy=not inplace)
        n = Fc.shape[1]
        Z = np.zeros((n, n), dtype=dt, order="F")
        sf = np.zeros(n)
        sg = np.zeros(n)
        sig = np.zeros(n)
    return dev, Fc, Gc, Z, sf, sg, sig


class Solver:
    """A handle (gsvd_create) with its configuration and stream."""

    def __init__(self, stream=None, **cfg):
        self._lib = load_library()
        self.config = make_config(**cfg)
        self._h = ctypes.c_void_p()
        s = 0
        if stream is not None:
            s = stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream)
        st = self._lib.gsvd_create(ctypes.byref(self._h), ctypes.byref(self.config), ctypes.c_void_p(s))
        if st != OK:
            raise RuntimeError("gsvd_create: " + strerror(st))

    def close(self):
        if self._h:
            self._lib.gsvd_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def solve(self, F, G, *, inplace: bool = False, right_vectors: bool = False) -> Result:
        """GSVD of (F, G): torch CUDA tensors (device path) or numpy arrays (host
        path).  right_vectors: also X = Z^-1."""
        dev, Fc, Gc, Z, sf, sg, sig = _prepare(F, G, inplace)
        p = _problem(Fc, Gc, Z, sf, sg, sig, dev)
        X = None
        if right_vectors:
            n = Z.shape[0]
            if dev:
                import torch
                X = torch.empty((n, n), dtype=Z.dtype, device=Z.device).t()
                p.X, p.ldx = X.data_ptr(), _ld(X, True)
            else:
                X = np.zeros((n, n), dtype=Z.dtype, order="F")
                p.X, p.ldx = X.ctypes.data, _ld(X, False)
        info = Info()
        if dev:
            import torch
            torch.cuda.current_stream().synchronize()
        self._lib.gsvd_solve(self._h, ctypes.byref(p), ctypes.byref(info))
        return Result(Fc, Gc, Z, sf, sg, sig, info.as_dict(), X)

    def autotune(self, m_f: int, m_g: int, n: int, cplx: bool = False) -> int:
        """gsvd_autotune: time the candidate block widths for this shape on a
        synthetic pair and record the fastest for later solves of its class;
        returns the width (0: nothing to choose)."""
        w = ctypes.c_int32(0)
        st = self._lib.gsvd_autotune(self._h, C128 if cplx else R64, ctypes.c_int64(m_f), ctypes.c_int64(m_g),
                                     ctypes.c_int64(n), ctypes.byref(w))
        if st != 0:
            raise RuntimeError("gsvd_autotune: %s" % strerror(st))
        return int(w.value)

    def solve_problems(self, probs) -> list:
        """Raw batched call on prepared Problem structs; returns the Info dicts."""
        arr = (Problem * len(probs))(*probs)
        infos = (Info * len(probs))()
        self._lib.gsvd_solve_batched(self._h, arr, len(probs), infos)
        return [i.as_dict() for i in infos]

    def solve_batched(self, pairs, *, inplace: bool = False) -> list:
        """GSVDs of a list of (F, G) device pairs in one call."""
        import torch
        preps = [_prepare(F, G, inplace) for F, G in pairs]
        probs = [_problem(Fc, Gc, Z, sf, sg, sig, True) for (_, Fc, Gc, Z, sf, sg, sig) in preps]
        torch.cuda.current_stream().synchronize()
        infos = self.solve_problems(probs)
        return [Result(Fc, Gc, Z, sf, sg, sig, inf) for (_, Fc, Gc, Z, sf, sg, sig), inf in zip(preps, infos)]

    def submit(self, F, G, *, inplace: bool = False):
        """Serving: enqueue one device problem; returns (ticket, Result buffers)."""
        dev, Fc, Gc, Z, sf, sg, sig = _prepare(F, G, inplace)
        if not dev:
            raise ValueError("submit takes device tensors")
        p = _problem(Fc, Gc, Z, sf, sg, sig, True)
        # the copies above run on torch's stream; the library's workers read
        # the buffers on their own streams, so they must be complete first
        import torch
        torch.cuda.current_stream().synchronize()
        t = ctypes.c_uint64()
        st = self._lib.gsvd_submit(self._h, ctypes.byref(p), ctypes.byref(t))
        if st != OK:
            raise RuntimeError("gsvd_submit: " + strerror(st))
        return t.value, Result(Fc, Gc, Z, sf, sg, sig, {})

    def poll(self, ticket: int):
        """EAGAIN while running; else the final status, with the Info dict."""
        info = Info()
        st = self._lib.gsvd_poll(self._h, ctypes.c_uint64(ticket), ctypes.byref(info))
        return st, info.as_dict()

    def workspace_bytes(self, dtype: int, mf: int, mg: int, n: int) -> int:
        return int(self._lib.gsvd_workspace_bytes(ctypes.byref(self.config), dtype, mf, mg, n))


def solve_small_noalloc(pairs, *, stream=None, **cfg) -> tuple:
    """Batch of small device problems (n <= 64) through gsvd_solve_small_noalloc.

    The library allocates no device memory for this call: the kernel's scratch
    is a fixed array inside the library.  For callers that must not allocate
    (a framework owning all device memory, a loop where cudaMalloc would
    synchronize).  The output buffers here are allocated by torch on the
    Python side, before the call.  Returns (status, [Result, ...]).
    """
    import torch
    lib = load_library()
    preps = [_prepare(F, G, False) for F, G in pairs]
    probs = [_problem(Fc, Gc, Z, sf, sg, sig, True) for (_, Fc, Gc, Z, sf, sg, sig) in preps]
    arr = (Problem * len(probs))(*probs)
    infos = (Info * len(probs))()
    c = make_config(**cfg)
    s = 0
    if stream is not None:
        s = stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream)
    torch.cuda.current_stream().synchronize()
    st = lib.gsvd_solve_small_noalloc(arr, len(probs), ctypes.byref(c), ctypes.c_void_p(s), infos)
    res = [Result(Fc, Gc, Z, sf, sg, sig, inf.as_dict()) for (_, Fc, Gc, Z, sf, sg, sig), inf in zip(preps, infos)]
    return st, res


def solve(F, G, *, inplace: bool = False, right_vectors: bool = False, **cfg) -> Result:
    """One-shot GSVD (creates and destroys a handle)."""
    with Solver(**cfg) as s:
        return s.solve(F, G, inplace=inplace, right_vectors=right_vectors)
