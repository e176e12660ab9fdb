"""Out-of-bounds write checks (GPU): every caller buffer is embedded in a
larger allocation whose padding holds a canary value -- leading dimensions
larger than the row counts (ld > m, odd paddings) and guard words after the
sigma vectors.  After the solve the padding must be bitwise unchanged and the
result must still be the oracle's GSVD (the solver honours ld everywhere).
"""
import numpy as np
import pytest

import oracle
from paper_1909_00101_gb300.inputs import make_pair
from gsvd_checks import rel_sigma_err

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

CANARY = -1234.5678


@pytest.fixture(scope="module")
def hz():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1909_00101_gb300.build import build
    build()
    import paper_1909_00101_gb300 as m
    m.load_library()
    return m


def _padded(a, pad):
    """Column-major device matrix a (m x n) inside an (m + pad) x n buffer
    whose extra rows hold the canary; returns (buffer, view)."""
    m, n = a.shape
    dt = torch.complex128 if np.iscomplexobj(a) else torch.float64
    buf = torch.full((n, m + pad), CANARY, dtype=dt, device="cuda")
    view = buf.t()[:m, :]
    view.copy_(torch.from_numpy(np.asarray(a)))
    return buf, view


def _guarded(n):
    buf = torch.full((n + 8,), CANARY, dtype=torch.float64, device="cuda")
    return buf, buf[:n]


@pytest.mark.parametrize("kw,shape,cplx", [
    (dict(path="pointwise"), (64, 48, 32), False),
    (dict(path="blocked", block_w=8, shorten=0), (200, 150, 96), False),
    (dict(path="blocked", block_w=8), (400, 300, 96), False),          # shortened
    (dict(path="blocked", block_w=8, precision="mixed", shorten=0), (200, 150, 96), False),
    (dict(path="blocked", block_w=4), (160, 130, 64), True),
])
def test_padding_untouched(hz, kw, shape, cplx):
    mf, mg, n = shape
    p = make_pair(mf, mg, n, cplx=cplx, seed=n + mf)
    Fb, F = _padded(p.F, 37)
    Gb, G = _padded(p.G, 5)
    Zb, Z = _padded(np.zeros((n, n), dtype=p.F.dtype), 11)
    vb = [_guarded(n) for _ in range(3)]
    s = hz.Solver(**kw)
    prob = hz._problem(F, G, Z, vb[0][1], vb[1][1], vb[2][1], True)
    import ctypes
    info = hz.Info()
    torch.cuda.synchronize()
    st = s._lib.gsvd_solve(s._h, ctypes.byref(prob), ctypes.byref(info))
    torch.cuda.synchronize()
    s.close()
    assert st == 0, info.as_dict()
    for buf, m in ((Fb, mf), (Gb, mg), (Zb, n)):
        pad = buf.t()[m:, :]
        assert bool(torch.all(pad == CANARY)), "padding rows written"
    for buf, _ in vb:
        assert bool(torch.all(buf[n:] == CANARY)), "guard words after a sigma vector written"
    ref = oracle.gsvd(p.F, p.G, extended=True)
    tol = 1e-10 if kw.get("precision") == "mixed" else 1e-11
    assert rel_sigma_err(vb[2][1].cpu().numpy(), ref["sigma"]) <= tol
