"""GPU parity of the variants of Sec. 2.6 (Table "Variants") on the
pointwise kernel and in the FP64 pivot step of the blocked path: the enhanced
dot products of App. A (+1), the D-hat rescaling (+2), and with criterion C2
the variants 4-7.  Each case runs the
library through the C ABI and the oracle in the same variant, with the
tolerance of the other parity tests (extended-precision oracle, R14 rule) and
the invariants; the row-cyclic order follows the oracle's sequence.
"""
import numpy as np
import pytest

import oracle
from paper_1909_00101_gb300.inputs import make_pair, POINTWISE_64x32
from gsvd_checks import invariants, rel_sigma_err

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def hz():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1909_00101_gb300.build import build
    build()
    import paper_1909_00101_gb300 as m
    m.load_library()
    return m


def _dev(a):
    return torch.from_numpy(np.asfortranarray(a)).cuda()


def _np(t):
    return t.cpu().numpy()


def _variant_args(variant):
    return dict(variant=variant & 3, criterion=2 if variant & 4 else 1)


def _check(p, r, variant, label):
    ref = oracle.gsvd(p.F, p.G, variant=variant)
    refx = oracle.gsvd(p.F, p.G, variant=variant, extended=True)
    assert ref["status"] == 0 and refx["status"] == 0
    sig = _np(r.sigma)
    tol = max(1e-12, 4.0 * rel_sigma_err(ref["sigma"], refx["sigma"]))
    err = rel_sigma_err(sig, refx["sigma"])
    print("%s variant %d: sigma err %.2e (tol %.2e), info %s" % (label, variant, err, tol, r.info))
    assert r.status == 0, r.info
    assert err <= tol
    n = p.F.shape[1]
    inv = invariants(p.F, p.G, _np(r.U), _np(r.V), _np(r.Z), _np(r.sigma_f), _np(r.sigma_g), sig)
    assert inv["FZ"] <= 1e-13 * n and inv["GZ"] <= 1e-13 * n, inv
    assert inv["UU"] <= 1e-12 * n and inv["VV"] <= 1e-12 * n, inv
    assert inv["scale"] <= 8 * 2.0 ** -53 and inv["sorted"], inv
    return ref


@pytest.mark.parametrize("variant", range(1, 8))
@pytest.mark.parametrize("cplx", [False, True])
def test_pointwise_variants_match_the_oracle(hz, variant, cplx):
    p = make_pair(48, 40, 24, cplx=cplx, seed=3 + variant)
    r = hz.solve(_dev(p.F), _dev(p.G), path="pointwise", **_variant_args(variant))
    _check(p, r, variant, "complex" if cplx else "real")


@pytest.mark.parametrize("variant", [1, 2, 3])
def test_row_cyclic_variants_follow_the_oracle(hz, variant):
    """Row-cyclic wavefront = the oracle's sequence: only the rounding of the
    dot products differs, so sigma and the sweep count agree closely."""
    p = make_pair(**POINTWISE_64x32)
    r = hz.solve(_dev(p.F), _dev(p.G), path="pointwise", order="row_cyclic", **_variant_args(variant))
    ref = _check(p, r, variant, "row-cyclic")
    assert rel_sigma_err(_np(r.sigma), ref["sigma"]) <= 1e-13
    assert abs(r.info["sweeps_fp64"] - ref["sweeps"]) <= 1


def test_dscale_variant_with_badly_scaled_columns(hz):
    """Columns of F and G scaled alike over six decades (sigma unchanged):
    without prescaling the D-hat variant meets b_ii far from 1 at every
    first visit."""
    p = make_pair(40, 36, 20, seed=11)
    d = np.logspace(-3, 3, 20)[np.random.default_rng(2).permutation(20)]
    F, G = p.F * d[None, :], p.G * d[None, :]
    r = hz.solve(_dev(F), _dev(G), path="pointwise", variant=2)
    ref = oracle.gsvd(F, G, variant=2, extended=True)
    assert r.status == 0 and rel_sigma_err(_np(r.sigma), ref["sigma"]) <= 1e-12


def test_variants_in_a_batch_equal_single_solves(hz):
    pairs = [make_pair(30, 25, 12, seed=40 + k, cplx=bool(k & 1)) for k in range(6)]
    s = hz.Solver(path="pointwise", variant=3)
    rb = s.solve_batched([(_dev(p.F), _dev(p.G)) for p in pairs])
    for p, b in zip(pairs, rb):
        a = s.solve(_dev(p.F), _dev(p.G))
        assert torch.equal(a.sigma, b.sigma) and torch.equal(a.Z, b.Z)
    s.close()


@pytest.mark.parametrize("variant", [1, 2, 3])
@pytest.mark.parametrize("cplx", [False, True])
def test_blocked_variants_match_the_oracle(hz, variant, cplx):
    """The variants in the FP64 pivot step of the blocked path (the inner
    level's dot products by App. A, the D-hat rescaling instead of the inner
    prescale) give the oracle's GSVD in the same variant."""
    p = make_pair(120, 100 if not cplx else 90, 72, lo=1e-3, hi=1e3, cond=1e2, cplx=cplx, seed=60 + variant)
    r = hz.solve(_dev(p.F), _dev(p.G), path="blocked", block_w=8 if not cplx else 4, shorten=0, variant=variant)
    assert r.info["path"] == 2
    _check(p, r, variant, "blocked %s" % ("complex" if cplx else "real"))


def test_variants_refused_where_the_pivot_step_has_none(hz):
    """Pair width 64 (w = 32, real) runs the one-CTA pivot step, which has
    only variant 0: a variant there is refused before any launch."""
    p = make_pair(300, 300, 128, seed=5)
    r = hz.solve(_dev(p.F), _dev(p.G), path="blocked", block_w=32, variant=1)
    assert r.status == hz.EINVAL
