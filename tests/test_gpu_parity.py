"""GPU parity: the CUDA library (through the C ABI) against the oracle.

Tolerance (floating point, sigma): every valid FP64 rounding sequence moves
the computed generalized singular values by about eps times their condition,
so the GPU is compared with the extended-precision oracle on the same rounded
inputs and must satisfy

    err(GPU vs oracle_ext) <= max(1e-12, 4 * err(oracle_fp64 vs oracle_ext)),

which is the stated 1e-12 wherever the FP64 oracle itself is within 2.5e-13.
The raw GPU-vs-FP64-oracle error is reported with every case.  Residuals:
||FZ - U Sigma_F|| / ||F|| <= 1e-13 n, ||GZ - V Sigma_G|| / ||G|| <= 1e-13 n,
orthogonality of U and V, Sigma_F^2 + Sigma_G^2 = 1, Sigma sorted.
Integer outputs (status, convergence) must match exactly where defined.
"""
import numpy as np
import pytest

import os
import sys

import oracle
from paper_1909_00101_gb300.inputs import make_pair, POINTWISE_64x32
from gsvd_checks import invariants, rel_sigma_err

sys.path.insert(0, os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden"))
import oracle_cases  # noqa: E402

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


_big_pairs = {}


def _big(recipe):
    """A full-size pair, drawn once per test session (drawing it takes seconds)."""
    key = tuple(sorted(recipe.items()))
    if key not in _big_pairs:
        _big_pairs[key] = make_pair(**recipe)
    return _big_pairs[key]


def _dev(a):
    return torch.from_numpy(np.asfortranarray(a)).cuda()


def _np(t):
    return t.cpu().numpy()


def stored_or_live(p_F, p_G, case=None):
    """(sigma_fp64, sigma_ext) of the oracle: the stored values of a case
    (after the check that the pair is the stored one; without a case name,
    a stored record of the same bytes if there is one), else computed now."""
    if case is None:
        from paper_1909_00101_gb300.inputs import sha256
        case = oracle_cases.by_sha256().get(sha256(p_F, p_G))
    if case is not None:
        rec = oracle_cases.load_checked(case, p_F, p_G)
        assert rec["status_fp64"] == 0 and rec["status_ext"] == 0
        return rec["sigma_fp64"], rec["sigma_ext"]
    ref = oracle.gsvd(p_F, p_G)
    refx = oracle.gsvd(p_F, p_G, extended=True)
    assert ref["status"] == 0 and refx["status"] == 0
    return ref["sigma"], refx["sigma"]


def sigma_vs_oracle(sig, p_F, p_G, case=None, label=""):
    """The R14 rule: err(GPU vs oracle_ext) <= max(1e-12, 4 err(oracle_fp64
    vs oracle_ext)); returns (err_ext, tol, err_fp64)."""
    s64, sx = stored_or_live(p_F, p_G, case)
    tol = max(1e-12, 4.0 * rel_sigma_err(s64, sx))
    err_x = rel_sigma_err(sig, sx)
    err_64 = rel_sigma_err(sig, s64)
    print("%s sigma err vs oracle_ext %.2e (tol %.2e), vs oracle_fp64 %.2e" % (label, err_x, tol, err_64))
    assert err_x <= tol, (label, err_x, tol)
    return err_x, tol, err_64


def check(p_F, p_G, r, *, n_res=1e-13, label="", case=None):
    s64, sx = stored_or_live(p_F, p_G, case)
    ref = {"sigma": s64}
    refx = {"sigma": sx}
    sig = _np(r.sigma)
    floor = rel_sigma_err(ref["sigma"], refx["sigma"])
    tol = max(1e-12, 4.0 * floor)
    err_x = rel_sigma_err(sig, refx["sigma"])
    err_64 = rel_sigma_err(sig, ref["sigma"])
    print("%s sigma err vs oracle_ext %.2e (tol %.2e), vs oracle_fp64 %.2e, info %s"
          % (label, err_x, tol, err_64, r.info))
    assert r.status == 0, r.info
    assert err_x <= tol, (err_x, tol)
    n = p_F.shape[1]
    inv = invariants(p_F, p_G, _np(r.U), _np(r.V), _np(r.Z), _np(r.sigma_f), _np(r.sigma_g), sig)
    assert inv["FZ"] <= n_res * n and inv["GZ"] <= n_res * n, inv
    assert inv["UU"] <= 1e-12 * n and inv["VV"] <= 1e-12 * n, inv
    assert inv["scale"] <= 8 * 2.0 ** -53 and inv["sorted"], inv
    assert rel_sigma_err(_np(r.sigma_f) / _np(r.sigma_g), sig) <= 8 * 2.0 ** -53
    return err_x


# ------------------------------------------------------------ pointwise ----

@pytest.mark.parametrize("order", ["round_robin", "row_cyclic"])
def test_pointwise_64x32_real(hz, order):
    p = make_pair(**POINTWISE_64x32)
    r = hz.solve(_dev(p.F), _dev(p.G), path="pointwise", order=order)
    check(p.F, p.G, r, label="pointwise-" + order)


def test_pointwise_row_cyclic_follows_the_oracle(hz):
    """Row-cyclic wavefront order = the oracle's sequence of transformations:
    only the rounding of the dot products differs."""
    p = make_pair(**POINTWISE_64x32)
    r = hz.solve(_dev(p.F), _dev(p.G), path="pointwise", order="row_cyclic")
    ref = oracle.gsvd(p.F, p.G)
    assert rel_sigma_err(_np(r.sigma), ref["sigma"]) <= 1e-13
    assert abs(r.info["sweeps_fp64"] - ref["sweeps"]) <= 1


@pytest.mark.parametrize("shape", [(40, 33, 33), (20, 17, 7), (9, 8, 2), (5, 3, 1)])
def test_pointwise_ragged_and_tiny(hz, shape):
    mf, mg, n = shape
    p = make_pair(mf, mg, n, seed=n)
    r = hz.solve(_dev(p.F), _dev(p.G), path="pointwise")
    check(p.F, p.G, r, label="pointwise%s" % (shape,))


def test_pointwise_complex(hz):
    p = make_pair(48, 40, 24, cplx=True, seed=3)
    r = hz.solve(_dev(p.F), _dev(p.G), path="pointwise")
    check(p.F, p.G, r, label="pointwise-complex")


# -------------------------------------------------------------- blocked ----

@pytest.mark.parametrize("shorten", [0, 2])
@pytest.mark.parametrize("w,shape", [(8, (160, 130, 96)), (16, (200, 180, 100)), (32, (300, 257, 150)),
                                     (8, (70, 65, 61))])
def test_blocked_real_fp64(hz, w, shape, shorten):
    mf, mg, n = shape
    p = make_pair(mf, mg, n, lo=1e-3, hi=1e3, cond=1e2, seed=w + n)
    r = hz.solve(_dev(p.F), _dev(p.G), path="blocked", block_w=w, shorten=shorten)
    assert r.info["path"] == 2 and r.info["block_w"] == w
    assert r.info["shortened"] == (1 if shorten else 0), r.info
    check(p.F, p.G, r, label="blocked w=%d %s shorten=%d" % (w, shape, shorten))


@pytest.mark.parametrize("cplx,w", [(False, 8), (False, 16), (True, 4), (True, 8)])
def test_blocked_apply_on_tcgen05(hz, cplx, w):
    """fp64_gemm = 2: the block apply of the FP64 sweeps issued as
    tcgen05.mma with the level sums in tensor memory (real-view widths 16 and
    32, 128-row tiles), against the oracle, and bitwise repeatable."""
    shape = (200, 180, 100) if not cplx else (120, 90, 72)
    p = make_pair(*shape, lo=1e-3, hi=1e3, cond=1e2, cplx=cplx, seed=116 if not cplx else w)
    r = hz.solve(_dev(p.F), _dev(p.G), path="blocked", block_w=w, shorten=0, fp64_gemm=2)
    check(p.F, p.G, r, label="tcgen05 apply cplx=%s w=%d" % (cplx, w))
    q = hz.solve(_dev(p.F), _dev(p.G), path="blocked", block_w=w, shorten=0, fp64_gemm=2)
    for a, b in ((r.sigma, q.sigma), (r.Z, q.Z), (r.U, q.U)):
        assert torch.equal(a, b)


@pytest.mark.parametrize("w", [4, 8, 16])
def test_blocked_complex_fp64(hz, w):
    p = make_pair(120, 90, 72, lo=1e-3, hi=1e3, cond=1e2, cplx=True, seed=w)
    r = hz.solve(_dev(p.F), _dev(p.G), path="blocked", block_w=w)
    check(p.F, p.G, r, label="blocked-complex w=%d" % w)


# QR shortening (Sec. 2): the sweeps run on the n x n triangular factors

@pytest.mark.parametrize("shape", [(512, 400, 160), (333, 1000, 97), (2000, 150, 129)])
def test_shortened_matches_oracle(hz, shape):
    """Tall pairs, ragged n (not a multiple of the 32-column Cholesky and
    triangular-solve blocks nor of the 64 x 64 GEMM tiles); default shorten."""
    mf, mg, n = shape
    p = make_pair(mf, mg, n, lo=1e-3, hi=1e3, cond=1e2, seed=n)
    r = hz.solve(_dev(p.F), _dev(p.G), path="blocked", block_w=8)
    assert r.info["shortened"] == 1 and r.info["shorten_skipped"] == 0, r.info
    check(p.F, p.G, r, label="shortened %s" % (shape,))


def test_shortened_mixed(hz):
    p = make_pair(700, 600, 192, lo=1e-4, hi=1e4, cond=1e3, seed=31)
    r = hz.solve(_dev(p.F), _dev(p.G), path="blocked", block_w=16, precision="mixed", inner_max_sweeps=1,
                 max_sweeps=60, fp32_max_sweeps=60)
    assert r.info["shortened"] == 1 and r.info["sweeps_fp32"] >= 1, r.info
    check(p.F, p.G, r, label="shortened mixed")


def test_shortened_equals_unshortened_within_tolerance(hz):
    """Both orders of work give the same GSVD to the FP64 tolerance; the
    right vectors Z agree column by column up to sign."""
    p = make_pair(600, 500, 128, lo=1e-2, hi=1e2, cond=1e2, seed=8)
    a = hz.solve(_dev(p.F), _dev(p.G), path="blocked", block_w=16, shorten=0)
    b = hz.solve(_dev(p.F), _dev(p.G), path="blocked", block_w=16, shorten=2)
    assert a.info["shortened"] == 0 and b.info["shortened"] == 1
    assert rel_sigma_err(_np(b.sigma), _np(a.sigma)) <= 1e-12
    za, zb = _np(a.Z), _np(b.Z)
    sgn = np.sign(np.sum(za * zb, axis=0))
    assert np.max(np.abs(za - zb * sgn[None, :])) / np.max(np.abs(za)) <= 1e-9


def test_shorten_skipped_on_singular_gram(hz):
    """A zero column of G makes G^T G singular: the first Cholesky meets an
    exact zero pivot, the solve falls back to the unshortened sweeps with F
    and G untouched, and those report G rank deficient."""
    p = make_pair(400, 300, 96, seed=41)
    G = p.G.copy(order="F")
    G[:, 5] = 0.0
    r = hz.solve(_dev(p.F), _dev(G), path="blocked", block_w=8, shorten=2)
    assert r.info["shortened"] == 0 and r.info["shorten_skipped"] == 1, r.info
    assert r.status == hz.ENOTPD


def test_shortened_bitwise_repeatable(hz):
    p = make_pair(500, 450, 100, seed=9)
    a = hz.solve(_dev(p.F), _dev(p.G), path="blocked", block_w=8, shorten=2)
    b = hz.solve(_dev(p.F), _dev(p.G), path="blocked", block_w=8, shorten=2)
    for x, y in ((a.U, b.U), (a.V, b.V), (a.Z, b.Z), (a.sigma, b.sigma)):
        assert torch.equal(x, y)


def test_blocked_bo_inner_one_sweep(hz):
    p = make_pair(150, 140, 96, seed=12)
    r = hz.solve(_dev(p.F), _dev(p.G), path="blocked", block_w=16, inner_max_sweeps=1)
    check(p.F, p.G, r, label="blocked BO")


def test_blocked_criterion_c2(hz):
    p = make_pair(150, 140, 96, seed=13)
    r = hz.solve(_dev(p.F), _dev(p.G), path="blocked", block_w=16, criterion=2)
    check(p.F, p.G, r, label="blocked C2")


@pytest.mark.parametrize("stop", [0, 50])
@pytest.mark.parametrize("cplx", [False, True])
def test_mixed_precision(hz, cplx, stop):
    """stop: FP32 sweeps to their own convergence (0) or handed over to the
    FP64 sweeps below 5 % big transformations (50, the default)."""
    p = make_pair(200, 160, 128, lo=1e-3, hi=1e3, cond=1e2, cplx=cplx, seed=21)
    r = hz.solve(_dev(p.F), _dev(p.G), path="blocked", block_w=16 if not cplx else 8, precision="mixed",
                 fp32_stop_permille=stop)
    assert r.info["sweeps_fp32"] >= 1
    check(p.F, p.G, r, label="mixed cplx=%s stop=%d" % (cplx, stop))


@pytest.mark.parametrize("cplx", [False, True])
@pytest.mark.parametrize("fp32_params", [0, 1])
def test_mixed_fp32_parameters(hz, cplx, fp32_params):
    """FP32 bulk sweeps with the pivot-pair step in FP32 (1, default) or FP64
    (0); the FP64 sweeps that follow bring the result to the FP64 tolerance
    all the same."""
    p = make_pair(200, 160, 128, lo=1e-3, hi=1e3, cond=1e2, cplx=cplx, seed=22)
    r = hz.solve(_dev(p.F), _dev(p.G), path="blocked", block_w=16 if not cplx else 8, precision="mixed",
                 fp32_params=fp32_params, shorten=0)
    assert r.info["sweeps_fp32"] >= 1
    check(p.F, p.G, r, label="mixed fp32_params=%d cplx=%s" % (fp32_params, cplx))


# ------------------------------------------------------- right vectors ----

@pytest.mark.parametrize("kw,shape", [(dict(path="pointwise"), (64, 48, 32)),
                                      (dict(path="blocked", block_w=8, shorten=0), (150, 130, 96)),
                                      (dict(path="blocked", block_w=8), (400, 300, 96)),
                                      (dict(path="blocked", block_w=16, precision="mixed"), (300, 260, 128))])
def test_right_vectors(hz, kw, shape):
    """X = Z^-1 (Sec. 1): X Z = I to working accuracy relative to ||X|| ||Z||,
    and X equals the inverse of the returned Z."""
    mf, mg, n = shape
    p = make_pair(mf, mg, n, lo=1e-3, hi=1e3, cond=1e2, seed=n + 3)
    r = hz.solve(_dev(p.F), _dev(p.G), right_vectors=True, **kw)
    assert r.status == 0, r.info
    X, Z = _np(r.X), _np(r.Z)
    eye = np.eye(n)
    err = np.max(np.abs(X @ Z - eye)) / (np.linalg.norm(X, 2) * np.linalg.norm(Z, 2))
    assert err <= 64 * n * 2.0 ** -53, err
    Zi = np.linalg.inv(Z)
    assert np.max(np.abs(X - Zi)) / np.max(np.abs(Zi)) <= 1e-9
    check(p.F, p.G, r, label="right vectors %s" % (kw,))


@pytest.mark.parametrize("kw", [dict(path="pointwise"), dict(path="blocked", block_w=8),
                                dict(path="blocked", block_w=8, precision="mixed")])
def test_right_vectors_complex(hz, kw):
    """X = Z^-1 for complex pairs: X = Sigma_F U^* F + Sigma_G V^* G."""
    n = 40 if kw["path"] == "pointwise" else 72
    p = make_pair(2 * n, n + 10, n, lo=1e-3, hi=1e3, cond=1e2, cplx=True, seed=n + 9)
    r = hz.solve(_dev(p.F), _dev(p.G), right_vectors=True, **kw)
    assert r.status == 0, r.info
    X, Z = _np(r.X), _np(r.Z)
    err = np.max(np.abs(X @ Z - np.eye(n))) / (np.linalg.norm(X, 2) * np.linalg.norm(Z, 2))
    assert err <= 64 * n * 2.0 ** -53, err
    Zi = np.linalg.inv(Z)
    assert np.max(np.abs(X - Zi)) / np.max(np.abs(Zi)) <= 1e-9
    check(p.F, p.G, r, label="complex right vectors %s" % (kw,))


def test_right_vectors_not_in_batched_calls(hz):
    """Batched calls reject a problem that asks for X (per-problem status)."""
    import ctypes
    p = make_pair(100, 90, 72, seed=6)
    F, G = _dev(p.F), _dev(p.G)
    Z = torch.empty((72, 72), dtype=torch.float64, device="cuda").t()
    X = torch.empty((72, 72), dtype=torch.float64, device="cuda").t()
    v = [torch.empty(72, dtype=torch.float64, device="cuda") for _ in range(3)]
    prob = hz._problem(F, G, Z, v[0], v[1], v[2], True)
    prob.X, prob.ldx = X.data_ptr(), 72
    infos = (hz.Info * 1)()
    with hz.Solver() as s:
        torch.cuda.synchronize()
        st = s._lib.gsvd_solve_batched(s._h, ctypes.byref(prob), 1, infos)
    assert st == hz.EINVAL and infos[0].status == hz.EINVAL


def test_right_vectors_host_path(hz):
    p = make_pair(100, 90, 72, seed=6)
    d = hz.solve(_dev(p.F), _dev(p.G), path="blocked", block_w=8, right_vectors=True)
    h = hz.solve(p.F.copy(order="F"), p.G.copy(order="F"), path="blocked", block_w=8, right_vectors=True)
    assert np.array_equal(_np(d.X), h.X)


# ------------------------------------------------------------ autotune ----

def test_autotuned_width_is_used_by_later_solves(hz):
    p = make_pair(600, 500, 256, seed=17)
    with hz.Solver(path="auto") as s:
        w = s.autotune(600, 500, 256)
        assert w in (8, 16, 32)
        r = s.solve(_dev(p.F), _dev(p.G))
        assert r.info["block_w"] == w and r.info["path"] == 2
    check(p.F, p.G, r, label="autotuned w=%d" % w)
    with hz.Solver(path="auto") as s:
        assert s.autotune(300, 260, 128, cplx=True) in (4, 8, 16)


# ------------------------------------------------------ stripe driver ----

def test_stripe_driver_with_the_library_pair_solver(hz):
    """Sec. 4 driver on one process (two stripes, no exchange partner) with the
    library solving the pair: the same GSVD as the oracle."""
    from paper_1909_00101_gb300 import stripes as S
    p = make_pair(40, 36, 16, lo=1e-2, hi=1e2, cond=10.0, seed=7)
    w = 8
    Fl, Gl, Zl = S.prescale_stripes(p.F, p.G, 0, 1, w, 16)
    with hz.Solver(path="blocked", block_w=4) as s:
        res = S.run(Fl, Gl, Zl, rank=0, world=1, dist=None, solve_pair=S.library_pair_solver(s))
    assert res.status == 0, res
    fin = S.finalize(res.F, res.G, res.Z)
    ref = oracle.gsvd(p.F, p.G)
    assert rel_sigma_err(np.sort(fin["sigma"])[::-1], ref["sigma"]) <= 1e-12


# ------------------------------------------------------- reproducibility ----

@pytest.mark.parametrize("kw", [dict(path="pointwise"), dict(path="blocked", block_w=16),
                                dict(path="blocked", block_w=16, precision="mixed")])
def test_bitwise_repeatable(hz, kw):
    p = make_pair(130, 120, 64, seed=5)
    a = hz.solve(_dev(p.F), _dev(p.G), **kw)
    b = hz.solve(_dev(p.F), _dev(p.G), **kw)
    for x, y in ((a.U, b.U), (a.V, b.V), (a.Z, b.Z), (a.sigma, b.sigma), (a.sigma_f, b.sigma_f)):
        assert torch.equal(x, y)


def test_host_pointer_path_equals_device_path(hz):
    p = make_pair(100, 90, 72, seed=6)
    d = hz.solve(_dev(p.F), _dev(p.G), path="blocked", block_w=8)
    h = hz.solve(p.F.copy(order="F"), p.G.copy(order="F"), path="blocked", block_w=8)
    assert np.array_equal(_np(d.sigma), h.sigma) and np.array_equal(_np(d.Z), h.Z)
    assert np.array_equal(_np(d.U), h.U)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_batched_blocked_problems_vs_oracle(hz, precision):
    """Problems of the 512-pair batch's distribution up to n = 256 (blocked
    path, shortened where tall) in one batched call, each compared with the
    oracle's sigma of that pair (stored) under the R14 rule; pointwise-size
    problems in the same call against the oracle computed now."""
    cases = ["batch_real_%d" % k for k in range(len(oracle_cases.BATCH_SHAPES))]
    pairs = [make_pair(**oracle_cases.CASES[c]) for c in cases]
    small = [make_pair(mf, mg, n, lo=1e-3, hi=1e3, cond=1e2, seed=1100 + k)
             for k, (mf, mg, n) in enumerate([(40, 35, 30), (64, 48, 32), (20, 20, 16)])]
    with hz.Solver(precision=precision) as s:
        res = s.solve_batched([(_dev(p.F), _dev(p.G)) for p in pairs + small])
    for c, p, r in zip(cases + [None] * len(small), pairs + small, res):
        check(p.F, p.G, r, label="batched %s n=%d" % (precision, p.F.shape[1]), case=c)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_batched_failures_stay_with_their_problem(hz, precision):
    """In one batched call the blocked problems advance together; a problem
    with a non-finite entry (EINVAL, untouched) and one with a zero column of
    G (ENOTPD) fail alone, and every other problem gets the bits of its
    single solve (shortening off: the batched path does not shorten)."""
    shapes = [(150, 130, 96), (200, 150, 120), (90, 80, 70), (130, 140, 100), (300, 260, 128)]
    pairs = [make_pair(*sh, lo=1e-3, hi=1e3, cond=1e2, seed=700 + k) for k, sh in enumerate(shapes)]
    F1 = pairs[1].F.copy(order="F")
    F1[7, 3] = np.nan
    G3 = pairs[3].G.copy(order="F")
    G3[:, 11] = 0.0
    inputs = [(p.F, p.G) for p in pairs]
    inputs[1] = (F1, pairs[1].G)
    inputs[3] = (pairs[3].F, G3)
    with hz.Solver(precision=precision, shorten=0) as s:
        res = s.solve_batched([(_dev(F), _dev(G)) for F, G in inputs])
        assert res[1].info["status"] == hz.EINVAL and torch.equal(res[1].U.cpu().isnan().any(), torch.tensor(True))
        assert res[3].info["status"] == hz.ENOTPD
        for k in (0, 2, 4):
            one = s.solve(_dev(inputs[k][0]), _dev(inputs[k][1]))
            assert res[k].info["status"] == 0 and one.status == 0, (res[k].info, one.info)
            assert res[k].info["sweeps_fp64"] == one.info["sweeps_fp64"]
            for a, b in ((res[k].sigma, one.sigma), (res[k].Z, one.Z), (res[k].U, one.U), (res[k].V, one.V)):
                assert torch.equal(a, b)
            check(pairs[k].F, pairs[k].G, res[k], label="batched %s n=%d" % (precision, shapes[k][2]))


def test_batched_equals_single(hz):
    shapes = [(40, 35, 30), (64, 48, 32), (20, 20, 16), (90, 80, 70), (33, 33, 33)]
    pairs = [make_pair(*s, seed=100 + k) for k, s in enumerate(shapes)]
    with hz.Solver() as s:
        batch = s.solve_batched([(_dev(p.F), _dev(p.G)) for p in pairs])
        for p, rb in zip(pairs, batch):
            r1 = s.solve(_dev(p.F), _dev(p.G))
            assert rb.info["status"] == 0
            assert torch.equal(rb.sigma, r1.sigma) and torch.equal(rb.Z, r1.Z)
            check(p.F, p.G, rb, label="batched n=%d" % p.F.shape[1])


def test_serving_results_equal_alone_and_in_mix(hz):
    shapes = [(64, 48, 32), (200, 150, 100), (90, 80, 70), (130, 120, 64), (300, 280, 160), (40, 40, 40)]
    pairs = [make_pair(*s, seed=200 + k, cplx=(k % 3 == 2)) for k, s in enumerate(shapes)]
    with hz.Solver(max_inflight=4) as s:
        alone = [s.solve(_dev(p.F), _dev(p.G)) for p in pairs]
        tickets = [s.submit(_dev(p.F), _dev(p.G)) for p in pairs]
        import time
        done = {}
        t0 = time.time()
        while len(done) < len(tickets) and time.time() - t0 < 120:
            for k, (t, res) in enumerate(tickets):
                if k in done:
                    continue
                st, info = s.poll(t)
                if st != hz.EAGAIN:
                    done[k] = (st, info)
            time.sleep(0.001)
        assert len(done) == len(tickets)
        for k, (t, res) in enumerate(tickets):
            assert done[k][0] == 0, done[k]
            assert torch.equal(res.sigma, alone[k].sigma) and torch.equal(res.Z, alone[k].Z)
            res.info = done[k][1]
            check(pairs[k].F, pairs[k].G, res, label="served %s%s" % (shapes[k], " complex" if k % 3 == 2 else ""))


# ---------------------------------------------------------------- status ----

def test_timeout_stops_at_a_sweep_boundary_with_valid_outputs(hz):
    """timeout_ms: once the deadline has passed no further sweep is issued;
    the status is ETIMEOUT, the outputs are a finalised decomposition of the
    pair at that point, and the handle serves the next solve normally."""
    p = make_pair(3000, 2500, 512, lo=1e-4, hi=1e4, cond=1e3, seed=71)
    with hz.Solver(path="blocked", block_w=16, shorten=0, inner_max_sweeps=1, max_sweeps=60,
                   timeout_ms=1) as s:
        r = s.solve(_dev(p.F), _dev(p.G))
    assert r.status == hz.ETIMEOUT, r.info
    assert r.info["sweeps_fp64"] == 1, r.info
    inv = invariants(p.F, p.G, _np(r.U), _np(r.V), _np(r.Z), _np(r.sigma_f), _np(r.sigma_g), _np(r.sigma))
    assert inv["FZ"] < 1e-12 and inv["GZ"] < 1e-12 and inv["scale"] <= 8 * 2.0 ** -53, inv
    with hz.Solver(path="blocked", block_w=16, shorten=0, inner_max_sweeps=1, max_sweeps=60,
                   timeout_ms=600000) as s:
        r2 = s.solve(_dev(p.F), _dev(p.G))
    assert r2.status == 0 and r2.info["sweeps_fp64"] > 1, r2.info


def test_serving_workspaces_come_back_to_the_pool(hz):
    """Served requests take their workspaces from the handle's stream-ordered
    pool and give them back: after a first round of requests, further rounds
    of the same sizes reserve no more device memory."""
    import time
    shapes = [(300, 280, 160), (200, 150, 100), (600, 500, 256), (90, 80, 70)]
    pairs = [make_pair(*sh, seed=500 + k) for k, sh in enumerate(shapes)]
    dev = [(_dev(p.F), _dev(p.G)) for p in pairs]

    def round_trip(s):
        tickets = [s.submit(F, G) for F, G in dev]
        done, t0 = set(), time.time()
        while len(done) < len(tickets) and time.time() - t0 < 120:
            for k, (t, _) in enumerate(tickets):
                if k not in done and s.poll(t)[0] != hz.EAGAIN:
                    done.add(k)
            time.sleep(0.001)
        assert len(done) == len(tickets)
        torch.cuda.synchronize()

    with hz.Solver(max_inflight=4) as s:
        round_trip(s)
        free0 = torch.cuda.mem_get_info()[0]
        for _ in range(3):
            round_trip(s)
        free1 = torch.cuda.mem_get_info()[0]
    # (a small slack for torch's own caching allocator, which holds the
    # requests' output buffers)
    assert free1 >= free0 - (32 << 20), (free0, free1)


def test_status_nonfinite_input(hz):
    p = make_pair(40, 40, 20, seed=1)
    F = p.F.copy()
    F[3, 4] = np.nan
    r = hz.solve(_dev(F), _dev(p.G))
    assert r.status == hz.EINVAL


@pytest.mark.parametrize("path", ["pointwise", "blocked"])
def test_status_rank_deficient_G(hz, path):
    """A zero column of G: the prescale (Sec. 2, z_j = 1/||g_j||) has no
    finite value, the solve reports ENOTPD (and still writes its outputs)."""
    p = make_pair(40, 40, 20, seed=2)
    G = p.G.copy()
    G[:, 5] = 0.0
    r = hz.solve(_dev(p.F), _dev(G), path=path, block_w=4 if path == "blocked" else 0, shorten=0)
    assert r.status == hz.ENOTPD


def test_status_rank_deficient_G_at_the_first_pivot(hz):
    """Two equal columns of G meet in the first pivot pair of the row-cyclic
    order, (0, 1): after the prescale both are (1/2, 1/2, 1/2, 1/2, 0, ...),
    so b_12 = x = 1 exactly and 1 - x^2 = 0: the 2x2 transformation of
    Sec. 2.1.2 does not exist and the solve reports ENOTPD."""
    p = make_pair(40, 40, 20, seed=2)
    G = p.G.copy()
    G[:, 0] = 0.0
    G[:4, 0] = 1.0
    G[:, 1] = G[:, 0]
    r = hz.solve(_dev(p.F), _dev(G), path="pointwise", order="row_cyclic")
    assert r.status == hz.ENOTPD


@pytest.mark.parametrize("path", ["pointwise", "blocked"])
def test_status_sweep_cap(hz, path):
    p = make_pair(100, 100, 60, seed=3)
    r = hz.solve(_dev(p.F), _dev(p.G), path=path, max_sweeps=1, block_w=8 if path == "blocked" else 0)
    assert r.status == hz.ENOCONV
    assert r.info["sweeps_fp64"] == 1
    # outputs are still a valid decomposition of the pair at that point
    inv = invariants(p.F, p.G, _np(r.U), _np(r.V), _np(r.Z), _np(r.sigma_f), _np(r.sigma_g), _np(r.sigma))
    assert inv["FZ"] < 1e-12 and inv["scale"] <= 8 * 2.0 ** -53


def test_n_equal_one(hz):
    rng = np.random.default_rng(0)
    F = rng.standard_normal((5, 1))
    G = rng.standard_normal((3, 1))
    r = hz.solve(_dev(F), _dev(G))
    ref = oracle.gsvd(F, G)
    assert r.status == 0
    assert rel_sigma_err(_np(r.sigma), ref["sigma"]) <= 4e-16


# ------------------------------------------------------------- full size ----

def _full_size_checks(hz, p, r, n_sample=16, case=None):
    """Properties that hold at any size, checked on the GPU in FP64; the
    oracle's sigma of this very pair (stored, keyed by the pair's SHA-256)
    under the R14 rule; and the generated sigma within n * eps * cond(X)
    (input rounding moves the exact GSVD of the rounded pair by about
    eps * cond(X) per column)."""
    F0 = _dev(p.F)
    G0 = _dev(p.G)
    n = p.F.shape[1]
    U, V, Z, sf, sg, sig = r.U, r.V, r.Z, r.sigma_f, r.sigma_g, r.sigma
    eps = 2.0 ** -53
    assert r.status == 0, r.info
    res_f = float(torch.linalg.norm(F0 @ Z - U * sf[None, :]) / torch.linalg.norm(F0))
    res_g = float(torch.linalg.norm(G0 @ Z - V * sg[None, :]) / torch.linalg.norm(G0))
    eye = torch.eye(n, dtype=U.dtype, device=U.device)
    orth_u = float(torch.linalg.norm(U.conj().t() @ U - eye))
    orth_v = float(torch.linalg.norm(V.conj().t() @ V - eye))
    scale = float(torch.max(torch.abs(sf * sf + sg * sg - 1.0)))
    s_np = sig.cpu().numpy()
    rel = float(np.max(np.abs(s_np - p.sigma) / p.sigma))
    print("full size: res_F %.2e res_G %.2e orth_U %.2e orth_V %.2e scale %.2e sigma err %.2e sweeps %d+%d"
          % (res_f, res_g, orth_u, orth_v, scale, rel, r.info["sweeps_fp32"], r.info["sweeps_fp64"]))
    assert res_f <= 1e-13 * n and res_g <= 1e-13 * n
    assert orth_u <= 1e-12 * n and orth_v <= 1e-12 * n
    assert scale <= 8 * eps
    assert np.all(np.diff(s_np) <= 0)
    assert rel <= n * eps * p.cond_x
    if case is not None:
        sigma_vs_oracle(s_np, p.F, p.G, case, label=case)
    # per-column backward errors of the GSVD relations on sampled columns:
    # ||F z_j - sigma_F,j u_j|| / (||F|| ||z_j||) and likewise for G (a check
    # through the Grams F*F, G*G would square the conditioning, App. G)
    idx = torch.from_numpy(np.linspace(0, n - 1, n_sample).astype(np.int64)).to(Z.device)
    zs = Z[:, idx]
    zn = torch.linalg.norm(zs, dim=0)
    bf = torch.linalg.norm(F0 @ zs - U[:, idx] * sf[idx][None, :], dim=0) / (torch.linalg.norm(F0, 2) * zn)
    bg = torch.linalg.norm(G0 @ zs - V[:, idx] * sg[idx][None, :], dim=0) / (torch.linalg.norm(G0, 2) * zn)
    assert float(torch.max(bf)) <= 8 * n * eps and float(torch.max(bg)) <= 8 * n * eps


def test_full_size_real_4096x2048_mixed(hz):
    """The benchmark workload in the benchmark's configuration (w = 16, BO, mixed)."""
    from paper_1909_00101_gb300.inputs import BLOCKED_REAL_4096x2048
    p = _big(BLOCKED_REAL_4096x2048)
    r = hz.solve(_dev(p.F), _dev(p.G), path="blocked", precision="mixed", inner_max_sweeps=1, max_sweeps=60,
                 fp32_max_sweeps=60)
    _full_size_checks(hz, p, r, case="blocked_real_4096x2048")
    assert r.info["shortened"] == 1, r.info
    # the FP32 bulk sweeps converge on their own (FP32 Gram/apply are right)
    # and leave few FP64 sweeps
    assert r.info["sweeps_fp32"] < 60 and r.info["sweeps_fp64"] <= 15, r.info


def test_full_size_real_4096x2048_unshortened(hz):
    """The same workload without the QR shortening (every sweep on 4096 rows)."""
    from paper_1909_00101_gb300.inputs import BLOCKED_REAL_4096x2048
    p = _big(BLOCKED_REAL_4096x2048)
    r = hz.solve(_dev(p.F), _dev(p.G), path="blocked", precision="mixed", inner_max_sweeps=1, max_sweeps=60,
                 fp32_max_sweeps=60, shorten=0)
    _full_size_checks(hz, p, r, case="blocked_real_4096x2048")
    assert r.info["shortened"] == 0, r.info


def test_full_size_complex_3072x1024_mixed(hz):
    from paper_1909_00101_gb300.inputs import BLOCKED_CPLX_3072x1024
    p = _big(BLOCKED_CPLX_3072x1024)
    r = hz.solve(_dev(p.F), _dev(p.G), path="blocked", precision="mixed", block_w=8, inner_max_sweeps=1,
                 max_sweeps=80, fp32_max_sweeps=80)
    _full_size_checks(hz, p, r, case="blocked_cplx_3072x1024")


def test_full_size_real_4096x2048_fp64(hz):
    """The benchmark workload in plain FP64 (the other arm of the benchmark)."""
    from paper_1909_00101_gb300.inputs import BLOCKED_REAL_4096x2048
    p = _big(BLOCKED_REAL_4096x2048)
    r = hz.solve(_dev(p.F), _dev(p.G), path="blocked", precision="fp64", inner_max_sweeps=1, max_sweeps=60)
    _full_size_checks(hz, p, r, case="blocked_real_4096x2048")


def test_full_size_complex_3072x1024_fp64(hz):
    from paper_1909_00101_gb300.inputs import BLOCKED_CPLX_3072x1024
    p = _big(BLOCKED_CPLX_3072x1024)
    r = hz.solve(_dev(p.F), _dev(p.G), path="blocked", precision="fp64", block_w=8, inner_max_sweeps=1,
                 max_sweeps=80)
    _full_size_checks(hz, p, r, case="blocked_cplx_3072x1024")


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_mid_size_real_unshortened_vs_oracle(hz, precision):
    """3000 + 2500 rows, n = 512, no shortening: every sweep runs on the full
    rows, so the Gram takes several row splits per pair and the apply
    hundreds of row tiles per launch; compared with the oracle's sigma of
    this very pair (stored) under the R14 rule, with every invariant."""
    case = "mid_real_3000x2500x512"
    p = make_pair(**oracle_cases.CASES[case])
    r = hz.solve(_dev(p.F), _dev(p.G), path="blocked", block_w=16, precision=precision, shorten=0,
                 inner_max_sweeps=1, max_sweeps=60, fp32_max_sweeps=60)
    assert r.info["shortened"] == 0, r.info
    check(p.F, p.G, r, label="mid-size real %s" % precision, case=case)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_mid_size_complex_vs_oracle(hz, precision):
    case = "mid_cplx_1500x1200x256"
    p = make_pair(**oracle_cases.CASES[case])
    r = hz.solve(_dev(p.F), _dev(p.G), path="blocked", block_w=8, precision=precision, inner_max_sweeps=1,
                 max_sweeps=60, fp32_max_sweeps=60)
    check(p.F, p.G, r, label="mid-size complex %s" % precision, case=case)


def test_shortened_products_longer_than_one_exact_sum(hz):
    """m_F, m_G > 65536: the shortening's Grams F^T F and G^T G run on the
    tensor cores in K pieces of at most 65536 rows (each summed exactly and
    rounded once into C); the solve keeps the full-size tolerances against
    the generated sigma and agrees with the unshortened solve."""
    p = make_pair(70000, 66000, 128, seed=12)
    a = hz.solve(_dev(p.F), _dev(p.G), path="blocked", block_w=16)
    assert a.info["shortened"] == 1, a.info
    _full_size_checks(hz, p, a)
    b = hz.solve(_dev(p.F), _dev(p.G), path="blocked", block_w=16, shorten=0)
    assert b.status == 0 and b.info["shortened"] == 0, b.info
    assert rel_sigma_err(_np(a.sigma), _np(b.sigma)) <= 1e-12
