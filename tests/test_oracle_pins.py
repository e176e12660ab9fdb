"""Pins of the oracle against what the paper and the mathematics fix (CPU only).

Each test would fail for a plausible mistake in the oracle: a dropped term or
wrong sign in the 2x2 formulas (transformation invariants), a wrong index or
transposed operand in the column updates (residuals, known sigma), a wrong
prescaling or final scaling (closed forms, Sigma_F^2 + Sigma_G^2 = I), a wrong
sort (Appendix G order), a wrong stopping rule (status and sweep counts).
"""
import json
import math
import os

import numpy as np
import pytest
import scipy.linalg

import oracle
from paper_1909_00101_gb300.inputs import make_pair, POINTWISE_64x32
from gsvd_checks import invariants, rel_sigma_err

GOLD = os.path.join(os.path.dirname(__file__), "golden")
EPS = 2.0 ** -53


# ---------------------------------------------------------------- 2x2 pins --

def _bound(Z, M):
    # rounding of the check's own products Z^* M Z: a few eps * ||Z||^2 ||M||
    return 64 * EPS * np.linalg.norm(Z) ** 2 * np.linalg.norm(M)


def _check_real_pivot(a11, a22, a12, x):
    Z, small, st = oracle.pivot_real(a11, a22, a12, x)
    assert st == 0
    A = np.array([[a11, a12], [a12, a22]])
    B = np.array([[1.0, x], [x, 1.0]])
    ZA = Z.T @ A @ Z
    ZB = Z.T @ B @ Z
    assert abs(ZA[0, 1]) <= _bound(Z, A), (a11, a22, a12, x, ZA)
    assert np.max(np.abs(ZB - np.eye(2))) <= _bound(Z, B), (a11, a22, a12, x, ZB)
    return Z, small


def _check_cplx_pivot(a11, a22, a12, b12):
    Z, small, st = oracle.pivot_cplx(a11, a22, a12, b12)
    assert st == 0
    A = np.array([[a11, a12], [np.conj(a12), a22]])
    B = np.array([[1.0, b12], [np.conj(b12), 1.0]])
    ZA = Z.conj().T @ A @ Z
    ZB = Z.conj().T @ B @ Z
    assert abs(ZA[0, 1]) <= _bound(Z, A), (a11, a22, a12, b12, ZA)
    assert np.max(np.abs(ZB - np.eye(2))) <= _bound(Z, B), (a11, a22, a12, b12, ZB)
    # the diagonal of Z^* A Z is real and positive
    assert abs(ZA[0, 0].imag) <= _bound(Z, A) and ZA[0, 0].real > 0 and ZA[1, 1].real > 0
    return Z, small


def test_real_pivot_random_invariants():
    """Z^T A Z diagonal and Z^T B Z = I (Sec. 2.1) for random SPD pivots."""
    rng = np.random.default_rng(1)
    for _ in range(3000):
        f = rng.standard_normal((6, 2)) * np.exp(rng.uniform(-3, 3, 2))
        g = rng.standard_normal((6, 2))
        g /= np.linalg.norm(g, axis=0)
        A = f.T @ f
        B = g.T @ g
        _check_real_pivot(A[0, 0], A[1, 1], A[0, 1], B[0, 1])


def test_real_pivot_edges():
    """Signed zeros, x -> +-1, equal diagonals, and the proportional exception."""
    for x in (0.0, -0.0, 1e-300, -1e-17, 0.3, -0.3, 0.999999, -0.999999):
        for a11, a22, a12 in ((2.0, 2.0, 0.9), (1.0, 3.0, 0.0), (1.0, 3.0, -0.0),
                              (5.0, 1.0, 1e-300), (1e-8, 1e8, 1e-3), (2.0, 2.0, -0.5)):
            if a12 * a12 >= a11 * a22:
                continue
            _check_real_pivot(a11, a22, a12, x)
    # proportional A = 2B: cot(2 theta) = 0/0, the exception of Sec. 2.1.2 (reading R2)
    for x in (0.3, -0.3, 0.9, -0.9):
        Z, _ = _check_real_pivot(2.0, 2.0, 2.0 * x, x)


def test_real_sort_formula_equals_transformed_diagonal():
    """The a11'', a22'' formula of Sec. 3.5.3 equals diag(Z^T A Z)."""
    rng = np.random.default_rng(2)
    for _ in range(200):
        f = rng.standard_normal((5, 2))
        g = rng.standard_normal((5, 2))
        g /= np.linalg.norm(g, axis=0)
        A = f.T @ f
        B = g.T @ g
        Z, _, _ = oracle.pivot_real(A[0, 0], A[1, 1], A[0, 1], B[0, 1])
        a1 = Z[0, 0] ** 2 * A[0, 0] + 2 * Z[0, 0] * Z[1, 0] * A[0, 1] + Z[1, 0] ** 2 * A[1, 1]
        a2 = Z[0, 1] ** 2 * A[0, 0] + 2 * Z[1, 1] * Z[0, 1] * A[0, 1] + Z[1, 1] ** 2 * A[1, 1]
        d = np.diag(Z.T @ A @ Z)
        assert abs(a1 - d[0]) <= 1e-13 * abs(d).max() and abs(a2 - d[1]) <= 1e-13 * abs(d).max()


def test_cplx_pivot_random_invariants():
    rng = np.random.default_rng(3)
    for _ in range(3000):
        f = (rng.standard_normal((6, 2)) + 1j * rng.standard_normal((6, 2))) * np.exp(rng.uniform(-3, 3, 2))
        g = rng.standard_normal((6, 2)) + 1j * rng.standard_normal((6, 2))
        g /= np.linalg.norm(g, axis=0)
        A = f.conj().T @ f
        B = g.conj().T @ g
        _check_cplx_pivot(A[0, 0].real, A[1, 1].real, A[0, 1], B[0, 1])


def test_cplx_pivot_edges():
    """h = +-0 with v of both signs (reading R3), b12 = 0, and the v = h = 0 exception."""
    for ph in (0.0, 0.7, -2.1, math.pi):
        e = complex(math.cos(ph), math.sin(ph))
        for v in (0.2, -0.2):
            for h0 in (0.0, -0.0):
                a12 = e * complex(0.5, v)
                _check_cplx_pivot(1.5, 1.5 + h0, a12, 0.3 * e)
        # exception: arg(b) = arg(a), equal diagonal
        _check_cplx_pivot(1.5, 1.5, 0.4 * e, 0.3 * e)
    _check_cplx_pivot(1.0, 3.0, complex(0.2, -0.1), 0j)
    _check_cplx_pivot(3.0, 1.0, complex(0.0, 0.5), complex(0.0, -0.0))


def test_cplx_pivot_reduces_to_real_on_real_data():
    """A complex pivot with real entries diagonalises like the real one (same invariants)."""
    rng = np.random.default_rng(4)
    for _ in range(300):
        f = rng.standard_normal((5, 2))
        g = rng.standard_normal((5, 2))
        g /= np.linalg.norm(g, axis=0)
        A = f.T @ f
        B = g.T @ g
        Zc, _ = _check_cplx_pivot(A[0, 0], A[1, 1], complex(A[0, 1]), complex(B[0, 1]))
        assert np.max(np.abs(Zc.imag)) <= 1e-15 * np.max(np.abs(Zc))


def test_small_transformation_criteria():
    """C1/C2 (Sec. 2.5): an already diagonal pivot gives an identity-like small transform."""
    Z, small, _ = oracle.pivot_real(4.0, 1.0, 1e-300, 0.0)
    assert small and Z[0, 0] == 1.0 and Z[1, 1] == 1.0
    Z, small, _ = oracle.pivot_real(4.0, 1.0, 1.0, 0.1)
    assert not small
    Z, small, _ = oracle.pivot_cplx(4.0, 1.0, 1e-300j, 0j, criterion=2)
    assert small


# ---------------------------------------------------------- closed forms --

def test_appendix_g_worked_example():
    """Appendix G: sigma = sqrt(Lambda) with the exact Lambda printed there."""
    gold = json.load(open(os.path.join(GOLD, "appG_4x4.json")))
    F = np.array(gold["F"], dtype=float)
    G = np.array(gold["G"], dtype=float)
    exact = np.sqrt(np.array(gold["lambda_exact_sorted_ascending"]))[::-1]
    printed = np.array(gold["gsvd_printed_ascending"])[::-1]
    for ext in (False, True):
        r = oracle.gsvd(F, G, extended=ext)
        assert r["status"] == 0
        assert rel_sigma_err(r["sigma"], exact) <= 4 * EPS
        assert rel_sigma_err(r["sigma"], printed) <= 8 * EPS
        inv = invariants(F, G, r["U"], r["V"], r["Z"], r["sigma_f"], r["sigma_g"], r["sigma"])
        assert inv["FZ"] < 1e-15 and inv["GZ"] < 1e-15
        assert inv["UU"] < 1e-14 and inv["VV"] < 1e-14 and inv["scale"] < 4 * EPS and inv["sorted"]


def test_n1_closed_form():
    """n = 1 (Sec. 2): U = F/||F||, V = G/||G||, Z = 1/sqrt(||F||^2+||G||^2)."""
    rng = np.random.default_rng(5)
    F = rng.standard_normal((7, 1))
    G = rng.standard_normal((3, 1))
    r = oracle.gsvd(F, G)
    nf, ng = np.linalg.norm(F), np.linalg.norm(G)
    h = math.sqrt(nf * nf + ng * ng)
    assert r["status"] == 0
    assert np.allclose(r["U"][:, 0], F[:, 0] / nf, rtol=1e-15, atol=1e-16)
    assert np.allclose(r["V"][:, 0], G[:, 0] / ng, rtol=1e-15, atol=1e-16)
    assert abs(r["Z"][0, 0] - 1 / h) <= 4 * EPS / h
    assert abs(r["sigma_f"][0] - nf / h) <= 4 * EPS and abs(r["sigma_g"][0] - ng / h) <= 4 * EPS
    assert abs(r["sigma"][0] - nf / ng) <= 4 * EPS * nf / ng


@pytest.mark.parametrize("cplx", [False, True])
def test_n2_textbook(cplx):
    """n = 2: sigma are the singular values of R_F R_G^{-1} (QR of F and G)."""
    rng = np.random.default_rng(6)
    for _ in range(50):
        F = rng.standard_normal((5, 2))
        G = rng.standard_normal((4, 2))
        if cplx:
            F = F + 1j * rng.standard_normal((5, 2))
            G = G + 1j * rng.standard_normal((4, 2))
        rf = np.linalg.qr(F, mode="r")
        rg = np.linalg.qr(G, mode="r")
        ref = np.linalg.svd(rf @ np.linalg.inv(rg), compute_uv=False)
        r = oracle.gsvd(F, G)
        assert r["status"] == 0
        assert rel_sigma_err(r["sigma"], ref) < 1e-13


@pytest.mark.parametrize("cplx", [False, True])
def test_brute_force_tiny_pencil(cplx):
    """n <= 8, well-conditioned B: sigma^2 = eigenvalues of the pencil (F*F, G*G)."""
    rng = np.random.default_rng(7)
    for n in range(2, 9):
        mf, mg = n + 3, n + 1
        F = rng.standard_normal((mf, n))
        G = rng.standard_normal((mg, n)) + 3 * np.eye(mg, n)
        if cplx:
            F = F + 1j * rng.standard_normal((mf, n))
            G = G + 1j * rng.standard_normal((mg, n))
        A = F.conj().T @ F
        B = G.conj().T @ G
        lam = scipy.linalg.eigh(A, B, eigvals_only=True)[::-1]
        r = oracle.gsvd(F, G)
        assert r["status"] == 0
        assert rel_sigma_err(r["sigma"] ** 2, lam) < 1e-11


@pytest.mark.parametrize("cplx", [False, True])
def test_generated_known_sigma_and_invariants(cplx):
    """Generated pairs: sigma within c*eps*cond of the construction; all invariants hold."""
    for seed, (mf, mg, n) in enumerate([(64, 48, 32), (40, 40, 33), (30, 70, 17)]):
        p = make_pair(mf, mg, n, lo=1e-2, hi=1e2, cond=1e2, cplx=cplx, seed=seed)
        r = oracle.gsvd(p.F, p.G)
        assert r["status"] == 0
        assert rel_sigma_err(r["sigma"], p.sigma) < 1e4 * n * EPS * 1e2
        inv = invariants(p.F, p.G, r["U"], r["V"], r["Z"], r["sigma_f"], r["sigma_g"], r["sigma"])
        assert inv["FZ"] < 1e-13 * n and inv["GZ"] < 1e-13 * n
        assert inv["UU"] < 1e-12 and inv["VV"] < 1e-12
        assert inv["scale"] <= 8 * EPS and inv["ratio"] <= 8 * EPS and inv["sorted"]
        assert inv["F_USX"] < 1e-12 and inv["G_VSX"] < 1e-12


@pytest.mark.parametrize("kexp", [4, 8, 12, 16])
def test_gsvd_stays_accurate_where_the_gevd_fails(kexp):
    """App. G, the GSVD-versus-GEVD experiment: cond(A) = 10 fixed and
    cond(B) = 10^k through the column scaling of G.  The method works on F
    and G, not on their Grams, and is invariant under that scaling (the
    prescaling removes it), so its sigma stay within a few eps of the
    extended-precision values of the same rounded pair for every k; the
    square roots of the pencil eigenvalues of (A, B) lose about
    eps * cond(B) (the printed table shows the same contrast)."""
    from paper_1909_00101_gb300.inputs import make_graded_pair
    F, G = make_graded_pair(48, 48, 32, kexp, seed=kexp)
    B = G.T @ G
    assert 10.0 ** (kexp - 1) < np.linalg.cond(B) < 10.0 ** (kexp + 1)
    ref = oracle.gsvd(F, G, extended=True)
    r = oracle.gsvd(F, G)
    assert r["status"] == 0 and ref["status"] == 0
    assert rel_sigma_err(r["sigma"], ref["sigma"]) <= 32 * EPS
    if kexp >= 12:
        with np.errstate(invalid="ignore"):
            lam = scipy.linalg.eigh(F.T @ F, B, eigvals_only=True)[::-1]
            gevd = rel_sigma_err(np.sqrt(lam), ref["sigma"])
        assert not gevd <= 1e-9   # NaN (negative eigenvalues) or far off


def test_extended_agrees_with_double():
    """Long double and double instantiations of the same source agree near eps (c1 shape)."""
    p = make_pair(**POINTWISE_64x32)
    r = oracle.gsvd(p.F, p.G)
    re = oracle.gsvd(p.F, p.G, extended=True)
    assert r["status"] == 0 and re["status"] == 0
    assert rel_sigma_err(r["sigma"], re["sigma"]) < 1e-12
    assert rel_sigma_err(re["sigma"], p.sigma) < 1e-12


def test_real_and_complex_paths_agree_on_real_data():
    p = make_pair(20, 15, 10, seed=3)
    r = oracle.gsvd(p.F, p.G)
    c = oracle.gsvd(p.F.astype(complex), p.G.astype(complex))
    assert rel_sigma_err(c["sigma"], r["sigma"]) < 1e-13


def test_column_permutation_invariance():
    """Permuting the input columns leaves the sorted sigma unchanged."""
    p = make_pair(30, 25, 12, seed=9)
    perm = np.random.default_rng(0).permutation(12)
    a = oracle.gsvd(p.F, p.G)["sigma"]
    b = oracle.gsvd(p.F[:, perm], p.G[:, perm])["sigma"]
    assert rel_sigma_err(b, a) < 1e-13


def test_unsorted_variant_same_sigma():
    p = make_pair(30, 25, 12, seed=10)
    a = oracle.gsvd(p.F, p.G, sort=True)
    b = oracle.gsvd(p.F, p.G, sort=False)
    assert b["status"] == 0 and rel_sigma_err(b["sigma"], a["sigma"]) < 1e-12


# --------------------------------------------------------------- status --

def test_status_codes():
    F = np.ones((3, 4))
    assert oracle.gsvd(F, np.ones((5, 4)))["status"] == -1          # mF < n
    F = np.eye(4)
    G = np.eye(4)
    G[1, 1] = np.nan
    assert oracle.gsvd(F, G)["status"] == -1                          # non-finite input
    G = np.eye(4)
    G[:, 2] = 0.0
    assert oracle.gsvd(F, G)["status"] == -4                          # zero column of G
    p = make_pair(20, 20, 10, seed=1)
    r = oracle.gsvd(p.F, p.G, max_sweeps=1)
    assert r["status"] == -3 and r["sweeps"] == 1                     # sweep cap


def test_rank_deficient_G_reports_not_pd():
    """Two equal columns of G make B-hat singular: x = 1 exactly, t^2 = 0."""
    F = np.random.default_rng(0).standard_normal((6, 3))
    G = np.random.default_rng(1).standard_normal((6, 3))
    G[:, 0] = G[:, 1] = [1.0, 1.0, 1.0, 1.0, 0.0, 0.0]
    r = oracle.gsvd(F, G)
    assert r["status"] == -4


def test_nearly_parallel_G_gives_huge_sigma():
    """Numerically (not exactly) parallel columns of G: an 'infinite' generalized value."""
    F = np.random.default_rng(0).standard_normal((6, 3))
    G = np.random.default_rng(1).standard_normal((6, 3))
    G[:, 1] = 2.0 * G[:, 0]
    r = oracle.gsvd(F, G)
    assert r["status"] == -4 or r["sigma"][0] > 1e12


# ------------------------------------------- variants (Table "Variants") --

def test_enhanced_real_dot_closed_forms():
    """App. A: c = RD(a b) and d = a b - c >= 0 split every product exactly,
    so a sum that cancels to a product's rounding error comes out exact,
    where the ordinary dot product returns the rounded products' sum."""
    from fractions import Fraction
    x = 1.0 + 2.0 ** -27                      # x^2 = 1 + 2^-26 + 2^-54: rounding error +2^-54
    a, b = [x, 1.0], [x, -(1.0 + 2.0 ** -26)]
    assert oracle.dot_real(a, b) == 0.0
    assert oracle.dot_real(a, b, enhanced=True) == 2.0 ** -54
    rng = np.random.default_rng(21)
    hits = 0
    for _ in range(200):                      # either sign of the product's rounding error
        y = float(rng.uniform(1.0, 2.0))
        p = y * y
        exact = Fraction(y) * Fraction(y) - Fraction(p)
        got = oracle.dot_real([y, 1.0], [y, -p], enhanced=True)
        assert Fraction(got) == exact
        hits += exact < 0
    assert 20 < hits < 180
    # exact products (small integers): both forms give the exact sum
    ia = rng.integers(-1000, 1000, 64).astype(float)
    ib = rng.integers(-1000, 1000, 64).astype(float)
    assert oracle.dot_real(ia, ib) == oracle.dot_real(ia, ib, enhanced=True) == float(np.dot(ia, ib))
    # random vectors: within the dot product's bound of the exact value
    for m in (1, 7, 100):
        va, vb = rng.standard_normal(m), rng.standard_normal(m)
        exact = sum(Fraction(float(p)) * Fraction(float(q)) for p, q in zip(va, vb))
        scale = sum(abs(Fraction(float(p)) * Fraction(float(q))) for p, q in zip(va, vb))
        got = Fraction(oracle.dot_real(va, vb, enhanced=True))
        assert abs(got - exact) <= (m + 2) * Fraction(EPS) * scale


def test_enhanced_complex_norm_bound():
    """App. A, the simpler procedure for ||a||^2: per element
    s = (e + c_small) + c_large with e = d_re + d_im is within 1.5 u (+ O(u^2))
    of |a|^2 (one rounding of e + c_small, at most half the total, and one of
    the sum); the ordinary re^2 + im^2 needs the 2 u bound."""
    from fractions import Fraction
    rng = np.random.default_rng(22)
    u = Fraction(EPS)
    worst_ord = Fraction(0)
    for _ in range(20000):
        re, im = rng.standard_normal(2) * math.exp(rng.uniform(-5, 5))
        ex = Fraction(float(re)) ** 2 + Fraction(float(im)) ** 2
        got = Fraction(oracle.nrm2sq_cplx([complex(re, im)], enhanced=True))
        assert abs(got - ex) <= (Fraction(3, 2) * u + 4 * u * u) * ex, (re, im)
        worst_ord = max(worst_ord, abs(Fraction(oracle.nrm2sq_cplx([complex(re, im)])) - ex) / ex)
    assert worst_ord > Fraction(3, 2) * u     # the ordinary form does exceed it
    v = rng.standard_normal(50) + 1j * rng.standard_normal(50)
    ex = sum(Fraction(float(z.real)) ** 2 + Fraction(float(z.imag)) ** 2 for z in v)
    got = Fraction(oracle.nrm2sq_cplx(v, enhanced=True))
    assert abs(got - ex) <= 52 * u * ex


def _dscaled_grid(rng, cplx):
    f = rng.standard_normal((6, 2)) * np.exp(rng.uniform(-3, 3, 2))[None, :]
    g = rng.standard_normal((6, 2)) * np.exp(rng.uniform(-3, 3, 2))[None, :]
    if cplx:
        f = f + 1j * rng.standard_normal((6, 2))
        g = g + 1j * rng.standard_normal((6, 2))
    return f.conj().T @ f, g.conj().T @ g


@pytest.mark.parametrize("cplx", [False, True])
def test_dscaled_pivot_invariants(cplx):
    """D-hat variants (Sec. 2.1): with b_ii, b_jj != 1, Z-hat = D Z-hat' still
    makes Z^* B Z = I and Z^* A Z diagonal for the unscaled pivot A, B."""
    rng = np.random.default_rng(23 + cplx)
    for _ in range(500):
        A, B = _dscaled_grid(rng, cplx)
        if cplx:
            Z, _, st = oracle.pivot_cplx_dscaled(A[0, 0].real, A[1, 1].real, A[0, 1], B[0, 0].real, B[1, 1].real,
                                                 B[0, 1])
        else:
            Z, _, st = oracle.pivot_real_dscaled(A[0, 0], A[1, 1], A[0, 1], B[0, 0], B[1, 1], B[0, 1])
        assert st == 0
        ZA = Z.conj().T @ A @ Z
        ZB = Z.conj().T @ B @ Z
        assert abs(ZA[0, 1]) <= _bound(Z, A) and np.max(np.abs(ZB - np.eye(2))) <= _bound(Z, B)


def test_dscaled_pivot_reduces_to_unscaled_at_unit_diagonal():
    """b_ii = b_jj = 1 exactly: D-hat = I, and the transformation is the unscaled one bit for bit."""
    rng = np.random.default_rng(25)
    for _ in range(100):
        a11, a22 = rng.uniform(0.1, 10, 2)
        a12, x = rng.uniform(-1, 1) * math.sqrt(a11 * a22), rng.uniform(-0.9, 0.9)
        Z0, s0, _ = oracle.pivot_real(a11, a22, a12, x)
        Z1, s1, _ = oracle.pivot_real_dscaled(a11, a22, a12, 1.0, 1.0, x)
        assert np.array_equal(Z0, Z1) and s0 == s1


@pytest.mark.parametrize("cplx", [False, True])
@pytest.mark.parametrize("variant", range(1, 8))
def test_variants_known_sigma_and_invariants(cplx, variant):
    """Every variant of Table "Variants" reaches the generated sigma and the
    invariants; with the per-step sort the columns end in descending order
    (the final sort finds them presorted), which in the D-hat variants needs
    the sort to compare a_ii / b_ii, not a_ii."""
    for seed, (mf, mg, n) in enumerate([(40, 30, 24), (30, 50, 17)]):
        p = make_pair(mf, mg, n, lo=1e-2, hi=1e2, cond=1e2, cplx=cplx, seed=seed)
        r = oracle.gsvd(p.F, p.G, variant=variant)
        assert r["status"] == 0
        assert rel_sigma_err(r["sigma"], p.sigma) < 1e4 * n * EPS * 1e2
        inv = invariants(p.F, p.G, r["U"], r["V"], r["Z"], r["sigma_f"], r["sigma_g"], r["sigma"])
        assert inv["FZ"] < 1e-13 * n and inv["GZ"] < 1e-13 * n
        assert inv["UU"] < 1e-12 and inv["VV"] < 1e-12
        assert inv["scale"] <= 8 * EPS and inv["sorted"]
        assert r["presorted"], (variant, seed)
        ref = oracle.gsvd(p.F, p.G, extended=True)
        assert rel_sigma_err(r["sigma"], ref["sigma"]) < 1e-12


@pytest.mark.parametrize("variant", range(8))
def test_one_transformation_sorts_the_pair(variant):
    """n = 2, one sweep: the single transformation diagonalises the pair and
    the sort after it (Sec. 2.1) puts the larger sigma first.  Columns of F
    and G scaled alike (sigma unchanged, b_jj far from 1) and sigma within a
    factor 1.2 make a sort on the wrong diagonal show."""
    rng = np.random.default_rng(33)
    for t in range(100):
        p = make_pair(5, 4, 2, lo=1.0, hi=1.2, cond=3.0, seed=100 + t)
        d = np.exp(rng.uniform(-4, 4, 2))
        r = oracle.gsvd(p.F * d[None, :], p.G * d[None, :], variant=variant, max_sweeps=1)
        assert r["sweeps"] == 1 and r["presorted"], (variant, t)


@pytest.mark.parametrize("variant", range(8))
def test_variants_appendix_g(variant):
    """Appendix G's pair (cond(G) = 4e10) in every variant: sigma within 4 eps."""
    gold = json.load(open(os.path.join(GOLD, "appG_4x4.json")))
    F = np.array(gold["F"], dtype=float)
    G = np.array(gold["G"], dtype=float)
    exact = np.sqrt(np.array(gold["lambda_exact_sorted_ascending"]))[::-1]
    r = oracle.gsvd(F, G, variant=variant)
    assert r["status"] == 0 and rel_sigma_err(r["sigma"], exact) <= 4 * EPS
