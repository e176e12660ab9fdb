"""The oracle pins have teeth: a plausible mistake planted in a copy of the
oracle (on the CPU only) makes at least one pin fail.

Each mutation is a small edit of hz_oracle.c (a flipped sign, a dropped
term, a swapped index or operand, two statements in the wrong order); the
mutated copy is compiled into a temporary library and run through a quick
subset of the pins.
"""
import json
import os
import shutil

import numpy as np
import pytest

import oracle
from paper_1909_00101_gb300.inputs import make_pair
from gsvd_checks import invariants, rel_sigma_err

SRC = os.path.join(os.path.dirname(oracle.__file__), "hz_oracle.c")
GOLD = os.path.join(os.path.dirname(__file__), "golden", "appG_4x4.json")

MUTATIONS = [
    # (name, original text, mutated text)
    ("xi_sign", "real_t xi = x / (sqrt(1 + x) + sqrt(1 - x));", "real_t xi = x / (sqrt(1 + x) - sqrt(1 - x));"),
    ("eta_dropped", "real_t cphi = c + xi * (s - eta * c);", "real_t cphi = c + xi * (s - c);"),
    ("cot_sign", "real_t num = t * (a22 - a11);", "real_t num = t * (a11 - a22);"),
    ("cos_no_sqrt", "*c = 1 / sqrt(1 + tn * tn);", "*c = 1 / (1 + tn * tn);"),
    ("z21_sign", "z[2] = -spsi / t;", "z[2] = spsi / t;"),
    ("apply_transposed", "Y[i * m + r] = yi * z[0] + yj * z[2];", "Y[i * m + r] = yi * z[0] + yj * z[1];"),
    ("prescale_sqrt", "real_t zj = 1 / sqrt(s);\n        for (int64_t r = 0; r < mf; ++r) f[j * mf + r] *= zj;\n        for (int64_t r = 0; r < mg; ++r) g[j * mg + r] *= zj;\n        z[j * n + j] = zj;\n    }\n\n    const real_t tol = HZO_EPS * sqrt((real_t)n); /* eps * sqrt(n), R5, R6 */",
     "real_t zj = 1 / sqrt(sqrt(s));\n        for (int64_t r = 0; r < mf; ++r) f[j * mf + r] *= zj;\n        for (int64_t r = 0; r < mg; ++r) g[j * mg + r] *= zj;\n        z[j * n + j] = zj;\n    }\n\n    const real_t tol = HZO_EPS * sqrt((real_t)n); /* eps * sqrt(n), R5, R6 */"),
    ("final_theta", "real_t th = 1 / sqrt(nf[j] * nf[j] + ng[j] * ng[j]);\n        for (int64_t r = 0; r < mf; ++r) F[k * ldf + r] = (double)(f[j * mf + r] / nf[j]);",
     "real_t th = 1 / (nf[j] * nf[j] + ng[j] * ng[j]);\n        for (int64_t r = 0; r < mf; ++r) F[k * ldf + r] = (double)(f[j * mf + r] / nf[j]);"),
    ("sort_order", "while (b >= 0 && nf[perm[b]] / ng[perm[b]] < key) {", "while (b >= 0 && nf[perm[b]] / ng[perm[b]] > key) {"),
    ("cplx_conj_missing", "for (int64_t r = 0; r < m; ++r) s += conj(a[r]) * b[r];", "for (int64_t r = 0; r < m; ++r) s += a[r] * b[r];"),
    ("cplx_psi_sign", "real_t cpsi = r2 * sqrt(1 - x * s2 + t * cg * c2);", "real_t cpsi = r2 * sqrt(1 + x * s2 + t * cg * c2);"),
    ("cplx_tau", "real_t tau = sgn1(h);", "real_t tau = 1;"),
    # variants (Table "Variants"): App. A dot products and the D-hat rescaling
    ("enh_d_sign", "sd += fma(a[r], b[r], -c);", "sd -= fma(a[r], b[r], -c);"),
    ("enh_cplx_e_dropped", "real_t e = fma(re, re, -cr) + fma(im, im, -ci);", "real_t e = 0 * fma(re, re, -cr);"),
    ("dscale_mul", "*aii = *aii / bii;", "*aii = *aii * bii;"),
    ("dscale_x_index", "*aij *= *d1;\n        *x *= *d1;", "*aij *= *d1;\n        *x *= *d2;"),
    ("drows_swapped", "z[2] *= d2;\n    z[3] *= d2;\n}\n\nstatic void drows_c", "z[2] *= d1;\n    z[3] *= d2;\n}\n\nstatic void drows_c"),
    ("sort_with_dscaled_z",
     "real_t a1 = zh[0] * zh[0] * aii + 2 * zh[0] * zh[2] * aij + zh[2] * zh[2] * ajj;\n"
     "                real_t a2 = zh[1] * zh[1] * aii + 2 * zh[3] * zh[1] * aij + zh[3] * zh[3] * ajj;\n"
     "                drows_r(zh, d1, d2);",
     "drows_r(zh, d1, d2);\n"
     "                real_t a1 = zh[0] * zh[0] * aii + 2 * zh[0] * zh[2] * aij + zh[2] * zh[2] * ajj;\n"
     "                real_t a2 = zh[1] * zh[1] * aii + 2 * zh[3] * zh[1] * aij + zh[3] * zh[3] * ajj;"),
]


def _pins_pass(lib) -> bool:
    """A quick subset of the pins; False as soon as one fails."""
    rng = np.random.default_rng(11)
    eps = 2.0 ** -53
    for _ in range(200):
        f = rng.standard_normal((6, 2))
        g = rng.standard_normal((6, 2))
        g /= np.linalg.norm(g, axis=0)
        A, B = f.T @ f, g.T @ g
        Z, _, st = oracle.pivot_real(A[0, 0], A[1, 1], A[0, 1], B[0, 1], lib=lib)
        bound = 64 * eps * np.linalg.norm(Z) ** 2
        if st != 0 or abs((Z.T @ A @ Z)[0, 1]) > bound * np.linalg.norm(A) or \
                np.max(np.abs(Z.T @ B @ Z - np.eye(2))) > bound * np.linalg.norm(B):
            return False
        fc = f + 1j * rng.standard_normal((6, 2))
        gc = g + 1j * rng.standard_normal((6, 2))
        gc /= np.linalg.norm(gc, axis=0)
        A, B = fc.conj().T @ fc, gc.conj().T @ gc
        Z, _, st = oracle.pivot_cplx(A[0, 0].real, A[1, 1].real, A[0, 1], B[0, 1], lib=lib)
        bound = 64 * eps * np.linalg.norm(Z) ** 2
        if st != 0 or abs((Z.conj().T @ A @ Z)[0, 1]) > bound * np.linalg.norm(A) or \
                np.max(np.abs(Z.conj().T @ B @ Z - np.eye(2))) > bound * np.linalg.norm(B):
            return False
    gold = json.load(open(GOLD))
    F = np.array(gold["F"], dtype=float)
    G = np.array(gold["G"], dtype=float)
    exact = np.sqrt(np.array(gold["lambda_exact_sorted_ascending"]))[::-1]
    r = oracle.gsvd(F, G, lib=lib)
    if r["status"] != 0 or rel_sigma_err(r["sigma"], exact) > 4 * eps:
        return False
    for cplx in (False, True):
        p = make_pair(24, 20, 12, cplx=cplx, seed=5)
        for variant in (0, 3):
            r = oracle.gsvd(p.F, p.G, variant=variant, lib=lib)
            if r["status"] != 0 or rel_sigma_err(r["sigma"], p.sigma) > 1e-10 or not r["presorted"]:
                return False
            inv = invariants(p.F, p.G, r["U"], r["V"], r["Z"], r["sigma_f"], r["sigma_g"], r["sigma"])
            if not (inv["FZ"] < 1e-12 and inv["GZ"] < 1e-12 and inv["UU"] < 1e-12 and inv["VV"] < 1e-12
                    and inv["scale"] <= 8 * eps and inv["sorted"]):
                return False
    return _variant_pins_pass(lib)


def _variant_pins_pass(lib) -> bool:
    """Quick subset of the variant pins: App. A closed form and bound, the
    sort after one D-hat transformation, D-hat pivot invariants."""
    from fractions import Fraction
    x = 1.0 + 2.0 ** -27
    if oracle.dot_real([x, 1.0], [x, -(1.0 + 2.0 ** -26)], enhanced=True, lib=lib) != 2.0 ** -54:
        return False
    rng = np.random.default_rng(12)
    u = Fraction(2.0 ** -53)
    for _ in range(3000):
        re, im = rng.standard_normal(2)
        ex = Fraction(float(re)) ** 2 + Fraction(float(im)) ** 2
        got = Fraction(oracle.nrm2sq_cplx([complex(re, im)], enhanced=True, lib=lib))
        if abs(got - ex) > (Fraction(3, 2) * u + 4 * u * u) * ex:
            return False
    for t in range(60):
        p = make_pair(5, 4, 2, lo=1.0, hi=1.2, cond=3.0, seed=100 + t)
        d = np.exp(rng.uniform(-4, 4, 2))
        if not oracle.gsvd(p.F * d[None, :], p.G * d[None, :], variant=2, max_sweeps=1, lib=lib)["presorted"]:
            return False
    eps = 2.0 ** -53
    for _ in range(100):
        f = rng.standard_normal((6, 2)) * np.exp(rng.uniform(-3, 3, 2))[None, :]
        g = rng.standard_normal((6, 2)) * np.exp(rng.uniform(-3, 3, 2))[None, :]
        A, B = f.T @ f, g.T @ g
        Z, _, st = oracle.pivot_real_dscaled(A[0, 0], A[1, 1], A[0, 1], B[0, 0], B[1, 1], B[0, 1], lib=lib)
        bound = 64 * eps * np.linalg.norm(Z) ** 2
        if st != 0 or abs((Z.T @ A @ Z)[0, 1]) > bound * np.linalg.norm(A) or \
                np.max(np.abs(Z.T @ B @ Z - np.eye(2))) > bound * np.linalg.norm(B):
            return False
    return True


def test_unmutated_oracle_passes_quick_pins():
    assert _pins_pass(oracle._load())


@pytest.mark.parametrize("name,orig,mut", MUTATIONS, ids=[m[0] for m in MUTATIONS])
def test_mutation_is_caught(tmp_path, name, orig, mut):
    src = open(SRC).read()
    assert src.count(orig) >= 1, "mutation anchor not found: " + name
    msrc = tmp_path / "hz_oracle.c"
    msrc.write_text(src.replace(orig, mut, 1))
    lib_path = oracle.build(force=True, src=str(msrc), lib_path=str(tmp_path / "libmut.so"))
    lib = oracle._load(lib_path)
    assert not _pins_pass(lib), "pins did not catch mutation " + name
