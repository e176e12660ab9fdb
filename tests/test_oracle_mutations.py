"""The oracle pins have teeth: a plausible mistake planted in a copy of the
oracle (on the CPU only) makes at least one pin fail.

Each mutation is a one-token edit of hz_oracle.c (a flipped sign, a dropped
term, a swapped index or operand); the mutated copy is compiled into a
temporary library and run through a quick subset of the pins.
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
        r = oracle.gsvd(p.F, p.G, lib=lib)
        if r["status"] != 0 or rel_sigma_err(r["sigma"], p.sigma) > 1e-10:
            return False
        inv = invariants(p.F, p.G, r["U"], r["V"], r["Z"], r["sigma_f"], r["sigma_g"], r["sigma"])
        if not (inv["FZ"] < 1e-12 and inv["GZ"] < 1e-12 and inv["UU"] < 1e-12 and inv["VV"] < 1e-12
                and inv["scale"] <= 8 * eps and inv["sorted"]):
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
