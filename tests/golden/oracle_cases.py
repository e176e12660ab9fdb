"""Recipes of the input pairs whose oracle values are stored under tests/golden/.

Each case is a ``make_pair`` call of ``paper_1909_00101_gb300.inputs``; the
generator is bit-identical on every IEEE machine, and each stored file also
records the SHA-256 of the pair's bytes, which the tests check before they
use the stored values.  ``make_oracle_sigma.py`` (same folder) computes the
values with the oracle alone.
"""
import json
import os

HERE = os.path.dirname(os.path.abspath(__file__))

CASES = {
    # the 4096 x 4096 x 2048 real benchmark pair: sigma in [1e-4, 1e4], cond(X) = 1e3
    "blocked_real_4096x2048": dict(mf=4096, mg=4096, n=2048, lo=1e-4, hi=1e4, cond=1e3, cplx=False, seed=0),
    # the complex 3072 x 2048 x 1024 pair: sigma in [1e-3, 1e3], cond(X) = 1e3
    "blocked_cplx_3072x1024": dict(mf=3072, mg=2048, n=1024, lo=1e-3, hi=1e3, cond=1e3, cplx=True, seed=0),
    # mid-size pairs solved unshortened: several Gram row splits, hundreds of apply tiles
    "mid_real_3000x2500x512": dict(mf=3000, mg=2500, n=512, lo=1e-4, hi=1e4, cond=1e3, cplx=False, seed=7),
    "mid_cplx_1500x1200x256": dict(mf=1500, mg=1200, n=256, lo=1e-3, hi=1e3, cond=1e3, cplx=True, seed=7),
}

# batched problems of the 512-pair batch's distribution (n log-uniform in
# [16, 256], m uniform in [n, 2n], sigma in [1e-3, 1e3], cond 1e2), the
# larger ones that take the blocked path
BATCH_SHAPES = [(300, 260, 256), (400, 390, 200), (250, 300, 160), (220, 130, 128), (150, 170, 97), (90, 80, 72)]
for _k, (_mf, _mg, _n) in enumerate(BATCH_SHAPES):
    CASES["batch_real_%d" % _k] = dict(mf=_mf, mg=_mg, n=_n, lo=1e-3, hi=1e3, cond=1e2, cplx=False, seed=1000 + _k)


def path(case: str) -> str:
    return os.path.join(HERE, "oracle_sigma_%s.json" % case)


def load(case: str) -> dict:
    """The stored record of a case, with sigma arrays decoded (float64)."""
    import numpy as np
    with open(path(case)) as f:
        rec = json.load(f)
    for k in ("sigma_ext", "sigma_fp64"):
        rec[k] = np.array([float.fromhex(x) for x in rec[k]])
    return rec


def load_checked(case: str, F, G) -> dict:
    """The stored record of a case after checking that (F, G) is the very pair
    it was computed on (SHA-256 of the bytes); raises if not."""
    from paper_1909_00101_gb300.inputs import sha256
    rec = load(case)
    got = sha256(F, G)
    if got != rec["sha256"]:
        raise AssertionError("input pair of %s differs from the stored one (sha256 %s, stored %s)"
                             % (case, got, rec["sha256"]))
    return rec
