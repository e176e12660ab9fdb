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


# pairs of the GPU parity tests whose oracle run is slow where long double is
# the 128-bit software format (AArch64): stored once, found by their SHA-256
_T = dict(lo=1e-3, hi=1e3, cond=1e2)
CASES.update({
    "t_autotune_600x500x256": dict(mf=600, mg=500, n=256, lo=1e-2, hi=1e2, cond=1e2, cplx=False, seed=17),
    "t_shortened_mixed_700x600x192": dict(mf=700, mg=600, n=192, lo=1e-4, hi=1e4, cond=1e3, cplx=False, seed=31),
    "t_shortened_512x400x160": dict(mf=512, mg=400, n=160, cplx=False, seed=160, **_T),
    "t_shortened_333x1000x97": dict(mf=333, mg=1000, n=97, cplx=False, seed=97, **_T),
    "t_shortened_2000x150x129": dict(mf=2000, mg=150, n=129, cplx=False, seed=129, **_T),
    "t_mixed_200x160x128": dict(mf=200, mg=160, n=128, cplx=False, seed=21, **_T),
    "t_mixed_cplx_200x160x128": dict(mf=200, mg=160, n=128, cplx=True, seed=21, **_T),
    "t_mixed_p32_200x160x128": dict(mf=200, mg=160, n=128, cplx=False, seed=22, **_T),
    "t_mixed_p32_cplx_200x160x128": dict(mf=200, mg=160, n=128, cplx=True, seed=22, **_T),
    "t_blocked_w32_300x257x150": dict(mf=300, mg=257, n=150, cplx=False, seed=182, **_T),
    "t_blocked_w16_200x180x100": dict(mf=200, mg=180, n=100, cplx=False, seed=116, **_T),
    "t_right_300x260x128": dict(mf=300, mg=260, n=128, cplx=False, seed=131, **_T),
    "t_serving_300x280x160": dict(mf=300, mg=280, n=160, lo=1e-2, hi=1e2, cond=1e2, cplx=False, seed=204),
    "t_serving_200x150x100": dict(mf=200, mg=150, n=100, lo=1e-2, hi=1e2, cond=1e2, cplx=False, seed=201),
    "t_serving_cplx_90x80x70": dict(mf=90, mg=80, n=70, lo=1e-2, hi=1e2, cond=1e2, cplx=True, seed=202),
})
for _w in (4, 8, 16):
    CASES["t_blocked_cplx_w%d_120x90x72" % _w] = dict(mf=120, mg=90, n=72, cplx=True, seed=_w, **_T)


def by_sha256() -> dict:
    """{sha256 of a pair: case} over the stored records (read once)."""
    global _INDEX
    if _INDEX is None:
        _INDEX = {}
        for c in CASES:
            try:
                with open(path(c)) as f:
                    head = f.read(4096)
                i = head.index('"sha256"')
                _INDEX[head[i:].split('"')[3]] = c
            except (OSError, ValueError, IndexError):
                pass
    return _INDEX


_INDEX = None


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
