"""Write the oracle's generalized singular values of the stored cases.

    python tests/golden/make_oracle_sigma.py [case ...]      (default: every case)

For each case of ``oracle_cases.CASES`` this draws the pair with
``paper_1909_00101_gb300.inputs.make_pair`` (platform-independent), runs the
oracle in double precision and in long double (the reference values of the
rounded pair; on x86-64 long double is the 80-bit format), each in its own
process, and writes ``oracle_sigma_<case>.json`` beside this file: the
recipe, the SHA-256 of the pair's bytes, both sigma vectors as exact hex
floats, the oracle's status, sweep and transformation counts and the run
times.  Only the oracle and the input generator are called; nothing here
touches the CUDA library.  The 4096 x 2048 pair takes hours on one core.
"""
import hashlib
import json
import multiprocessing as mp
import os
import platform
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
for p in (ROOT, HERE):
    if p not in sys.path:
        sys.path.insert(0, p)


def _run(args):
    case, extended = args
    import oracle
    from oracle_cases import CASES
    from paper_1909_00101_gb300.inputs import make_pair, sha256
    os.environ.setdefault("OMP_NUM_THREADS", "1")
    p = make_pair(**CASES[case])
    t = time.time()
    r = oracle.gsvd(p.F, p.G, extended=extended, max_sweeps=100)
    dt = time.time() - t
    return dict(sha256=sha256(p.F, p.G), sigma=[float(x).hex() for x in r["sigma"]], status=int(r["status"]),
                sweeps=int(r["sweeps"]), transf_all=int(r["transf_all"]), transf_big=int(r["transf_big"]),
                seconds=round(dt, 1))


def main(cases):
    from oracle_cases import CASES, path
    jobs = [(c, x) for c in cases for x in (False, True)]
    ctx = mp.get_context("spawn")
    with ctx.Pool(min(len(jobs), os.cpu_count() or 1)) as pool:
        res = dict(zip(jobs, pool.map(_run, jobs, chunksize=1)))
    with open(os.path.join(ROOT, "oracle", "hz_oracle.c"), "rb") as f:
        src_hash = hashlib.sha256(f.read()).hexdigest()
    for c in cases:
        d, x = res[(c, False)], res[(c, True)]
        assert d["sha256"] == x["sha256"]
        sd = [float.fromhex(v) for v in d["sigma"]]
        sx = [float.fromhex(v) for v in x["sigma"]]
        err = max(abs(a - b) / abs(b) for a, b in zip(sd, sx))
        rec = dict(case=c, recipe=CASES[c], sha256=d["sha256"], n=len(sd),
                   oracle_source_sha256=src_hash, machine=platform.machine(),
                   err_fp64_vs_ext=err,
                   status_fp64=d["status"], status_ext=x["status"], sweeps_fp64=d["sweeps"], sweeps_ext=x["sweeps"],
                   transf_all_fp64=d["transf_all"], transf_big_fp64=d["transf_big"],
                   seconds_fp64=d["seconds"], seconds_ext=x["seconds"],
                   sigma_ext=x["sigma"], sigma_fp64=d["sigma"])
        with open(path(c), "w") as f:
            json.dump(rec, f, indent=0)
            f.write("\n")
        print("%s: n %d, fp64 %d sweeps %.0f s, ext %d sweeps %.0f s, err(fp64 vs ext) %.2e"
              % (c, len(sd), d["sweeps"], d["seconds"], x["sweeps"], x["seconds"], err), flush=True)


if __name__ == "__main__":
    from oracle_cases import CASES
    main(sys.argv[1:] or list(CASES))
