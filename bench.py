"""Benchmark of the GB300 implicit Hari-Zimmermann GSVD engine.

One step = one whole GSVD solve (prescale, the blocked sweep loop with its
convergence test, the final scaling and sort) of the blocked real workload
F 4096x2048, G 4096x2048 (sigma log-spaced in [1e-4, 1e4], cond(X) = 1e3,
seed 0), with the inputs resident in HBM: each step first restores the
pristine F, G (device-to-device copy, inside the timed region) because the
solve works in place.  F + G + Z = 160 MB exceed the 126 MB L2, so no flush
is needed between steps.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--precision mixed|fp64]
    python bench.py --impl reference ...     # the oracle on the host cores

Prints one JSON line (rank 0).  N > 1: one process per GPU, each solving its
own copy (replicas, no collective on the data path); value = all solves / max
time over ranks.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOAD = "blocked_real_F4096x2048_G4096x2048"
METRIC = "GSVD solves/s"
# measured FP64 peak for the DMMA contraction: the measured bf16 dense
# peak times the nominal FP64/bf16 ratio (1.25 / 2250); FP32 FFMA peak from
# unit counts and clocks: 152 SMs x 128 lanes x 2 flop x 2.07 GHz
FP64_NOMINAL_TF, BF16_NOMINAL_TF = 1.25, 2250.0
FP32_ALU_PEAK_TF = 152 * 128 * 2 * 2.07e9 / 1e12


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            m = json.load(f)
        return m.get("bf16_tflops", 1900.0), "of measured"
    except Exception:
        return 1900.0, "of fallback"


def hbm_peak_gbs():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["hbm_gbs"])
    except Exception:
        return 6800.0


class Clocks:
    """nvidia-smi sampling during the timed region."""

    def __init__(self, dev_index=0):
        self.samples = []
        self.dev = dev_index
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.dev),
                 "--query-gpu=clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
                 "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
                 "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            threading.Thread(target=self._read, daemon=True).start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.samples.append([x.strip() for x in line.split(",")])

    def stop(self):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
        out = {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": len(self.samples)}
        try:
            sm = [float(s[0]) for s in self.samples if s[0].replace(".", "").isdigit()]
            mx = [float(s[1]) for s in self.samples if s[1].replace(".", "").isdigit()]
            if sm:
                out["sm_mhz"] = float(np.median(sm))
            if mx:
                out["sm_max_mhz"] = max(mx)
            names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
            reasons = set()
            for s in self.samples:
                for k, nm in enumerate(names):
                    if len(s) > 4 + k and s[4 + k].lower().startswith("active"):
                        reasons.add(nm)
            out["reasons"] = sorted(reasons)
        except Exception:
            pass
        out["rule"] = timing_rule(out)
        return out


def timing_rule(clk: dict) -> str:
    """The timing rule on the clocks seen in the timed region: a thermal or
    hardware slowdown, or a median SM clock well below the maximum with no
    reason given (a clock lock), rejects the number; a power cap is kept."""
    bad = [r for r in clk.get("reasons", []) if r in ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown")]
    if bad:
        return "rejected: " + ", ".join(bad)
    sm, mx = clk.get("sm_mhz"), clk.get("sm_max_mhz")
    if sm is None or mx is None:
        return "unknown: no clock samples"
    if sm < 0.85 * mx and not clk.get("reasons"):
        return "rejected: SM clock %.0f of %.0f MHz with no reason" % (sm, mx)
    return "ok (power cap noted)" if "sw_power_cap" in clk.get("reasons", []) else "ok"


def dist_setup(gpus):
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if gpus > 1 and ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if os.environ.get("BENCH_BACKEND", "nccl") == "nccl" else "gloo")
        return dist, rank, ws, local
    return None, rank, ws, local


def whole_job_rate(total_ms: float, steps: int, dist, world: int, device="cpu"):
    """Whole-job throughput of N replicas: the slowest rank's time (max over
    ranks) for world x steps solves.  Returns (solves/s, max ms)."""
    if dist is not None:
        import torch
        t = torch.tensor([total_ms], dtype=torch.float64, device=device)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        total_ms = float(t.item())
    return world * steps / (total_ms / 1e3), total_ms


GOLDEN = os.path.join(ROOT, "tests", "golden", "oracle_sigma_%s.json")


def stored_oracle(case, F, G):
    """The oracle's stored record of a pair (written once by
    tests/golden/make_oracle_sigma.py, which calls only the oracle), or None
    when it is missing or was computed on other bytes (SHA-256 check)."""
    from paper_1909_00101_gb300.inputs import sha256
    try:
        with open(GOLDEN % case) as f:
            rec = json.load(f)
    except OSError:
        return None
    if rec.get("sha256") != sha256(F, G):
        return None
    for k in ("sigma_ext", "sigma_fp64"):
        rec[k] = np.array([float.fromhex(x) for x in rec[k]])
    return rec


def accuracy_vs_oracle(sig, rec):
    """sigma against the oracle's values of the same pair: the error against
    the extended-precision oracle, the R14 bound max(1e-12, 4 x the FP64
    oracle's own error) and the raw error against the FP64 oracle."""
    if rec is None:
        return {"vs_oracle": None}
    floor = float(np.max(np.abs(rec["sigma_fp64"] - rec["sigma_ext"]) / rec["sigma_ext"]))
    ex = float(np.max(np.abs(sig - rec["sigma_ext"]) / rec["sigma_ext"]))
    e64 = float(np.max(np.abs(sig - rec["sigma_fp64"]) / rec["sigma_fp64"]))
    return {"max_rel_sigma_err_vs_oracle_ext": ex, "max_rel_sigma_err_vs_oracle_fp64": e64,
            "tolerance": max(1e-12, 4.0 * floor), "within_tolerance": ex <= max(1e-12, 4.0 * floor),
            "oracle_fp64_vs_ext": floor, "oracle_sweeps": rec["sweeps_fp64"]}


def oracle_sample(F, G, n, budget_s=10.0, sweeps=None):
    """Time the oracle as it stands on a bounded sample of this workload:
    the first pivots of its sweep 1 on this pair, and extrapolate to a whole
    solve as seconds per pivot x n(n-1)/2 pivots per sweep x the oracle's
    exact sweep count on this very pair (from its stored record).  Sweep 1
    transforms nearly every pivot, later sweeps skip more of them, so the
    extrapolation bounds the solve time from above."""
    import oracle
    oracle.build()
    # calibrate the pivot count to about budget_s
    t = time.perf_counter()
    oracle.gsvd(F, G, max_pivots=2000)
    per = max(1e-7, (time.perf_counter() - t) / 2000)
    pivots = int(max(2000, min(2_000_000, budget_s / per)))
    t = time.perf_counter()
    oracle.gsvd(F, G, max_pivots=pivots)
    t_sample = time.perf_counter() - t
    src = "the oracle's exact sweep count on this pair (stored record)"
    if sweeps is None:
        sweeps, src = 30, "no stored record: 30 sweeps assumed"
    t_solve = t_sample / pivots * (n * (n - 1) / 2) * sweeps
    return {"value": 1.0 / t_solve, "unit": "solves/s", "cores": 1, "kind": "oracle",
            "sample": "%d pivots of sweep 1 of the %dx%d pair in %.1f s, extrapolated to n(n-1)/2 pivots x %d "
                      "sweeps (%s); single-threaded C, -O2 -ffp-contract=off"
                      % (pivots, F.shape[0], n, t_sample, sweeps, src),
            "est_seconds_per_solve": t_solve}


def steps_of(info, n):
    """Outer steps (Gram + inner + apply launches each) of one solve: pair
    visits / pairs per step, the round robin on the blocks of the sweeps'
    columns (n of them after the QR shortening)."""
    w = info["block_w"]
    if not w:
        return 0
    nblk = -(-n // w)
    slots = (nblk + (nblk & 1)) // 2
    return int(round(info["visits"] / max(1, slots)))


# DRAM bytes per launch of the sweep kernels at the benchmark's size, from one
# ncu capture (dram__bytes_read.sum + dram__bytes_write.sum, 64 pair visits per
# launch; profiles/sweep_kernels_dram_2048x2048.md): bytes per pair visit,
# scaled by the visits of a launch.  A figure holds for the kernel it was taken
# on: each entry names the SHA-256 of that kernel's source text, and a changed
# kernel gives null.
TRAFFIC = {
    "gram_f64": {"kernel": "k_gram_oz", "source": "k_ozaki.cu", "bytes_per_visit": (67.16e6 + 0.01e6) / 64,
                 "source_sha256": "860a1806e0ecd77257ef0138f7514488402a5ef23507740c9ae6d6b4e423b1a3"},
    "inner_f64": {"kernel": "k_inner2", "source": "k_blocked.cu", "bytes_per_visit": 4.00e6 / 64,
                  "source_sha256": "b637aa08c35fe57f6ea47b4e749c1ad9784d40529237f229aac3a104d2dfd617"},
    "apply_f64": {"kernel": "k_apply_oz", "source": "k_ozaki.cu", "bytes_per_visit": (101.26e6 + 36.8e6) / 64,
                  "source_sha256": "df068c29cfbc202a928c5549a43d4d568a8a10996b2a74d47d2d292db96071ea"},
    "gram_f32": {"kernel": "k_gram32", "source": "k_blocked.cu", "bytes_per_visit": 33.58e6 / 64,
                 "source_sha256": "57e668b5be7f57d6eb8bfbbe721f290317d8ca6ed6d9958b7dd74bdb2bdd7339"},
    "inner_f32": {"kernel": "k_inner", "source": "k_blocked.cu", "bytes_per_visit": 2.668e6 / 64,
                  "source_sha256": "7d7c84d273e049749c4c1d888e656d1b8c5ea4afe8c0863c0cee36e8f6e9590c"},
    "apply_f32": {"kernel": "k_apply32", "source": "k_blocked.cu", "bytes_per_visit": (50.61e6 + 0.04e6) / 64,
                  "source_sha256": "cb02e515db0e5c8e01f6a67a79bcfb0a30b20d850750175c357073c6f327a158"},
}


def kernel_source_sha256(source, kernel):
    """SHA-256 of a kernel's definition: from the line that declares it
    (`... kernel(`) to the first line that closes it at column 0."""
    import hashlib
    with open(os.path.join(ROOT, "paper_1909_00101_gb300", "csrc", source)) as f:
        lines = f.read().split("\n")
    for i, ln in enumerate(lines):
        if "__global__" in ln or (i > 0 and "__global__" in lines[i - 1]):
            if (" %s(" % kernel) in ln or ln.strip().startswith(kernel + "("):
                j = i
                while j < len(lines) and lines[j] != "}":
                    j += 1
                return hashlib.sha256("\n".join(lines[i:j + 1]).encode()).hexdigest()
    return None


def traffic_per_launch(kernel, units):
    ent = TRAFFIC.get(kernel)
    if not ent:
        return None
    if kernel_source_sha256(ent["source"], ent["kernel"]) != ent["source_sha256"]:
        return None
    return ent["bytes_per_visit"] * units


def lib_kw(args) -> dict:
    """Library options given on the command line (else the library's defaults)."""
    kw = {}
    if getattr(args, "fp32_params", None) is not None:
        kw["fp32_params"] = args.fp32_params
    if getattr(args, "fp64_gemm", None) is not None:
        kw["fp64_gemm"] = args.fp64_gemm
    if getattr(args, "fp32_stop", None) is not None:
        kw["fp32_stop_permille"] = args.fp32_stop
    return kw


def run_reference(args):
    """The oracle as it stands, on the host cores, on this workload (bounded samples)."""
    from paper_1909_00101_gb300.inputs import make_pair, BLOCKED_REAL_4096x2048
    p = make_pair(**BLOCKED_REAL_4096x2048)
    n = p.F.shape[1]
    rec = stored_oracle("blocked_real_4096x2048", p.F, p.G)
    vals = []
    for _ in range(args.warmup):
        pass  # the oracle has no warm state
    t0 = time.perf_counter()
    cb = None
    for _ in range(args.steps):
        cb = oracle_sample(p.F, p.G, n, budget_s=max(2.0, 30.0 / max(1, args.steps)),
                           sweeps=rec["sweeps_fp64"] if rec else None)
        vals.append(cb["value"])
    elapsed = time.perf_counter() - t0
    v = float(np.median(vals))
    cb["value"] = v
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "solves/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 / v, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "m_f": 4096, "m_g": 4096, "n": n, "sigma_range": [1e-4, 1e4],
                       "cond_x": 1e3, "seed": 0},
            "cpu_baseline": cb, "e2e": {"value": v, "unit": "solves/s", "h2d_bytes_per_step": 0,
                                        "d2h_bytes_per_step": 0},
            "sample_wall_s": elapsed}
    print(json.dumps(line))


# ---------------------------------------------------------------------------
# Other workloads (python bench.py --workload ...), one JSON line each:
#   pointwise_real_F64x32_G48x32   latency p50/p99 of single solves on the
#                                  pointwise in-shared-memory kernel, and the
#                                  throughput of 1024 such solves in one call
#   blocked_cplx_F3072x1024_G2048x1024  one complex solve, mixed vs plain FP64
#   batched_real_512               512 real pairs (n log-uniform in [16, 256],
#                                  m uniform in [n, 2n], seeds 1000..1511) in
#                                  one gsvd_solve_batched call
#   serving_poisson                a Poisson stream (n log-uniform in
#                                  [32, 1024], m in [n, 2n], real:complex 3:1)
#                                  through gsvd_submit/gsvd_poll: saturated
#                                  throughput, then p50/p99 latency at 0.7x it
# ---------------------------------------------------------------------------



def _dev(a):
    import torch
    return torch.from_numpy(np.asfortranarray(a)).cuda()


def _err(sig, ref):
    return float(np.max(np.abs(np.asarray(sig) - ref) / ref))


def pointwise(args, hz, out):
    import torch
    from paper_1909_00101_gb300.inputs import make_pair, POINTWISE_64x32
    p = make_pair(**POINTWISE_64x32)
    F0, G0 = _dev(p.F), _dev(p.G)
    for prec in ("fp64",):
        with hz.Solver(path="pointwise", order="round_robin") as s:
            for _ in range(args.warmup):
                s.solve(F0, G0)
            ts = []
            for _ in range(max(args.steps, 50)):
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                r = s.solve(F0, G0)
                ts.append(time.perf_counter() - t0)
            out["latency_us"] = {"p50": 1e6 * float(np.percentile(ts, 50)), "p99": 1e6 * float(np.percentile(ts, 99)),
                                 "device_us": r.info["t_total_us"], "sweeps": r.info["sweeps_fp64"]}
            out["accuracy"] = {"max_rel_sigma_err_vs_construction": _err(r.sigma.cpu().numpy(), p.sigma)}
            # throughput: 1024 solves of this shape in one batched call (one CTA each)
            pairs = [(F0, G0)] * 1024
            s.solve_batched(pairs)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            res = s.solve_batched(pairs)
            torch.cuda.synchronize()
            dt = time.perf_counter() - t0
            out["batched_1024"] = {"solves_per_s": 1024 / dt, "ms": 1e3 * dt,
                                   "all_ok": all(r.info["status"] == 0 for r in res)}
    # the oracle on one host core, same pair
    import oracle
    oracle.build()
    oracle.gsvd(p.F, p.G)
    t0 = time.perf_counter()
    k = 0
    while time.perf_counter() - t0 < 3.0:
        oracle.gsvd(p.F, p.G)
        k += 1
    dt = (time.perf_counter() - t0) / k
    out["cpu_baseline"] = {"value": 1.0 / dt, "unit": "solves/s", "cores": 1, "kind": "oracle",
                           "sample": "%d oracle solves of the same 64x32/48x32 pair in %.1f s" % (k, dt * k)}
    out["value"] = 1e6 / out["latency_us"]["p50"]
    out["unit"] = "solves/s (single solve latency)"
    out["metric"] = "GSVD solves/s and latency, pointwise 64x32"


def complex_blocked(args, hz, out):
    import torch
    from paper_1909_00101_gb300.inputs import make_pair, BLOCKED_CPLX_3072x1024
    p = make_pair(**BLOCKED_CPLX_3072x1024)
    F0, G0 = _dev(p.F), _dev(p.G)
    arms = {}
    for prec in ("mixed", "fp64"):
        with hz.Solver(path="blocked", precision=prec, inner_max_sweeps=1, max_sweeps=80, fp32_max_sweeps=80,
                       profile=True, block_w=args.block_w or 8, **lib_kw(args)) as s:
            s.solve(F0, G0)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            r = s.solve(F0, G0)
            torch.cuda.synchronize()
            dt = time.perf_counter() - t0
            i = r.info
            arms[prec] = {"s_per_solve": dt, "solves_per_s": 1 / dt, "sweeps_fp32": i["sweeps_fp32"],
                          "sweeps_fp64": i["sweeps_fp64"], "status": i["status"], "block_w": i["block_w"],
                          "max_rel_sigma_err_vs_construction": _err(r.sigma.cpu().numpy(), p.sigma),
                          "kernel_ms": [round(x / 1e3, 1) for x in i["t_kernel_us"]]}
    out["arms"] = arms
    out["value"] = arms["mixed"]["solves_per_s"]
    out["unit"] = "solves/s"
    out["metric"] = "GSVD solves/s, complex 3072x1024/2048x1024, mixed vs plain FP64"


def _oracle_status(fg):
    import oracle
    r = oracle.gsvd(fg[0], fg[1])
    return r["status"], r["sigma"]


def batched(args, hz, out):
    import torch
    from paper_1909_00101_gb300.inputs import make_pair, batch_shapes
    shapes = batch_shapes(512, n_lo=16, n_hi=256, seed=0)
    pairs = [make_pair(mf, mg, n, lo=1e-3, hi=1e3, cond=1e2, seed=1000 + k) for k, (mf, mg, n) in enumerate(shapes)]
    dev = [(_dev(q.F), _dev(q.G)) for q in pairs]
    arms = {}
    for prec in ("mixed", "fp64"):
        # the batched path does not shorten; the autotuner picks the block
        # width of each blocked class (n rounded up to a power of two) from
        # one timed sweep per candidate width {8, 16, 32}
        with hz.Solver(precision=prec, inner_max_sweeps=1, max_sweeps=80, fp32_max_sweeps=80, shorten=0,
                       **lib_kw(args)) as s:
            tuned = {}
            for nc in (96, 192):
                tuned[nc] = s.autotune(int(1.5 * nc), int(1.5 * nc), nc)
            s.solve_batched(dev[:32])
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            res = s.solve_batched(dev)
            torch.cuda.synchronize()
            dt = time.perf_counter() - t0
            errs = [_err(r.sigma.cpu().numpy(), q.sigma) for r, q in zip(res, pairs)]
            sig_first = [r.sigma.cpu().numpy() for r in res[:64]]
            per = [r.info["t_total_us"] / 1e3 for r in res]
            arms[prec] = {"solves_per_s": 512 / dt, "s_total": dt, "ok": sum(r.info["status"] == 0 for r in res),
                          "autotuned_block_w": {"n in (64, 128]": tuned[96], "n in (128, 256]": tuned[192]},
                          "block_w_used": sorted({r.info["block_w"] for r in res if r.info["path"] == 2}),
                          "per_problem_ms_p50": float(np.percentile(per, 50)),
                          "per_problem_ms_p99": float(np.percentile(per, 99)),
                          "pointwise": sum(r.info["path"] == 1 for r in res),
                          "max_rel_sigma_err_vs_construction": float(np.max(errs)), "_sig64": sig_first}
    out["arms"] = arms
    out["value"] = arms["mixed"]["solves_per_s"]
    out["unit"] = "solves/s"
    out["metric"] = "GSVD solves/s, 512 real pairs n in [16, 256], mixed vs plain FP64"
    # the oracle on all host cores (spawned workers), on the first 64 problems of the batch
    import multiprocessing as mp
    import os
    cores = len(os.sched_getaffinity(0))
    sample = [(q.F, q.G) for q in pairs[:64]]
    ctx = mp.get_context("spawn")
    t0 = time.perf_counter()
    with ctx.Pool(cores) as pool:
        st = pool.map(_oracle_status, sample)
    dt = time.perf_counter() - t0
    out["cpu_baseline"] = {"value": len(sample) / dt, "unit": "solves/s", "cores": cores, "kind": "oracle",
                           "sample": "the first 64 problems of the batch, %d spawned workers, %.1f s, %d ok"
                                     % (cores, dt, sum(x[0] == 0 for x in st))}
    for prec in arms:
        sg = arms[prec].pop("_sig64")
        arms[prec]["max_rel_sigma_err_vs_oracle_fp64_first64"] = float(max(_err(a, b[1]) for a, b in zip(sg, st)))


def _oracle_check(job):
    """One oracle solve (process-pool worker): (index, err vs ext oracle, R14 tolerance)."""
    k, F, G, sig = job
    import oracle
    r = oracle.gsvd(F, G)
    rx = oracle.gsvd(F, G, extended=True)
    if r["status"] != 0 or rx["status"] != 0:
        return k, None, None
    floor = float(np.max(np.abs(r["sigma"] - rx["sigma"]) / rx["sigma"]))
    return k, float(np.max(np.abs(sig - rx["sigma"]) / rx["sigma"])), max(1e-12, 4.0 * floor)


def serving(args, hz, out):
    """c5: one seeded Poisson arrival trace served through gsvd_submit /
    gsvd_poll by both arms (mixed and plain FP64) at the same rates, taken as
    fractions of the plain-FP64 saturated throughput; p50/p99 latency from
    arrival to the poll that sees the result; sigma of a stratified sample of
    requests against the oracle (spawned host workers)."""
    import multiprocessing as mp
    import torch
    from paper_1909_00101_gb300.inputs import make_pair, uniform
    R, NP = args.requests, args.pool
    # the pool of distinct pairs: n log-uniform in [32, 1024], m_F, m_G uniform
    # in [n, 2n], real:complex 3:1, sigma in [1e-4, 1e4], cond(X) = 1e3
    u = uniform(7, 0, 3 * NP)
    pool = []
    for k in range(NP):
        n = int(round(np.exp(np.log(32) + (np.log(1024) - np.log(32)) * u[3 * k])))
        mf = n + min(int(u[3 * k + 1] * (n + 1)), n)
        mg = n + min(int(u[3 * k + 2] * (n + 1)), n)
        pool.append(make_pair(mf, mg, n, lo=1e-4, hi=1e4, cond=1e3, cplx=(k % 4 == 3), seed=2000 + k))
    dev = [(_dev(q.F), _dev(q.G)) for q in pool]
    rng = np.random.default_rng(11)
    order = rng.integers(0, NP, R)
    unit_gaps = rng.exponential(1.0, R)        # one trace, scaled to each rate
    sat_n = min(R, args.sat_requests)

    def run(s, arrivals, keep=None):
        t0 = time.perf_counter()
        pending, lat, ok, results, bad = {}, [], 0, {}, []
        k = 0
        while k < len(arrivals) or pending:
            now = time.perf_counter() - t0
            while k < len(arrivals) and arrivals[k] <= now:
                F, G = dev[order[k]]
                t, res = s.submit(F, G)
                pending[t] = (k, arrivals[k], res)
                k += 1
            for t in list(pending):
                st, info = s.poll(t)
                if st != hz.EAGAIN:
                    kk, a, res = pending.pop(t)
                    lat.append(time.perf_counter() - t0 - a)
                    ok += st == 0
                    if st != 0 and len(bad) < 20:
                        q = int(order[kk])
                        bad.append({"request": kk, "pair": q, "shape": list(pool[q].F.shape) + [pool[q].G.shape[0]],
                                    "complex": bool(np.iscomplexobj(pool[q].F)), "status": int(st)})
                    if keep is not None and kk in keep:
                        results[kk] = res.sigma.cpu().numpy()
            time.sleep(0.0002)
        run.bad = bad
        return time.perf_counter() - t0, lat, ok, results

    solvers = {prec: hz.Solver(precision=prec, inner_max_sweeps=1, max_sweeps=80, fp32_max_sweeps=80,
                               max_inflight=16, hbm_budget_bytes=60 << 30, **lib_kw(args))
               for prec in ("mixed", "fp64")}
    arms = {prec: {} for prec in solvers}
    # saturated throughput (the first sat_n requests of the trace, all at t = 0)
    for prec, s in solvers.items():
        run(s, [0.0] * min(32, sat_n))  # warm-up: the pool reserves its memory
        T, lat, ok, _ = run(s, [0.0] * sat_n)
        arms[prec]["saturated"] = {"requests": sat_n, "solves_per_s": sat_n / T, "ok": ok}
    base = arms["fp64"]["saturated"]["solves_per_s"]
    # stratified sample for the oracle: requests by n bin, small enough for the host
    bins = [(32, 64), (64, 128), (128, 192)]
    per_bin = max(1, args.oracle_sample // len(bins))
    keep = set()
    for lo_n, hi_n in bins:
        idx = [k for k in range(R) if lo_n <= pool[order[k]].F.shape[1] < hi_n]
        keep.update(idx[:per_bin])
    for frac in args.loads:
        lam = frac * base
        arrivals = list(np.cumsum(unit_gaps / lam) - unit_gaps[0] / lam)
        for prec, s in solvers.items():
            T, lat, ok, res = run(s, arrivals, keep=keep)
            ent = {"lambda_per_s": lam, "solves_per_s": R / T, "ok": ok,
                   "latency_ms_p50": 1e3 * float(np.percentile(lat, 50)),
                   "latency_ms_p99": 1e3 * float(np.percentile(lat, 99))}
            if run.bad:
                ent["failed_requests"] = run.bad
            if prec == "mixed" and frac == args.loads[0] and keep:
                ctx = mp.get_context("spawn")
                cores = len(os.sched_getaffinity(0))
                jobs = [(k, pool[order[k]].F, pool[order[k]].G, res[k]) for k in sorted(keep) if k in res]
                t0 = time.perf_counter()
                with ctx.Pool(cores) as pp:
                    chk = pp.map(_oracle_check, jobs, chunksize=1)
                good = [c for c in chk if c[1] is not None]
                out["oracle_check"] = {"requests": len(jobs), "cores": cores, "seconds": time.perf_counter() - t0,
                                       "bins_n": bins, "max_err_vs_oracle_ext": max(c[1] for c in good),
                                       "all_within_tolerance": all(c[1] <= c[2] for c in good),
                                       "outside_tolerance": [{"request": c[0], "pair": int(order[c[0]]),
                                                              "err": c[1], "tol": c[2]}
                                                             for c in good if c[1] > c[2]]}
            arms[prec]["load_%.2f" % frac] = ent
    for s in solvers.values():
        s.close()
    out["arms"] = arms
    first = "load_%.2f" % args.loads[0]
    out["value"] = arms["mixed"][first]["solves_per_s"]
    out["unit"] = "solves/s"
    out["metric"] = "GSVD serving: solves/s and p50/p99 latency, Poisson arrivals, mixed vs plain FP64"
    out["config_extra"] = {"requests": R, "distinct_pairs": NP, "n_range": [32, 1024], "real_to_complex": "3:1",
                           "hbm_budget_gib": 60, "max_inflight": 16, "loads_of_fp64_saturated": list(args.loads),
                           "saturation_requests": sat_n, "trace_seed": 11}


def run_mode(args):
    import torch
    from __graft_entry__ import build
    build()
    import paper_1909_00101_gb300 as hz
    torch.cuda.init()
    out = {"workload": args.workload, "n_gpus": 1, "data": "synthetic", "higher_is_better": True}
    fn = {"pointwise_real_F64x32_G48x32": pointwise, "blocked_cplx_F3072x1024_G2048x1024": complex_blocked,
          "batched_real_512": batched, "serving_poisson": serving}[args.workload]
    fn(args, hz, out)
    print(json.dumps(out))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="mixed", choices=["mixed", "fp64"])
    ap.add_argument("--block-w", type=int, default=0)
    ap.add_argument("--inner", type=int, default=1, help="inner sweep cap of the FP64 sweeps (1 = BO, 30 = FB)")
    ap.add_argument("--max-sweeps", type=int, default=60)
    ap.add_argument("--fp32-params", type=int, default=None, choices=[0, 1],
                    help="2x2 parameters of the FP32 bulk sweeps in FP32 (1) or FP64 (0); default: library's")
    ap.add_argument("--fp64-gemm", type=int, default=None, choices=[0, 1, 2],
                    help="FP64 Gram/apply as exact BF16 slices on mma.sync (1), apply on tcgen05 (2), "
                         "or FP64 DMMA (0); default: library's")
    ap.add_argument("--fp32-stop", type=int, default=None,
                    help="FP32 sweeps stop below this many per mille big transformations; default: library's")
    ap.add_argument("--shorten", type=int, default=1, choices=[0, 1, 2],
                    help="QR shortening of Sec. 2: 0 never, 1 when m_F + m_G >= 2.6 n, 2 always")
    ap.add_argument("--compare", type=int, default=1, help="also time the other precision (1 step)")
    ap.add_argument("--e2e-steps", type=int, default=1)
    ap.add_argument("--cpu-baseline", type=int, default=1)
    ap.add_argument("--clocks", type=int, default=1, help="0: no nvidia-smi sampling (profiler runs)")
    ap.add_argument("--workload", default=WORKLOAD,
                    choices=[WORKLOAD, "pointwise_real_F64x32_G48x32", "blocked_cplx_F3072x1024_G2048x1024",
                             "batched_real_512", "serving_poisson"])
    ap.add_argument("--requests", type=int, default=2000, help="serving: requests in the Poisson stream")
    ap.add_argument("--pool", type=int, default=200, help="serving: distinct pairs the requests draw from")
    ap.add_argument("--sat-requests", type=int, default=400, help="serving: requests of the saturation runs")
    ap.add_argument("--loads", type=float, nargs="+", default=[0.7, 0.9],
                    help="serving: arrival rates as fractions of the plain-FP64 saturated throughput")
    ap.add_argument("--oracle-sample", type=int, default=102, help="serving: requests checked by the oracle")
    args = ap.parse_args()
    if args.workload != WORKLOAD and args.impl == "ours":
        run_mode(args)
        return

    if args.impl == "reference":
        if int(os.environ.get("RANK", "0")) != 0:
            return
        run_reference(args)
        return

    import torch
    dist, rank, world, local = dist_setup(args.gpus)
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    from __graft_entry__ import build
    build()
    import paper_1909_00101_gb300 as hz
    from paper_1909_00101_gb300.inputs import make_pair, BLOCKED_REAL_4096x2048

    p = make_pair(**BLOCKED_REAL_4096x2048)
    mf, n = p.F.shape
    mg = p.G.shape[0]
    F0 = torch.from_numpy(p.F).to(dev)
    G0 = torch.from_numpy(p.G).to(dev)
    # column-major working buffers (the solve overwrites them with U, V)
    F = torch.empty((n, mf), dtype=torch.float64, device=dev).t()
    G = torch.empty((n, mg), dtype=torch.float64, device=dev).t()
    Z = torch.empty((n, n), dtype=torch.float64, device=dev).t()
    sf = torch.empty(n, dtype=torch.float64, device=dev)
    sg = torch.empty_like(sf)
    sig = torch.empty_like(sf)
    stream = torch.cuda.current_stream(dev)

    def make_solver(prec, profile):
        kw = dict(precision=prec, path="blocked", profile=profile, max_sweeps=args.max_sweeps,
                  fp32_max_sweeps=args.max_sweeps, shorten=args.shorten)
        kw.update(lib_kw(args))
        if args.block_w:
            kw["block_w"] = args.block_w
        if args.inner:
            kw["inner_max_sweeps"] = args.inner
        return hz.Solver(stream=stream, **kw)

    prob = hz._problem(F, G, Z, sf, sg, sig, True)

    def step(solver):
        F.copy_(F0)
        G.copy_(G0)
        info = hz.Info()
        import ctypes
        solver._lib.gsvd_solve(solver._h, ctypes.byref(prob), ctypes.byref(info))
        return info.as_dict()

    # the timed solver runs without per-launch events; a profiled pass after
    # the timed region gives the kernel shares and per-launch durations
    solver = make_solver(args.precision, False)
    for _ in range(args.warmup):
        step(solver)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    clocks = Clocks(local)
    if args.clocks:
        clocks.start()
    evs = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps + 1)]
    infos = []
    evs[0].record(stream)
    for k in range(args.steps):
        infos.append(step(solver))
        evs[k + 1].record(stream)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    clk = clocks.stop()
    step_ms = [evs[k].elapsed_time(evs[k + 1]) for k in range(args.steps)]
    total_ms = evs[0].elapsed_time(evs[-1])
    value, total_ms = whole_job_rate(total_ms, args.steps, dist, world, dev)

    # accuracy of the last timed step: sigma against the oracle's values of
    # this pair and against the construction, residuals
    last = infos[-1]
    sig_np = sig.cpu().numpy()
    rel = float(np.max(np.abs(sig_np - p.sigma) / p.sigma))
    rec = stored_oracle("blocked_real_4096x2048", p.F, p.G)
    acc_oracle = accuracy_vs_oracle(sig_np, rec)
    Fd = F0
    res_f = float(torch.linalg.norm(Fd @ Z - F * sf[None, :]) / torch.linalg.norm(Fd))
    res_g = float(torch.linalg.norm(G0 @ Z - G * sg[None, :]) / torch.linalg.norm(G0))
    orth_u = float(torch.linalg.norm(F.t() @ F - torch.eye(n, dtype=torch.float64, device=dev)))

    # roofline of every kernel class from the event-timed launches of the timed
    # steps; the top-level entry is the dominant class.  Algorithmic work per
    # pair visit (pair width b, m = m_F + m_G): Gram b(b+1) m flops, apply
    # 2 b^2 (m + n) flops per applied visit, inner 2 b^3 / 3 (two Choleskys) +
    # b(b-1)/2 pivots x 32 b flops (four dots of b, six column updates of b).
    # With the QR shortening the sweeps run on n x n factors: m_F = m_G = n.
    names = ["gram_f64", "inner_f64", "apply_f64", "gram_f32", "inner_f32", "apply_f32"]
    prof_solver = make_solver(args.precision, True)
    infos_p = [step(prof_solver)]
    torch.cuda.synchronize()
    prof_solver.close()
    tk = np.sum([i["t_kernel_us"] for i in infos_p], axis=0)
    nk = np.sum([i["n_kernel"] for i in infos_p], axis=0)
    dom = int(np.argmax(tk))
    w = last["block_w"]
    b = 2 * w
    shortened = bool(last["shortened"])
    sm_f, sm_g = (n, n) if shortened else (mf, mg)
    visits = sum(i["visits"] for i in infos_p)
    v32 = sum(i["visits_fp32"] for i in infos_p)
    applied32 = sum(i["visits_applied_fp32"] for i in infos_p)
    applied64 = sum(i["visits_applied"] for i in infos_p) - applied32
    bf16, peak_note = measured_peaks()
    fp64_peak = bf16 * FP64_NOMINAL_TF / BF16_NOMINAL_TF
    rooflines = {}
    for k in range(6):
        if nk[k] == 0:
            continue
        avg_s = tk[k] / nk[k] / 1e6
        fp32 = names[k].endswith("f32")
        # visits per launch of this phase's kernel (FP32 bulk or FP64 sweeps)
        ph_visits = v32 if fp32 else visits - v32
        if names[k].startswith("gram"):
            units = ph_visits / nk[k]
            flops = units * b * (b + 1) * (sm_f + sm_g)
        elif names[k].startswith("apply"):
            units = (applied32 if fp32 else applied64) / nk[k]
            flops = units * 2.0 * b * b * (sm_f + sm_g + n)
        else:
            units = ph_visits / nk[k]
            flops = units * (2.0 * b ** 3 / 3 + b * (b - 1) / 2 * 32.0 * b)
        ach = flops / avg_s / 1e12
        tr = traffic_per_launch(names[k], units)
        if fp32:
            ent = {"bound": "alu", "achieved": ach, "peak": FP32_ALU_PEAK_TF, "unit": "TFLOP/s",
                   "frac": ach / FP32_ALU_PEAK_TF, "traffic": tr,
                   "peak_note": "FP32 FFMA: 152 SMs x 128 lanes x 2 flop x 2.07 GHz"}
        else:
            ent = {"bound": "alu", "achieved": ach, "peak": fp64_peak, "unit": "TFLOP/s",
                   "frac": ach / fp64_peak, "traffic": tr,
                   "peak_note": "FP64 pipe (DMMA issues on it): bf16 dense %s x 1.25/2250 nominal FP64/bf16"
                                % peak_note}
        if names[k] == "inner_f64":
            ent["note"] = ("latency-bound: 31 dependent inner steps per pair visit, each an FP64 2x2 parameter "
                           "chain and a cluster barrier; two CTAs per pair visit")
        elif names[k] == "inner_f32":
            ent["note"] = ("latency-bound: two Choleskys and 31 dependent inner steps per pair visit (FP32 "
                           "parameters, one pair per half-warp); one CTA per pair visit, 64 of 152 SMs")
        elif not fp32 and (args.fp64_gemm if args.fp64_gemm is not None else 1) >= 1:
            # the FP64 Gram and apply run as exact BF16 digit products on the
            # tensor pipe: the FP64-equivalent rate may exceed the FP64 pipe's
            # peak; the HBM fraction of the algorithmic bytes is given beside it
            by = units * 8.0 * b * ((sm_f + sm_g) if names[k].startswith("gram") else 2.0 * (sm_f + sm_g + n))
            ent["note"] = ("FP64-equivalent flops of exact BF16 digit products (36 per FP64 product): "
                           "frac > 1 = faster than the FP64 pipe could do them; limited by the integer "
                           "slicing and recombination")
            ent["hbm"] = {"algorithmic_bytes_per_launch": by, "achieved_gbs": by / avg_s / 1e9,
                          "frac": by / avg_s / 1e9 / hbm_peak_gbs(), "peak_note": "HBM copy %s" % peak_note}
        ent.update({"kernel": names[k], "avg_launch_us": avg_s * 1e6, "launches": int(nk[k]),
                    "units_per_launch": units, "flops_per_launch": flops})
        rooflines[names[k]] = ent
    if shortened:
        # the QR phase (CholeskyQR2 of F and G, U = Q_F U'', V = Q_G V''),
        # timed on the host around its launches and syncs: per m x n matrix
        # two Grams m n^2, two Choleskys n^3 / 3, two triangular solves m n^2,
        # R2 R1 n^3 / 3, Q U'' 2 m n^2  =>  6 m n^2 + n^3 flops
        t_qr = sum(i["t_qr_us"] for i in infos_p) / len(infos_p) / 1e6
        qr_flops = sum(6.0 * mm * n * n + float(n) ** 3 for mm in (mf, mg))
        ach = qr_flops / t_qr / 1e12
        rooflines["qr_phase_f64"] = {"bound": "alu", "achieved": ach, "peak": fp64_peak, "unit": "TFLOP/s",
                                     "frac": ach / fp64_peak, "traffic": None, "kernel": "qr_phase_f64",
                                     "phase_us": t_qr * 1e6, "flops_per_solve": qr_flops,
                                     "launches": int(last["qr_launches"]),
                                     "note": "whole phase incl. host syncs (two Cholesky checks)"}
    roof = dict(rooflines[names[dom]]) if nk[dom] else None
    kshare = {names[k]: round(float(tk[k] / max(1e-9, tk.sum())), 4) for k in range(6) if nk[k]}

    out = {"metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": world, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f64" if args.precision == "fp64" else "f32+f64",
           "data": "synthetic",
           "config": {"workload": WORKLOAD, "m_f": mf, "m_g": mg, "n": n, "precision": args.precision,
                      "block_w": w, "inner_max_sweeps": args.inner or 30, "shorten": args.shorten, "sigma_range": [1e-4, 1e4],
                      "cond_x": 1e3, "seed": 0, "l2": "inputs (160 MB) larger than L2"},
           "latency_ms": {"p50": float(np.percentile(step_ms, 50)), "p99": float(np.percentile(step_ms, 99)),
                          "min": float(np.min(step_ms))},
           "accuracy": dict(acc_oracle, max_rel_sigma_err_vs_construction=rel, res_FZ=res_f, res_GZ=res_g,
                            orth_U=orth_u, status=last["status"]),
           "solve": {k: last[k] for k in ("sweeps_fp32", "sweeps_fp64", "transf_all", "transf_big",
                                          "t_total_us", "t_fp32_us", "t_refine_us", "visits",
                                          "visits_applied", "chol_skipped", "shortened", "t_qr_us")},
           "kernel_time_share": kshare,
           "kernel_time_source": "one profiled solve after the timed region (per-launch CUDA events on the "
                                 "solve's stream); the timed steps run without them",
           "flop_convention": "per pair visit, pair width b = 2w, m = m_F + m_G (n x n factors when shortened): "
                              "Gram b(b+1) m; apply 2 b^2 (m + n) per applied visit; inner 2 b^3/3 (two "
                              "Choleskys) + b(b-1)/2 pivots x 32 b (four dots and six column updates of "
                              "length b, real data)",
           "roofline": roof, "rooflines": rooflines, "clocks": clk,
           "gpu_launches": None}
    # launches of our kernels in the timed region: per sweep 3 per outer step
    # (the steps of a sweep: visits / pairs per step) plus one rescale per
    # sweep, the prescale/finalize/check kernels and the QR shortening's
    out["gpu_launches"] = int(sum(3 * steps_of(i, n) + i["sweeps_fp32"] + i["sweeps_fp64"] + 14 + i["qr_launches"]
                                  for i in infos))

    if args.compare and rank == 0:
        other = "fp64" if args.precision == "mixed" else "mixed"
        s2 = make_solver(other, False)
        step(s2)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        inf2 = step(s2)
        e1.record(stream)
        torch.cuda.synchronize()
        rel2 = float(np.max(np.abs(sig.cpu().numpy() - p.sigma) / p.sigma))
        out["compare_" + other] = {"ms_per_solve": e0.elapsed_time(e1), "solves_per_s": 1e3 / e0.elapsed_time(e1),
                                   "sweeps_fp32": inf2["sweeps_fp32"], "sweeps_fp64": inf2["sweeps_fp64"],
                                   "max_rel_sigma_err_vs_construction": rel2, "status": inf2["status"]}
        s2.close()

    # end to end through the C ABI with host buffers (copies inside the timed region)
    if rank == 0 and args.e2e_steps > 0:
        Fh = np.asfortranarray(p.F).copy(order="F")
        Gh = np.asfortranarray(p.G).copy(order="F")
        Zh = np.zeros((n, n), order="F")
        vh = [np.zeros(n) for _ in range(3)]
        ph = hz._problem(Fh, Gh, Zh, vh[0], vh[1], vh[2], False)
        import ctypes
        se = make_solver(args.precision, False)
        ts = []
        for _ in range(args.e2e_steps):
            Fh[:] = p.F
            Gh[:] = p.G
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            info = hz.Info()
            se._lib.gsvd_solve(se._h, ctypes.byref(ph), ctypes.byref(info))
            ts.append(time.perf_counter() - t0)
        se.close()
        out["e2e"] = {"value": 1.0 / float(np.median(ts)), "unit": "solves/s",
                      "h2d_bytes_per_step": int(Fh.nbytes + Gh.nbytes),
                      "d2h_bytes_per_step": int(Fh.nbytes + Gh.nbytes + Zh.nbytes + 3 * 8 * n),
                      "status": info.status}

    if rank == 0 and args.cpu_baseline:
        out["cpu_baseline"] = oracle_sample(p.F, p.G, n, sweeps=rec["sweeps_fp64"] if rec else None)
    solver.close()
    if rank == 0:
        print(json.dumps(out))
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
