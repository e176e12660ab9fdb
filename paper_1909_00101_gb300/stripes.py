"""A CPU simulation of the multi-GPU stripe algorithm of Sec. 4: the schedule,
the exchange map and a host driver over processes.

This is not the library's data plane: the stripes, their exchange and the
application of each pair's transformation to the pair's columns (a host
matrix product) run on the host, as CPU tensors between processes; the device work of a pair solve can
be the library's (library_pair_solver) or, in the tests, the oracle's.

The columns of F, G and Z are cut into ns = 2 s stripes of equal width (s
processes, one per GPU).  In each outer step every process holds two stripes,
runs the single-GPU algorithm on that pair (the pair is a GSVD problem of its
own: any nonsingular transformation Z_pq that it returns is applied to the
pair's columns of F, G and Z), and then sends each of its two transformed
stripes to the process that holds that stripe in the next step, as its first
or second stripe.  The steps of a sweep follow the round-robin ordering of the
ns stripes (every pair of stripes meets once per sweep); a sweep ends with one
sum-reduction of the big-transformation counters, and the algorithm stops
after a sweep without big transformations (Sec. 4.2, Sec. 2.5).

The exchange map follows Sec. 4.1.3: for step k and process r it gives the
pair (p, q) the process holds and, for each of its two stripes, the target
process encoded as -(t + 1) when the stripe becomes the target's first stripe
and t + 1 when it becomes the second.

n not divisible into 2 s stripes of one width is bordered first (border,
unborder: Sec. 3.1, Sec. 4.1).  solve() runs the whole method for a process
that holds the full pair and gathers the GSVD on process 0.

The pair solver is passed in.  Stripes travel as CPU tensors in a gloo
group.  Any process that fails ends the others' waits by a timeout, which
the driver reports as a status instead of hanging; that holds for the final
gather of solve() too.
"""
from __future__ import annotations

from dataclasses import dataclass
from datetime import timedelta

import numpy as np


def round_robin(ns: int) -> list:
    """Round-robin ("circle method") ordering of ns (even) stripes: ns - 1
    steps of ns / 2 disjoint pairs (p, q), p < q; stripe ns - 1 stays, the
    others rotate.  Every pair of stripes occurs in exactly one step."""
    if ns < 2 or ns % 2:
        raise ValueError("need an even number of stripes >= 2")
    steps = []
    for s in range(ns - 1):
        pairs = []
        for k in range(ns // 2):
            if k == 0:
                a, b = ns - 1, s
            else:
                a, b = (s + k) % (ns - 1), (s - k + (ns - 1)) % (ns - 1)
            pairs.append((min(a, b), max(a, b)))
        steps.append(pairs)
    return steps


@dataclass(frozen=True)
class StepMap:
    p: int    # global index of the first local stripe
    q: int    # global index of the second local stripe
    t0: int   # target of the first stripe: -(t + 1) as the target's first stripe, t + 1 as its second
    t1: int   # target of the second stripe, encoded alike


def exchange_map(s: int) -> list:
    """The map (k, r) -> (p, q, t0, t1) of Sec. 4.1.3 for s processes and 2 s
    stripes: [k][r] for the ns - 1 steps of a sweep.  The step after the last
    one is step 0 of the next sweep."""
    ns = 2 * s
    steps = round_robin(ns)
    holder = []
    for pairs in steps:
        h = {}
        for r, (p, q) in enumerate(pairs):
            h[p] = (r, 0)
            h[q] = (r, 1)
        holder.append(h)
    out = []
    for k, pairs in enumerate(steps):
        nxt = holder[(k + 1) % len(steps)]
        row = []
        for r, (p, q) in enumerate(pairs):
            codes = []
            for stripe in (p, q):
                t, slot = nxt[stripe]
                codes.append(-(t + 1) if slot == 0 else t + 1)
            row.append(StepMap(p, q, codes[0], codes[1]))
        out.append(row)
    return out


def decode(code: int) -> tuple:
    """(target process, slot 0 or 1) of an encoded target."""
    return (-code - 1, 0) if code < 0 else (code - 1, 1)


def senders(maps: list, k: int, r: int) -> tuple:
    """(process, its local stripe 0 or 1) that sends this process's slot 0 and
    slot 1 stripes after step k."""
    src = [None, None]
    for rr, m in enumerate(maps[k]):
        for local, code in enumerate((m.t0, m.t1)):
            t, slot = decode(code)
            if t == r:
                src[slot] = (rr, local)
    return src[0], src[1]


@dataclass
class StripeResult:
    status: int            # 0 ok, -3 no convergence in max_sweeps, -6 a wait timed out (another process failed)
    sweeps: int
    p: int                 # global stripe indices held at the end (first, second)
    q: int
    F: np.ndarray          # the two stripes of F, G, Z after the sweeps (not normalised)
    G: np.ndarray
    Z: np.ndarray


def prescale_stripes(F: np.ndarray, G: np.ndarray, p: int, q: int, w: int, n: int) -> tuple:
    """Sec. 3.3 prescaling of two stripes (global stripes p and q of width w):
    z_j = 1 / ||g_j||, f_j *= z_j, g_j *= z_j, and Z0's columns for them
    (n x 2w, z_j in the global row of column j)."""
    s = np.sqrt(np.sum(np.abs(G) ** 2, axis=0))
    if np.any(s == 0.0) or not np.all(np.isfinite(s)):
        raise ValueError("G is rank deficient")
    z = 1.0 / s
    Z0 = np.zeros((n, 2 * w), dtype=np.result_type(F.dtype, G.dtype))
    cols = list(range(p * w, p * w + w)) + list(range(q * w, q * w + w))
    for j, c in enumerate(cols):
        Z0[c, j] = z[j]
    return F * z[None, :], G * z[None, :], Z0


def border(F: np.ndarray, G: np.ndarray, s: int, unit: int = 1) -> tuple:
    """Bordering of Sec. 3.1 and Sec. 4.1: n is enlarged by k columns to a
    multiple of 2 s unit, so that the 2 s stripes have one width, a multiple
    of unit.  F and G each gain k rows and k columns; added column n + i has
    a one in added row m_Y + i and zeros elsewhere.  The added columns keep
    F and G of full column rank and are orthogonal to the original ones, so
    no transformation mixes them in (their Gram couplings are exact zeros)
    and each ends with the generalized singular value 1.  Returns (F, G, k);
    k = 0 returns the inputs."""
    if s < 1 or unit < 1:
        raise ValueError("need s >= 1 and unit >= 1")
    n = F.shape[1]
    k = (-n) % (2 * s * unit)
    if k == 0:
        return F, G, 0

    def grow(Y):
        m = Y.shape[0]
        B = np.zeros((m + k, n + k), dtype=Y.dtype, order="F")
        B[:m, :n] = Y
        B[m + np.arange(k), n + np.arange(k)] = 1.0
        return B
    return grow(F), grow(G), k


def unborder(U: np.ndarray, V: np.ndarray, Z: np.ndarray, sigma_f: np.ndarray, sigma_g: np.ndarray,
             sigma: np.ndarray, mf: int, mg: int, n: int) -> tuple:
    """The GSVD of the original pair from that of the bordered one (columns in
    any order, e.g. assembled from the processes' stripes): an added column
    is one whose u_j lies in the added rows.  Original columns never mix
    with added ones, so their U, V and Z have exact zeros in the added rows;
    anything else raises ValueError.  Returns U (m_F x n), V (m_G x n),
    Z (n x n) and the three sigma vectors, original columns in the given
    order."""
    added = np.any(U[mf:, :] != 0, axis=0)
    keep = ~added
    if int(keep.sum()) != n:
        raise ValueError("expected %d original columns, found %d" % (n, int(keep.sum())))
    if np.any(V[mg:, keep] != 0) or np.any(Z[n:, keep] != 0):
        raise ValueError("an original column was mixed with an added one")
    return U[:mf, keep], V[:mg, keep], Z[:n, keep], sigma_f[keep], sigma_g[keep], sigma[keep]


def _wire(x: np.ndarray):
    import torch
    x = np.ascontiguousarray(x)
    if np.iscomplexobj(x):
        return torch.from_numpy(np.ascontiguousarray(x.view(np.float64)))
    return torch.from_numpy(x)


def _unwire(t, cplx: bool) -> np.ndarray:
    a = t.numpy()
    return np.ascontiguousarray(a).view(np.complex128) if cplx else a


def _run(F, G, Z, *, rank, world, dist, solve_pair, max_sweeps=30, timeout_s=30.0, group=None) -> StripeResult:
    import torch
    maps = exchange_map(world)
    nsteps = len(maps)
    w = F.shape[1] // 2
    mf, mg, n = F.shape[0], G.shape[0], Z.shape[0]
    rows = mf + mg + n
    tmo = timedelta(seconds=timeout_s)
    # the pair's columns of F, G and Z stacked (rows x 2w), one buffer
    buf = np.concatenate([F, G, Z], axis=0)
    cplx = np.iscomplexobj(buf)
    sweeps = 0
    for sweep in range(max_sweeps):
        big = 0
        for k in range(nsteps):
            m = maps[k][rank]
            Fpq, Gpq = buf[:mf], buf[mf:mf + mg]
            Zpq, b = solve_pair(np.ascontiguousarray(Fpq), np.ascontiguousarray(Gpq))
            buf = buf @ Zpq
            big += int(b)
            # exchange: each local stripe to its holder in the next step
            # (complex stripes travel as their real view)
            out = [_wire(buf[:, :w]), _wire(buf[:, w:])]
            inc = [torch.empty_like(out[0]) for _ in range(2)]
            src = senders(maps, k, rank)
            works = []
            local_copy = {}
            for slot in (0, 1):
                sr, sl = src[slot]
                if sr == rank:
                    local_copy[slot] = sl
                else:
                    works.append(dist.irecv(inc[slot], src=sr, tag=slot + 1, group=group))
            for local, code in enumerate((m.t0, m.t1)):
                t, slot = decode(code)
                if t != rank:
                    works.append(dist.isend(out[local], dst=t, tag=slot + 1, group=group))
            for slot, sl in local_copy.items():
                inc[slot].copy_(out[sl])
            try:
                for wk in works:
                    wk.wait(tmo)
            except RuntimeError:
                return StripeResult(-6, sweeps, m.p, m.q, buf[:mf], buf[mf:mf + mg], buf[mf + mg:])
            buf = np.concatenate([_unwire(inc[0], cplx), _unwire(inc[1], cplx)], axis=1)
        sweeps += 1
        tot = torch.tensor([big], dtype=torch.int64)
        try:
            if world > 1:
                dist.all_reduce(tot, group=group, async_op=True).wait(tmo)
        except RuntimeError:
            m = maps[0][rank]
            return StripeResult(-6, sweeps, m.p, m.q, buf[:mf], buf[mf:mf + mg], buf[mf + mg:])
        if int(tot.item()) == 0:
            m = maps[0][rank]
            return StripeResult(0, sweeps, m.p, m.q, buf[:mf], buf[mf:mf + mg], buf[mf + mg:])
    m = maps[0][rank]
    return StripeResult(-3, sweeps, m.p, m.q, buf[:mf], buf[mf:mf + mg], buf[mf + mg:])


def run(F, G, Z, *, rank, world, dist, solve_pair, max_sweeps: int = 30, timeout_s: float = 30.0,
        group=None) -> StripeResult:
    """The sweeps of Sec. 4.2 for this process.

    F (m_F x 2w), G (m_G x 2w), Z (n x 2w): this process's two stripes of
    step 0 (its pair in exchange_map(world)[0][rank]), prescaled
    (prescale_stripes).  solve_pair(Fpq, Gpq) -> (Zpq, big): a nonsingular
    transformation of the pair and its count of big transformations.  dist:
    torch.distributed with an initialised process group; group: the group
    the stripes travel in (None = the default one).  The stripes are host
    arrays and travel as CPU tensors, between host buffers as the paper's
    CPU stripes do, so the group's backend must move CPU tensors (gloo; on
    GPU processes whose default group is NCCL, pass a gloo group made with
    dist.new_group(backend="gloo")).  A wait that runs
    out of time (a failed peer) gives status -6; no convergence in
    max_sweeps gives -3.  At the end every process holds the stripes of step
    0 again (the map wraps around after each sweep).
    """
    return _run(F, G, Z, rank=rank, world=world, dist=dist, solve_pair=solve_pair, max_sweeps=max_sweeps,
                timeout_s=timeout_s, group=group)


def library_pair_solver(solver):
    """solve_pair for run() on a GPU process: the library's solve of the pair
    (host arrays in, through the C ABI; the pair's Z and its count of big
    transformations out).  solver: a paper_1909_00101_gb300.Solver.  Its
    max_sweeps is the number S of sweeps per pair visit: 1 is the
    block-oriented choice that Sec. 4.1.4 recommends across GPUs (a pair
    solve that stops at the cap still returns a valid transformation)."""
    def solve_pair(Fp, Gp):
        r = solver.solve(np.asfortranarray(Fp), np.asfortranarray(Gp))
        if r.status not in (0, -3):
            raise RuntimeError("pair solve failed: status %d" % r.status)
        return np.asarray(r.Z), int(r.info["transf_big"])
    return solve_pair


def finalize(F: np.ndarray, G: np.ndarray, Z: np.ndarray) -> dict:
    """Sec. 3.4 for a process's columns: Sigma_F = ||f_j||, Sigma_G = ||g_j||,
    Theta_j = (Sigma_F^2 + Sigma_G^2)^(-1/2), U = F / ||f||, V = G / ||g||,
    Z Theta, and Sigma = ||f_j|| / ||g_j|| (not sorted)."""
    sf = np.sqrt(np.sum(np.abs(F) ** 2, axis=0))
    sg = np.sqrt(np.sum(np.abs(G) ** 2, axis=0))
    th = 1.0 / np.sqrt(sf * sf + sg * sg)
    return {"U": F / sf[None, :], "V": G / sg[None, :], "Z": Z * th[None, :], "sigma_f": sf * th,
            "sigma_g": sg * th, "sigma": sf / sg}


def _gather_parts(part, rank, world, dist, group, timeout_s):
    """Process 0 collects every process's part (point to point: a length, then
    the pickled bytes), each wait bounded by timeout_s.  Returns the list on
    process 0 (None when a wait ran out: a peer failed), [] elsewhere (None
    when its send timed out)."""
    import pickle

    import torch
    tmo = timedelta(seconds=timeout_s)
    try:
        if rank != 0:
            payload = torch.frombuffer(bytearray(pickle.dumps(part)), dtype=torch.uint8)
            size = torch.tensor([payload.numel()], dtype=torch.int64)
            dist.isend(size, dst=0, tag=101, group=group).wait(tmo)
            dist.isend(payload, dst=0, tag=102, group=group).wait(tmo)
            return []
        parts = [part] + [None] * (world - 1)
        for src in range(1, world):
            size = torch.zeros(1, dtype=torch.int64)
            dist.irecv(size, src=src, tag=101, group=group).wait(tmo)
            payload = torch.empty(int(size.item()), dtype=torch.uint8)
            dist.irecv(payload, src=src, tag=102, group=group).wait(tmo)
            parts[src] = pickle.loads(payload.numpy().tobytes())
        return parts
    except RuntimeError:
        return None


def solve(F: np.ndarray, G: np.ndarray, *, rank: int, world: int, dist, solve_pair, unit: int = 1,
          max_sweeps: int = 30, timeout_s: float = 30.0, group=None):
    """The whole multi-process GSVD of Sec. 4 for one process that holds the
    full pair (F, G): bordering (Sec. 3.1, Sec. 4.1) to 2 world stripes of one
    width (a multiple of unit), this process's two stripes of step 0 with the
    prescaling of Sec. 3.3, the sweeps (run), the final rescaling of Sec. 3.4
    on its columns, and a gather to process 0, which removes the bordering
    and sorts by descending Sigma (stable).  Returns (status, result): on
    process 0 result is a dict with U, V, Z, sigma_f, sigma_g, sigma and
    sweeps; elsewhere None.  The status is the worst of the processes'
    (0 ok, -3 no convergence, -6 a wait timed out)."""
    mf, n = F.shape
    mg = G.shape[0]
    Fb, Gb, k = border(F, G, world, unit=unit)
    nb = n + k
    w = nb // (2 * world)
    m = exchange_map(world)[0][rank]
    cols = list(range(m.p * w, m.p * w + w)) + list(range(m.q * w, m.q * w + w))
    Fl, Gl, Zl = prescale_stripes(Fb[:, cols], Gb[:, cols], m.p, m.q, w, nb)
    res = run(Fl, Gl, Zl, rank=rank, world=world, dist=dist, solve_pair=solve_pair, max_sweeps=max_sweeps,
              timeout_s=timeout_s, group=group)
    fin = finalize(res.F, res.G, res.Z)
    part = (res.status, res.sweeps, res.p, res.q, fin)
    if world == 1:
        parts = [part]
    else:
        parts = _gather_parts(part, rank, world, dist, group, timeout_s)
        if parts is None:
            return -6, None
    if rank != 0:
        return res.status, None
    status = 0
    for st, *_ in parts:
        if st != 0 and (status == 0 or st < status):
            status = st
    dt = np.result_type(F.dtype, G.dtype)
    U = np.zeros((Fb.shape[0], nb), dtype=dt)
    V = np.zeros((Gb.shape[0], nb), dtype=dt)
    Z = np.zeros((nb, nb), dtype=dt)
    sf, sg, sig = np.zeros(nb), np.zeros(nb), np.zeros(nb)
    for _, _, p, q, f in parts:
        for slot, stripe in ((0, p), (1, q)):
            c = slice(stripe * w, stripe * w + w)
            loc = slice(slot * w, slot * w + w)
            U[:, c], V[:, c], Z[:, c] = f["U"][:, loc], f["V"][:, loc], f["Z"][:, loc]
            sf[c], sg[c], sig[c] = f["sigma_f"][loc], f["sigma_g"][loc], f["sigma"][loc]
    if k:
        U, V, Z, sf, sg, sig = unborder(U, V, Z, sf, sg, sig, mf, mg, n)
    order = np.argsort(-sig, kind="stable")
    out = {"U": U[:, order], "V": V[:, order], "Z": Z[:, order], "sigma_f": sf[order], "sigma_g": sg[order],
           "sigma": sig[order], "sweeps": max(pp[1] for pp in parts)}
    return status, out
