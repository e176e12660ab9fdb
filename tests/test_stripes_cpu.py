"""The multi-GPU stripe algorithm of Sec. 4 on CPU ranks (gloo): the
exchange map, a full distributed solve against the oracle, and a failed rank
that the others detect on the host by a timeout instead of hanging."""
import multiprocessing as pymp
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_1909_00101_gb300 import stripes as S  # noqa: E402


def _port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


@pytest.mark.parametrize("s", [1, 2, 3, 4, 6])
def test_exchange_map_is_a_round_robin_with_consistent_targets(s):
    ns = 2 * s
    maps = S.exchange_map(s)
    assert len(maps) == ns - 1
    met = set()
    for k, row in enumerate(maps):
        held = [x for m in row for x in (m.p, m.q)]
        assert sorted(held) == list(range(ns))          # disjoint pairs covering every stripe
        for m in row:
            assert m.p < m.q and (m.p, m.q) not in met
            met.add((m.p, m.q))
        # targets: where each stripe is held in the next step (first or second)
        nxt = maps[(k + 1) % len(maps)]
        slots = {}
        for r, m in enumerate(row):
            for stripe, code in ((m.p, m.t0), (m.q, m.t1)):
                t, slot = S.decode(code)
                assert (code < 0) == (slot == 0)
                assert (nxt[t].p if slot == 0 else nxt[t].q) == stripe
                slots[(t, slot)] = slots.get((t, slot), 0) + 1
        assert all(v == 1 for v in slots.values()) and len(slots) == ns
        for r in range(s):
            src0, src1 = S.senders(maps, k, r)
            assert src0 is not None and src1 is not None
    assert len(met) == ns * (ns - 1) // 2                # every pair once per sweep


def _solve_pair(Fp, Gp):
    import oracle
    r = oracle.gsvd(Fp, Gp)
    assert r["status"] == 0
    return r["Z"], r["transf_big"]


def _solve_pair_one_sweep(Fp, Gp):
    """S = 1 sweep per pair visit (BO at the outermost level, which Sec. 4.1.4
    recommends for several GPUs): the sweep cap ends the pair solve, whose Z
    is still a valid nonsingular transformation."""
    import oracle
    r = oracle.gsvd(Fp, Gp, max_sweeps=1)
    assert r["status"] in (0, -3)
    return r["Z"], r["transf_big"]


def _rank_main(rank, world, port, out, F, G, w, fail_rank, one_sweep=False):
    import torch.distributed as dist
    from datetime import timedelta
    dist.init_process_group("gloo", init_method="tcp://127.0.0.1:%d" % port, rank=rank, world_size=world,
                            timeout=timedelta(seconds=20))
    try:
        if rank == fail_rank:
            raise SystemExit(3)  # this rank fails before its first step
        m = S.exchange_map(world)[0][rank]
        cols = list(range(m.p * w, m.p * w + w)) + list(range(m.q * w, m.q * w + w))
        Fl, Gl, Zl = S.prescale_stripes(F[:, cols], G[:, cols], m.p, m.q, w, F.shape[1])
        res = S.run(Fl, Gl, Zl, rank=rank, world=world, dist=dist,
                    solve_pair=_solve_pair_one_sweep if one_sweep else _solve_pair, max_sweeps=40,
                    timeout_s=3.0 if fail_rank >= 0 else 30.0)
        fin = S.finalize(res.F, res.G, res.Z)
        np.savez(os.path.join(out, "r%d.npz" % rank), status=res.status, sweeps=res.sweeps, p=res.p, q=res.q, **fin)
    finally:
        if rank != fail_rank:
            dist.destroy_process_group()


def _spawn(world, F, G, w, out, fail_rank=-1, one_sweep=False):
    ctx = pymp.get_context("spawn")
    port = _port()
    ps = [ctx.Process(target=_rank_main, args=(r, world, port, out, F, G, w, fail_rank, one_sweep))
          for r in range(world)]
    for p in ps:
        p.start()
    for p in ps:
        p.join(120)
    return [p.exitcode for p in ps]


@pytest.mark.parametrize("world,cplx", [(2, False), (3, False), (2, True)])
def test_ranks_match_the_oracle(tmp_path, world, cplx):
    import oracle
    from paper_1909_00101_gb300.inputs import make_pair
    w = 4
    n = 2 * world * w
    p = make_pair(40, 36, n, lo=1e-2, hi=1e2, cond=10.0, cplx=cplx, seed=5)
    codes = _spawn(world, p.F, p.G, w, str(tmp_path))
    assert codes == [0] * world
    U = np.zeros_like(p.F)
    Z = np.zeros((n, n), dtype=p.F.dtype)
    sf = np.zeros(n)
    sig = np.zeros(n)
    for r in range(world):
        d = np.load(tmp_path / ("r%d.npz" % r))
        assert int(d["status"]) == 0
        for slot, stripe in ((0, int(d["p"])), (1, int(d["q"]))):
            c = slice(stripe * w, stripe * w + w)
            loc = slice(slot * w, slot * w + w)
            U[:, c] = d["U"][:, loc]
            Z[:, c] = d["Z"][:, loc]
            sf[c] = d["sigma_f"][loc]
            sig[c] = d["sigma"][loc]
    ref = oracle.gsvd(p.F, p.G)
    got = np.sort(sig)[::-1]
    assert np.max(np.abs(got - ref["sigma"]) / ref["sigma"]) <= 1e-12
    assert np.linalg.norm(U.conj().T @ U - np.eye(n)) <= 1e-12 * n
    assert np.linalg.norm(p.F @ Z - U * sf[None, :]) / np.linalg.norm(p.F) <= 1e-13 * n


def _assemble(out, world, w, mf, mg, n, dtype):
    U = np.zeros((mf, n), dtype=dtype)
    V = np.zeros((mg, n), dtype=dtype)
    Z = np.zeros((n, n), dtype=dtype)
    sf, sg, sig = np.zeros(n), np.zeros(n), np.zeros(n)
    for r in range(world):
        d = np.load(os.path.join(out, "r%d.npz" % r))
        assert int(d["status"]) == 0
        for slot, stripe in ((0, int(d["p"])), (1, int(d["q"]))):
            c = slice(stripe * w, stripe * w + w)
            loc = slice(slot * w, slot * w + w)
            U[:, c], V[:, c], Z[:, c] = d["U"][:, loc], d["V"][:, loc], d["Z"][:, loc]
            sf[c], sg[c], sig[c] = d["sigma_f"][loc], d["sigma_g"][loc], d["sigma"][loc]
    return U, V, Z, sf, sg, sig


def test_one_sweep_per_pair_visit(tmp_path):
    """BO at the outermost level (S = 1, Sec. 4.1.4): each pair visit runs one
    sweep; the outer sweeps continue until none has a big transformation, and
    the result is the oracle's GSVD."""
    import oracle
    from paper_1909_00101_gb300.inputs import make_pair
    world, w = 2, 4
    n = 2 * world * w
    p = make_pair(40, 36, n, lo=1e-2, hi=1e2, cond=10.0, seed=9)
    codes = _spawn(world, p.F, p.G, w, str(tmp_path), one_sweep=True)
    assert codes == [0] * world
    U, V, Z, sf, sg, sig = _assemble(str(tmp_path), world, w, 40, 36, n, p.F.dtype)
    ref = oracle.gsvd(p.F, p.G)
    assert np.max(np.abs(np.sort(sig)[::-1] - ref["sigma"]) / ref["sigma"]) <= 1e-12
    assert np.linalg.norm(p.F @ Z - U * sf[None, :]) / np.linalg.norm(p.F) <= 1e-13 * n


def test_bordering_shapes():
    F = np.arange(12.0).reshape(4, 3)
    G = np.arange(15.0).reshape(5, 3) + 1.0
    Fb, Gb, k = S.border(F, G, 2, unit=2)           # n = 3 -> 8 (stripes of width 2)
    assert k == 5 and Fb.shape == (9, 8) and Gb.shape == (10, 8)
    assert np.array_equal(Fb[:4, :3], F) and np.array_equal(Gb[:5, :3], G)
    assert np.array_equal(Fb[4:, 3:], np.eye(5)) and np.array_equal(Gb[5:, 3:], np.eye(5))
    assert not Fb[:4, 3:].any() and not Fb[4:, :3].any() and not Gb[:5, 3:].any() and not Gb[5:, :3].any()
    assert S.border(F, G, 3, unit=1)[2] == 3 and S.border(Fb, Gb, 2, unit=2)[2] == 0
    with pytest.raises(ValueError):
        S.border(F, G, 0)


def test_bordered_ranks_match_the_oracle(tmp_path):
    """n = 10 on two ranks, stripes of width 4: six added columns; after the
    sweeps they are found and removed, and the original pair's GSVD remains."""
    import oracle
    from paper_1909_00101_gb300.inputs import make_pair
    world, unit = 2, 4
    p = make_pair(40, 36, 10, lo=1e-2, hi=1e2, cond=10.0, seed=15)
    Fb, Gb, k = S.border(p.F, p.G, world, unit=unit)
    nb = p.F.shape[1] + k
    w = nb // (2 * world)
    assert k == 6 and w == 4
    codes = _spawn(world, Fb, Gb, w, str(tmp_path))
    assert codes == [0] * world
    full = _assemble(str(tmp_path), world, w, Fb.shape[0], Gb.shape[0], nb, Fb.dtype)
    # every added column ends with sigma = 1 (unit f_j and g_j)
    added = np.any(full[0][40:, :] != 0, axis=0)
    assert int(added.sum()) == k and np.allclose(full[5][added], 1.0, rtol=0, atol=1e-15)
    U, V, Z, sf, sg, sig = S.unborder(*full, 40, 36, 10)
    ref = oracle.gsvd(p.F, p.G)
    assert np.max(np.abs(np.sort(sig)[::-1] - ref["sigma"]) / ref["sigma"]) <= 1e-12
    assert np.linalg.norm(U.T @ U - np.eye(10)) <= 1e-12 * 10
    assert np.linalg.norm(p.F @ Z - U * sf[None, :]) / np.linalg.norm(p.F) <= 1e-13 * 10
    assert np.linalg.norm(p.G @ Z - V * sg[None, :]) / np.linalg.norm(p.G) <= 1e-13 * 10
    # a mixed column is refused
    bad = [x.copy() for x in full]
    bad[2][nb - 1, np.flatnonzero(~added)[0]] = 1e-300
    with pytest.raises(ValueError):
        S.unborder(*bad, 40, 36, 10)


def _solve_main(rank, world, port, out, F, G, unit):
    import torch.distributed as dist
    from datetime import timedelta
    dist.init_process_group("gloo", init_method="tcp://127.0.0.1:%d" % port, rank=rank, world_size=world,
                            timeout=timedelta(seconds=30))
    try:
        grp = dist.new_group(backend="gloo")   # the stripes' own group, as on NCCL processes
        st, res = S.solve(F, G, rank=rank, world=world, dist=dist, solve_pair=_solve_pair, unit=unit, group=grp)
        if rank == 0:
            np.savez(os.path.join(out, "global.npz"), status=st, **{k: v for k, v in res.items()})
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world,n,cplx", [(2, 13, False), (3, 24, False), (2, 11, True)])
def test_whole_solve_gathered_on_process_zero(tmp_path, world, n, cplx):
    """S.solve: bordering, the sweeps on every process, and the gathered,
    unbordered, sorted GSVD on process 0 equal the oracle's."""
    import oracle
    from gsvd_checks import invariants
    from paper_1909_00101_gb300.inputs import make_pair
    p = make_pair(40, 36, n, lo=1e-2, hi=1e2, cond=10.0, cplx=cplx, seed=n)
    ctx = pymp.get_context("spawn")
    port = _port()
    ps = [ctx.Process(target=_solve_main, args=(r, world, port, str(tmp_path), p.F, p.G, 2)) for r in range(world)]
    for q in ps:
        q.start()
    for q in ps:
        q.join(120)
    assert [q.exitcode for q in ps] == [0] * world
    d = np.load(tmp_path / "global.npz")
    assert int(d["status"]) == 0 and d["U"].shape == (40, n) and d["Z"].shape == (n, n)
    ref = oracle.gsvd(p.F, p.G)
    assert np.max(np.abs(d["sigma"] - ref["sigma"]) / ref["sigma"]) <= 1e-12
    inv = invariants(p.F, p.G, d["U"], d["V"], d["Z"], d["sigma_f"], d["sigma_g"], d["sigma"])
    assert inv["FZ"] < 1e-13 * n and inv["GZ"] < 1e-13 * n and inv["UU"] < 1e-12 and inv["VV"] < 1e-12
    assert inv["sorted"] and inv["scale"] <= 8 * 2.0 ** -53


def test_single_process_solve_needs_no_process_group():
    """world = 1: two stripes on one process, exchanged locally; no
    torch.distributed calls, and the result is the oracle's GSVD."""
    import oracle
    from paper_1909_00101_gb300.inputs import make_pair
    p = make_pair(30, 26, 9, seed=21)
    st, res = S.solve(p.F, p.G, rank=0, world=1, dist=None, solve_pair=_solve_pair)
    ref = oracle.gsvd(p.F, p.G)
    assert st == 0 and res["U"].shape == (30, 9)
    assert np.max(np.abs(res["sigma"] - ref["sigma"]) / ref["sigma"]) <= 1e-12


def test_a_failed_rank_ends_the_others_waits(tmp_path):
    from paper_1909_00101_gb300.inputs import make_pair
    world, w = 2, 4
    p = make_pair(40, 36, 2 * world * w, seed=6)
    codes = _spawn(world, p.F, p.G, w, str(tmp_path), fail_rank=1)
    assert codes[1] != 0 and codes[0] == 0
    d = np.load(tmp_path / "r0.npz")
    assert int(d["status"]) == -6


def _solve_fail_main(rank, world, port, out, F, G, fail_at):
    import time
    import torch.distributed as dist
    from datetime import timedelta
    dist.init_process_group("gloo", init_method="tcp://127.0.0.1:%d" % port, rank=rank, world_size=world,
                            timeout=timedelta(seconds=60))
    if rank == 1 and fail_at == "start":
        raise SystemExit(3)                      # fails before its first step
    if rank == 1 and fail_at == "gather":
        def die(*a, **k):
            raise SystemExit(3)                  # finishes its sweeps, fails before the gather
        S._gather_parts = die
    t0 = time.time()
    st, res = S.solve(F, G, rank=rank, world=world, dist=dist, solve_pair=_solve_pair, timeout_s=3.0)
    np.savez(os.path.join(out, "r%d.npz" % rank), status=st, seconds=time.time() - t0, has=res is not None)


@pytest.mark.parametrize("fail_at", ["start", "gather"])
def test_whole_solve_with_a_failed_rank_returns_a_status(tmp_path, fail_at):
    """solve() on process 0 returns (-6, None) within its bounded waits when a
    peer dies, before its first step or just before the final gather; it
    never blocks for the process group's own (longer) timeout."""
    from paper_1909_00101_gb300.inputs import make_pair
    p = make_pair(40, 36, 16, seed=6)
    ctx = pymp.get_context("spawn")
    port = _port()
    ps = [ctx.Process(target=_solve_fail_main, args=(r, 2, port, str(tmp_path), p.F, p.G, fail_at))
          for r in range(2)]
    for q in ps:
        q.start()
    for q in ps:
        q.join(120)
    assert ps[1].exitcode != 0 and ps[0].exitcode == 0
    d = np.load(tmp_path / "r0.npz")
    assert int(d["status"]) == -6 and not bool(d["has"])
    assert float(d["seconds"]) < 40.0
