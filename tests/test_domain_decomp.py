"""x-slab domain decomposition of one instance, checked on the oracle.

Each "rank" owns a slab of c-bin columns, receives the particles of the two
columns on either side (the halo), runs the oracle's step on owned + halo
particles with global ids and the global contact distance, keeps its owned
particles and hands the ones that left its slab to their new owners.  Because
the pair decision is local (closest candidate in the 3^D neighbourhood, mutual
choice), the decomposed run must equal the undivided run bit for bit: state,
partners and per-c-bin moments.  A halo of one column must not suffice.

The ranks run in one process (2, 3 and 4 ranks, buffers exchanged in memory)
and as two gloo processes (buffers exchanged by torch.distributed).
"""
import importlib.util
import os
import socket

import numpy as np
import pytest

import oracle as orc

_ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _by_path(name, rel):
    spec = importlib.util.spec_from_file_location(name, os.path.join(_ROOT, *rel.split("/")))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


decomp = _by_path("kmc_decomp", "paper_1210_8084_gb300/decomp.py")
inputs = _by_path("kmc_inputs", "paper_1210_8084_gb300/inputs.py")

# rows exchanged between ranks: id, position (3), velocity (3), virial
_NCOL = 8


def _rows(ids, pos, vel, W):
    return np.column_stack([ids.astype(np.float64), pos, vel, W])


def _unrows(b):
    return b[:, 0].astype(np.int64), b[:, 1:4].copy(), b[:, 4:7].copy(), b[:, 7].copy()


def _columns(P, pos):
    _, cidx = orc.cell_keys(P, pos)
    cx = cidx[:, 0].astype(np.int64)
    cx[np.isnan(pos[:, 0])] = -1          # absorbed: no column, no owner
    return cx


def _case(name):
    """(params factory, ids, pos, vel, dt_mode) of a small seeded problem."""
    if name == "slab_walls":        # 1-D slab c-bins, walls in x (the Sod tube)
        n = 3000
        pos, vel = inputs.sod_tube(n, seed=3)
        dim, cells, bc = 3, (24, 1, 1), (1, 0, 0)
        lam = 2e-3
    elif name == "box_periodic":    # 3-D c-bins, periodic everywhere: halos wrap
        n = 2500
        pos, vel = inputs.periodic_box(n, seed=5)
        dim, cells, bc = 3, (10, 3, 3), (0, 0, 0)
        lam = 1e-2
    elif name == "plane_absorb":    # 2-D positions, absorbing x walls
        n = 2000
        pos, vel = inputs.sod_tube(n, seed=7)
        dim, cells, bc = 2, (16, 6, 1), (2, 0, 0)
        lam = 5e-3
    else:
        raise KeyError(name)
    V = 1.0
    R2 = orc.contact_R2(lam, 0.0, n / V)
    dx = 1.0 / cells[0]

    def params(step, dt):
        return orc.make_params(dim, cells, (0, 0, 0), (1, 1, 1), bc, R2, dt, seed=11, step=step)

    return params, np.arange(n, dtype=np.int64), pos.astype(np.float64), vel.astype(np.float64), 0.5 * dx


def _undivided(params, pos, vel, steps, dt_fixed, adaptive):
    out = []
    for k in range(steps):
        dt = orc.adaptive_dt(params(k, 1.0), vel, dt_rest=dt_fixed) if adaptive else dt_fixed
        P = params(k, dt)
        pos, vel, best, paired, raw, der, glob, npairs = orc.step(P, pos, vel)
        out.append(dict(pos=pos, vel=vel, paired=paired, raw=raw, der=der, glob=glob, npairs=npairs))
    return out


def _rank_step(P, own, halo):
    """The oracle's step on owned + halo particles (increasing global ids);
    returns the owned particles' end-of-step rows and partners (global ids)."""
    ids = np.concatenate([own[0], halo[0]])
    pos = np.concatenate([own[1], halo[1]])
    vel = np.concatenate([own[2], halo[2]])
    mine = np.concatenate([np.ones(len(own[0]), bool), np.zeros(len(halo[0]), bool)])
    order = np.argsort(ids, kind="stable")
    ids, pos, vel, mine = ids[order], pos[order], vel[order], mine[order]
    best = orc.best_partners(P, pos, vel)
    po, vo, W, paired = orc.collide_move(P, pos, vel, best, ids=ids)
    partner = np.where(paired >= 0, ids[np.maximum(paired, 0)], -1)
    return (ids[mine], po[mine], vo[mine], W[mine]), partner[mine]


def _sorted(state):
    o = np.argsort(state[0], kind="stable")
    return tuple(a[o] for a in state)


def _decomposed(params, ids, pos, vel, steps, dt_fixed, adaptive, world, width=decomp.HALO, weighted=False):
    """All ranks in one process; buffers exchanged by transposing send lists."""
    P0 = params(0, dt_fixed)
    n_x = P0.n_cells[0]
    periodic = P0.bc[0] == 0
    cx = _columns(P0, pos)
    w = np.bincount(cx[cx >= 0], minlength=n_x) if weighted else None
    bounds = decomp.slab_bounds(n_x, world, w)
    own = decomp.owner(cx, bounds)
    W0 = np.zeros(len(ids))
    ranks = [_sorted((ids[own == r], pos[own == r], vel[own == r], W0[own == r])) for r in range(world)]
    out = []
    for k in range(steps):
        if adaptive:
            dt = min(orc.adaptive_dt(params(k, 1.0), st[2], dt_rest=dt_fixed) for st in ranks)
        else:
            dt = dt_fixed
        P = params(k, dt)
        # halo exchange
        sends = []
        for r, st in enumerate(ranks):
            idx = decomp.halo_sends(_columns(P, st[1]), r, bounds, periodic, width)
            sends.append([_rows(st[0][i], st[1][i], st[2][i], st[3][i]) for i in idx])
        new, partners, crossed = [], {}, 0
        for r, st in enumerate(ranks):
            got = [sends[q][r] for q in range(len(ranks)) if q != r]
            halo = _unrows(np.concatenate(got) if got else np.zeros((0, _NCOL)))
            res, partner = _rank_step(P, st, halo)
            partners.update(zip(res[0].tolist(), partner.tolist()))
            crossed += int(np.sum(np.isin(partner, halo[0])))
            new.append(res)
        # migration
        moves = []
        for r, st in enumerate(new):
            idx, stay = decomp.migration_sends(_columns(P, st[1]), r, bounds)
            moves.append(([_rows(st[0][i], st[1][i], st[2][i], st[3][i]) for i in idx], stay))
        ranks = []
        migrated = 0
        for r, st in enumerate(new):
            keep = _rows(st[0], st[1], st[2], st[3])[moves[r][1]]
            got = [moves[q][0][r] for q in range(len(new)) if q != r]
            migrated += sum(len(g) for g in got)
            ranks.append(_sorted(_unrows(np.concatenate([keep] + got))))
        raw = sum(orc.moments(P, st[1], st[2], st[3])[0] for st in ranks)
        der = sum(orc.moments(P, st[1], st[2], st[3])[1] for st in ranks)
        glob = sum(orc.moments(P, st[1], st[2], st[3])[2] for st in ranks)
        out.append(dict(ranks=ranks, partners=partners, raw=raw, der=der, glob=glob,
                        crossed=crossed, migrated=migrated))
    return out


def _compare(ref, dec, n):
    """Bit-exact state, partners and per-c-bin moments; global sums to rounding."""
    for k, (a, b) in enumerate(zip(ref, dec)):
        ids = np.concatenate([st[0] for st in b["ranks"]])
        pos = np.concatenate([st[1] for st in b["ranks"]])
        vel = np.concatenate([st[2] for st in b["ranks"]])
        alive = np.flatnonzero(~np.isnan(a["pos"][:, 0]))
        assert np.array_equal(np.sort(ids), alive), f"step {k}: particle sets differ"
        o = np.argsort(ids)
        assert np.array_equal(pos[o], a["pos"][alive]), f"step {k}: positions differ"
        assert np.array_equal(vel[o], a["vel"][alive]), f"step {k}: velocities differ"
        got = np.array([b["partners"].get(i, -2) for i in range(n)])
        was_alive = np.array([i in b["partners"] for i in range(n)])
        assert np.array_equal(got[was_alive], a["paired"][was_alive]), f"step {k}: partners differ"
        assert np.array_equal(b["raw"], a["raw"]), f"step {k}: per-c-bin sums differ"
        assert np.array_equal(b["der"], a["der"]), f"step {k}: derived moments differ"
        np.testing.assert_allclose(b["glob"], a["glob"], rtol=1e-12, atol=1e-12)


@pytest.mark.parametrize("world", [2, 3, 4])
@pytest.mark.parametrize("name", ["slab_walls", "box_periodic", "plane_absorb"])
def test_decomposed_equals_undivided(name, world):
    params, ids, pos, vel, dt = _case(name)
    steps = 4
    ref = _undivided(params, pos, vel, steps, dt, adaptive=False)
    dec = _decomposed(params, ids, pos, vel, steps, dt, adaptive=False, world=world, weighted=(world == 3))
    _compare(ref, dec, len(ids))
    # the case exercises what the halo is for: pairs across slab faces, migration
    assert sum(d["crossed"] for d in dec) > 0
    assert sum(d["migrated"] for d in dec) > 0
    assert sum(r["npairs"] for r in ref) > 0


def test_decomposed_adaptive_dt_is_the_global_minimum():
    params, ids, pos, vel, dt = _case("slab_walls")
    ref = _undivided(params, pos, vel, 3, dt, adaptive=True)
    dec = _decomposed(params, ids, pos, vel, 3, dt, adaptive=True, world=3)
    _compare(ref, dec, len(ids))


def test_one_column_halo_is_not_enough():
    """A partner beside the slab face chooses among columns up to two away: a
    one-column halo changes some pair decisions."""
    params, ids, pos, vel, dt = _case("slab_walls")
    ref = _undivided(params, pos, vel, 1, dt, adaptive=False)
    dec = _decomposed(params, ids, pos, vel, 1, dt, adaptive=False, world=4, width=1)
    got = np.array([dec[0]["partners"][i] for i in range(len(ids))])
    assert np.any(got != ref[0]["paired"])


def test_slab_bounds_and_halo_columns():
    b = decomp.slab_bounds(10, 3)
    assert b.tolist() == [0, 3, 6, 10]
    w = np.array([8, 8, 8, 8, 1, 1, 1, 1, 1, 1], float)       # dense left, as in the Sod tube
    b = decomp.slab_bounds(10, 2, w)
    assert b.tolist() == [0, 2, 10]
    b = decomp.slab_bounds(4, 4, np.array([100, 0, 0, 0.0]))  # one column each, whatever the weights
    assert b.tolist() == [0, 1, 2, 3, 4]
    with pytest.raises(ValueError):
        decomp.slab_bounds(3, 4)
    b = np.array([0, 3, 6, 10])
    assert decomp.owner([0, 2, 3, 9, -1, 10], b).tolist() == [0, 0, 1, 2, -1, -1]
    assert decomp.halo_columns(0, b, periodic=False).tolist() == [3, 4]
    assert decomp.halo_columns(0, b, periodic=True).tolist() == [3, 4, 8, 9]
    assert decomp.halo_columns(1, b, periodic=False).tolist() == [1, 2, 6, 7]
    assert decomp.halo_columns(2, b, periodic=True).tolist() == [0, 1, 4, 5]
    # slabs narrower than the halo reach two ranks away
    b = np.array([0, 1, 2, 3, 4, 5])
    assert decomp.halo_columns(2, b, periodic=False).tolist() == [0, 1, 3, 4]
    sends = decomp.halo_sends(np.array([2, 2]), 2, b, periodic=False)
    assert [s.tolist() for s in sends] == [[0, 1], [0, 1], [], [0, 1], [0, 1]]
    idx, stay = decomp.migration_sends(np.array([2, 3, -1, 0]), 2, b)
    assert [s.tolist() for s in idx] == [[3], [], [], [1], []] and stay.tolist() == [True, False, False, False]


# ----------------------------------------------------------- two gloo ranks

def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _gloo_rank(rank, world, port, steps, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    import torch.distributed as dist
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        params, ids, pos, vel, dt_fixed = _case("slab_walls")
        P0 = params(0, dt_fixed)
        periodic = P0.bc[0] == 0
        bounds = decomp.slab_bounds(P0.n_cells[0], world)
        own = decomp.owner(_columns(P0, pos), bounds) == rank
        st = _sorted((ids[own], pos[own], vel[own], np.zeros(int(own.sum()))))
        partners = {}
        for k in range(steps):
            dt = decomp.allreduce_min(orc.adaptive_dt(params(k, 1.0), st[2], dt_rest=dt_fixed))
            P = params(k, dt)
            idx = decomp.halo_sends(_columns(P, st[1]), rank, bounds, periodic)
            got = decomp.exchange([_rows(st[0][i], st[1][i], st[2][i], st[3][i]) for i in idx])
            halo = _unrows(np.concatenate([g for q, g in enumerate(got) if q != rank]))
            st, partner = _rank_step(P, st, halo)
            partners.update({f"{k}:{i}": p for i, p in zip(st[0].tolist(), partner.tolist())})
            idx, stay = decomp.migration_sends(_columns(P, st[1]), rank, bounds)
            blocks = [_rows(st[0][i], st[1][i], st[2][i], st[3][i]) for i in idx]
            got = decomp.exchange(blocks)
            keep = _rows(*st)[stay]
            st = _sorted(_unrows(np.concatenate([keep] + [g for q, g in enumerate(got) if q != rank])))
        out[rank] = dict(ids=st[0], pos=st[1], vel=st[2], partners=partners)
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_equal_undivided():
    mp = pytest.importorskip("torch.multiprocessing")
    ctx = mp.get_context("spawn")
    port = _free_port()
    steps = 3
    with ctx.Manager() as m:
        out = m.dict()
        procs = [ctx.Process(target=_gloo_rank, args=(r, 2, port, steps, out)) for r in range(2)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(180)
        assert all(p.exitcode == 0 for p in procs), [p.exitcode for p in procs]
        res = [dict(out[r]) for r in range(2)]
    params, ids, pos, vel, dt = _case("slab_walls")
    ref = _undivided(params, pos, vel, steps, dt, adaptive=True)
    gids = np.concatenate([r["ids"] for r in res])
    o = np.argsort(gids)
    assert np.array_equal(gids[o], ids)
    assert np.array_equal(np.concatenate([r["pos"] for r in res])[o], ref[-1]["pos"])
    assert np.array_equal(np.concatenate([r["vel"] for r in res])[o], ref[-1]["vel"])
    for k in range(steps):
        got = np.array([res[0]["partners"].get(f"{k}:{i}", res[1]["partners"].get(f"{k}:{i}")) for i in ids])
        assert np.array_equal(got, ref[k]["paired"])


def _exchange_rank(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    import torch.distributed as dist
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        g = np.random.default_rng(rank)
        # block q of rank r has (r + 2 q) % 4 rows (some empty), tagged (r, q, row)
        blocks = []
        for q in range(world):
            m = (rank + 2 * q) % 4
            blocks.append(np.column_stack([np.full(m, rank), np.full(m, q), np.arange(m), g.random(m)]))
        got = decomp.exchange(blocks)
        out[rank] = dict(sent=[b.tolist() for b in blocks], got=[b.tolist() for b in got],
                         dtmin=decomp.allreduce_min(1.0 + rank))
    finally:
        dist.destroy_process_group()


def test_exchange_three_gloo_ranks_with_empty_blocks():
    """Every block arrives at its rank intact, empty blocks included, and the
    minimum reduces over all ranks."""
    mp = pytest.importorskip("torch.multiprocessing")
    ctx = mp.get_context("spawn")
    port = _free_port()
    world = 3
    with ctx.Manager() as m:
        out = m.dict()
        procs = [ctx.Process(target=_exchange_rank, args=(r, world, port, out)) for r in range(world)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(120)
        assert all(p.exitcode == 0 for p in procs), [p.exitcode for p in procs]
        res = [dict(out[r]) for r in range(world)]
    for r in range(world):
        assert res[r]["dtmin"] == 1.0
        for q in range(world):
            assert res[r]["got"][q] == res[q]["sent"][r]


def _failing_rank(rank, world, port, out):
    import datetime
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    import torch.distributed as dist
    dist.init_process_group("gloo", rank=rank, world_size=world, timeout=datetime.timedelta(seconds=10))
    if rank == 1:
        os._exit(3)   # dies between steps, before the halo exchange
    import time
    t0 = time.time()
    try:
        decomp.exchange([np.zeros((2, 4)), np.ones((3, 4))])
        out[rank] = dict(error=None, seconds=time.time() - t0)
    except Exception as e:   # the collective fails instead of waiting forever
        out[rank] = dict(error=type(e).__name__, seconds=time.time() - t0)


def test_exchange_reports_a_dead_rank():
    """A rank that dies between steps: the survivor's next exchange raises
    (peer gone or process-group timeout) instead of hanging."""
    mp = pytest.importorskip("torch.multiprocessing")
    ctx = mp.get_context("spawn")
    port = _free_port()
    with ctx.Manager() as m:
        out = m.dict()
        procs = [ctx.Process(target=_failing_rank, args=(r, 2, port, out)) for r in range(2)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(120)
        for p in procs:
            if p.is_alive():
                p.kill()
        assert procs[1].exitcode == 3
        res = dict(out[0])
    assert res["error"] is not None and res["seconds"] < 60, res
