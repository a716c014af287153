"""Per-c-bin moments, the sort permutation, batched instances and the bounded
device wait, through the C ABI against the CPU oracle.

Moments (Sect. "Numerical studies in the hydrodynamic limit", Eqs. vel_b,
stress, 18, 19): the device sums every particle's contribution in 64-bit fixed
point (a grid of 2^-e with e chosen from the instance's largest speed, so that
no sum over the instance's n particles can reach 2^62); the oracle sums in
binary64.  Bounds used below, per c-bin b with N_b particles:
  * counts: exact;
  * Sum v:   N_b n v_max 2^-61 (fixed-point rounding, twice the worst case)
             + 2^-50 Sum |v| (the oracle's own binary64 summation);
  * Sum v^2: N_b n v_max^2 2^-61 + 2^-50 Sum v^2, plus 2^-23 Sum v^2 on the
             binary32 path (the device squares in binary32);
  * Sum W (collisional virial, Eq. stress): the device evaluates r_ij(t_poca)
    . dp_i in the state precision from the same state; its error is a few
    units of rounding of the separation times |dp| and of dp times the
    separation, bounded here by 1e-6 (binary32) or 1e-13 (binary64) x reach x
    Sum (|v' - v| + |v| + |v'|) over the bin's collided particles, reach =
    R + 2 v_max dt.
"""
import math

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

WALL, PER = 1, 0


def _setup():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__ as g
    g.build()


def _oracle_R2(lam, n, dim, lo, hi):
    import oracle
    V = float(np.prod([hi[d] - lo[d] for d in range(dim)]))
    return oracle.contact_R2(lam, 0.0, n / V)


GEOMS = {
    # name: n, dim, n_cells, lo, hi, bc, lam, dt, kind
    "slab": (60_000, 3, (60, 1, 1), (0, 0, 0), (1, 1, 1), (WALL, PER, PER), 1e-3, 0.2 / 60, "sod"),
    "cubic": (40_000, 3, (20, 6, 6), (0, 0, 0), (1, 0.3, 0.3), (WALL, PER, PER), 1e-3, 0.01, "sod"),
    "plane2d": (100_000, 2, (40, 40, 1), (0, 0, 0), (1, 1, 1), (WALL, WALL, PER), 5e-4, 0.005, "quad"),
}


def _state(geom, prec, seed=7):
    from paper_1210_8084_gb300 import inputs
    n, dim, n_cells, lo, hi, bc, lam, dt, kind = GEOMS[geom]
    if kind == "quad":
        pos, vel = inputs.quadrants_2d(n, seed=seed)
        vel[:, 0] += 0.3   # a bulk flow, so that the bulk velocity is not only noise
    else:
        pos, vel = inputs.sod_tube(n, seed=seed, lo=lo, hi=hi)
        vel[:, 1] -= 0.2
    if prec == 32:
        pos, vel = inputs.cast_state(pos, vel, np.float32, lo, hi, bc)
    return pos.astype(np.float64), vel.astype(np.float64)


def _params(geom, prec, step=0, seed=5):
    import oracle
    n, dim, n_cells, lo, hi, bc, lam, dt, kind = GEOMS[geom]
    return oracle.make_params(dim, n_cells, lo, hi, bc, R2=_oracle_R2(lam, n, dim, lo, hi), dt=dt, seed=seed,
                              step=step, decide32=prec == 32)


def _config(k, geom, prec, seed=5, flags=0):
    n, dim, n_cells, lo, hi, bc, lam, dt, kind = GEOMS[geom]
    return k.make_config(dim_pos=dim, n_cells=n_cells, lo=lo, hi=hi, bc=bc, lam=lam, dt=dt, seed=seed,
                         precision=prec, flags=flags)


def _bin_sum(P, pos, vel, x):
    """Per-c-bin sum of a per-particle quantity x, binned by the oracle."""
    import oracle
    return oracle.moments(P, pos, vel, np.ascontiguousarray(x, dtype=np.float64))[0][:, 7]


def _check_raw(raw_d, raw_o, P, pos, vel, prec, n):
    """Counts exact; Sum v and Sum v^2 within the fixed-point and summation bounds."""
    assert np.array_equal(raw_d[:, 0], raw_o[:, 0]), "particle counts per c-bin"
    N = raw_o[:, 0]
    vmax = np.linalg.norm(vel, axis=1).max() * (1 + 1e-6)
    abs_v = _bin_sum(P, pos, vel, np.abs(vel).sum(1))
    sq = _bin_sum(P, pos, vel, (vel * vel).sum(1))
    tol_v = N * n * vmax * 2.0 ** -61 + 2.0 ** -50 * abs_v
    tol_2 = N * n * vmax * vmax * 2.0 ** -61 + 2.0 ** -50 * sq + (2.0 ** -23 * sq if prec == 32 else 0.0)
    for d in range(3):
        err = np.abs(raw_d[:, 1 + d] - raw_o[:, 1 + d])
        assert np.all(err <= tol_v), ("Sum v", d, (err / np.maximum(tol_v, 1e-300)).max())
        err = np.abs(raw_d[:, 4 + d] - raw_o[:, 4 + d])
        assert np.all(err <= tol_2), ("Sum v^2", d, (err / np.maximum(tol_2, 1e-300)).max())
    return tol_v, tol_2


def _check_derived(der_d, der_o, raw_o, tol_v, tol_2, tol_w, Vc, dim, dt):
    """n, u, T, p_kin, p_vir, p from the raw bounds (first-order propagation, x2)."""
    N = raw_o[:, 0]
    ok = N > 0
    assert np.array_equal(der_d[~ok], der_o[~ok])
    N = N[ok]
    dd, do = der_d[ok], der_o[ok]
    assert np.allclose(dd[:, 0], do[:, 0], rtol=1e-15, atol=0), "n"
    tu = 2 * tol_v[ok] / N + 1e-15 * np.abs(do[:, 1:4]).max()
    for d in range(3):
        assert np.all(np.abs(dd[:, 1 + d] - do[:, 1 + d]) <= tu), ("u", d)
    u = np.abs(do[:, 1:4]).sum(1)
    tT = 2 * (tol_2[ok] / N + 2 * u * tol_v[ok] / N) / 3 + 1e-14 * do[:, 4]
    assert np.all(np.abs(dd[:, 4] - do[:, 4]) <= tT), "T"
    tp = tT * do[:, 0] + 1e-14 * do[:, 5]
    assert np.all(np.abs(dd[:, 5] - do[:, 5]) <= tp), "p_kin"
    tv = 2 * tol_w[ok] / (2 * dim * Vc * dt) + 1e-14 * np.abs(do[:, 6])
    assert np.all(np.abs(dd[:, 6] - do[:, 6]) <= tv), "p_vir"
    assert np.all(np.abs(dd[:, 7] - do[:, 7]) <= tp + tv + 1e-14 * np.abs(do[:, 7])), "p"


@pytest.mark.parametrize("prec", [32, 64])
@pytest.mark.parametrize("geom", list(GEOMS))
def test_moments_of_a_set_state_match_oracle(geom, prec):
    """kmc_moments of a state just set (no step): per c-bin counts, sums and
    the derived n, u, T, p_kin against the oracle's moments of the same state
    (zero virial)."""
    _setup()
    import oracle
    import paper_1210_8084_gb300 as k
    pos, vel = _state(geom, prec)
    n, dim, n_cells, lo, hi, bc, lam, dt, kind = GEOMS[geom]
    sim = k.Simulation(_config(k, geom, prec), pos, vel)
    raw, der, glob = sim.moments()
    sim.close()
    P = _params(geom, prec)
    raw_o, der_o, glob_o = oracle.moments(P, pos, vel, None)
    tol_v, tol_2 = _check_raw(raw, raw_o, P, pos, vel, prec, n)
    assert np.all(raw[:, 7] == 0) and np.all(der[:, 6] == 0)
    Vc = float(np.prod([(hi[d] - lo[d]) / n_cells[d] for d in range(dim)]))
    _check_derived(der, der_o, raw_o, tol_v, tol_2, np.zeros(len(raw_o)), Vc, dim, dt)
    assert glob[0, 0] == n
    assert abs(glob[0, 1] - glob_o[1]) <= (1e-6 if prec == 32 else 1e-12) * glob_o[1]


@pytest.mark.parametrize("prec", [32, 64])
@pytest.mark.parametrize("geom", list(GEOMS))
def test_moments_after_one_step_match_oracle(geom, prec):
    """One step from the same state (pairs bit-exact), then the moments of the
    end state, virial included, c-bin by c-bin.  (a) The reduction: the oracle's
    moments of the device's end state with the oracle's per-particle virial
    (the pairs are the same particles) within the stated bounds.  (b) End to
    end: against the oracle's own end state, on the c-bins whose members agree,
    with the bounds widened by the state differences Sum |v_dev - v_orc|."""
    _setup()
    import oracle
    import paper_1210_8084_gb300 as k
    pos, vel = _state(geom, prec)
    n, dim, n_cells, lo, hi, bc, lam, dt, kind = GEOMS[geom]
    sim = k.Simulation(_config(k, geom, prec, flags=k.KMC_FLAG_RECORD), pos, vel)
    sim.step(1, want_moments=1)
    best, partner = sim.partners()
    p_d, v_d = sim.state()
    raw, der, glob = sim.moments()
    sim.close()
    p_d, v_d = p_d.astype(np.float64), v_d.astype(np.float64)
    P = _params(geom, prec)
    ob = oracle.best_partners(P, pos, vel)
    po, vo, W, paired = oracle.collide_move(P, pos, vel, ob)
    assert np.array_equal(partner, paired)
    coll = paired >= 0
    assert coll.sum() > n // 20
    Vc = float(np.prod([(hi[d] - lo[d]) / n_cells[d] for d in range(dim)]))
    reach = math.sqrt(P.R2) + 2 * np.linalg.norm(vel, axis=1).max() * dt
    # scale of a collided particle's W: its velocity change and both speeds (the
    # rounding of v' is relative to the speeds, that of r_ij(t_poca) to the reach)
    dvel = np.where(coll, np.linalg.norm(vo - vel, axis=1) + np.linalg.norm(vo, axis=1)
                    + np.linalg.norm(vel, axis=1), 0.0)
    rel_w = 1e-6 if prec == 32 else 1e-13

    # (a) the reduction on the device's own end state
    raw_a, der_a, _ = oracle.moments(P, p_d, v_d, W)
    tol_v, tol_2 = _check_raw(raw, raw_a, P, p_d, v_d, prec, n)
    tol_w = rel_w * reach * _bin_sum(P, p_d, v_d, dvel) + 2.0 ** -50 * _bin_sum(P, p_d, v_d, np.abs(W))
    err_w = np.abs(raw[:, 7] - raw_a[:, 7])
    assert np.all(err_w <= tol_w), (err_w / np.maximum(tol_w, 1e-300)).max()
    assert np.abs(raw_a[:, 7]).max() > 0
    _check_derived(der, der_a, raw_a, tol_v, tol_2, tol_w, Vc, dim, dt)

    # (b) against the oracle's end state
    raw_o, der_o, glob_o = oracle.moments(P, po, vo, W)
    kd, _ = oracle.cell_keys(P, p_d)
    ko, _ = oracle.cell_keys(P, po)
    moved = kd != ko
    if prec == 64:
        assert not moved.any()
    assert moved.sum() <= 10
    bad = np.zeros(len(raw_o), bool)
    bad[kd[moved]] = True
    bad[ko[moved]] = True
    good = ~bad
    assert np.array_equal(raw[good, 0], raw_o[good, 0])
    dv_abs = _bin_sum(P, po, vo, np.abs(v_d - vo).sum(1))
    dv_sq = _bin_sum(P, po, vo, (np.abs(v_d - vo) * np.abs(v_d + vo)).sum(1))
    for d in range(3):
        assert np.all(np.abs(raw[good, 1 + d] - raw_o[good, 1 + d]) <= (tol_v + dv_abs)[good]), d
        assert np.all(np.abs(raw[good, 4 + d] - raw_o[good, 4 + d]) <= (tol_2 + dv_sq)[good]), d
    assert np.all(np.abs(raw[good, 7] - raw_o[good, 7]) <= tol_w[good])
    assert glob[0, 6] == coll.sum() / 2


def test_moments_are_bit_reproducible():
    """Two runs of the same configuration give the same moment bits (the sums
    do not depend on the order of atomics), binary32 state."""
    _setup()
    import paper_1210_8084_gb300 as k
    pos, vel = _state("slab", 32)
    outs = []
    for _ in range(2):
        sim = k.Simulation(_config(k, "slab", 32), pos, vel)
        sim.step(4, want_moments=1)
        outs.append(sim.moments())
        sim.close()
    for a, b in zip(*outs):
        assert np.array_equal(a, b)


PERM_CASES = [
    # name, geom, sub_cells, prec
    ("cubic_tile_fp32", "cubic", (1, 1, 1), 32),
    ("slab_subdivided_fp32", "slab", (0, 0, 0), 32),
    ("slab_plain_fp64", "slab", (1, 1, 1), 64),
    ("plane2d_fp32", "plane2d", (1, 1, 1), 32),
    ("plane2d_subdivided_fp64", "plane2d", (2, 3, 1), 64),
]


@pytest.mark.parametrize("case", PERM_CASES, ids=[c[0] for c in PERM_CASES])
def test_sort_permutation_is_canonical(case):
    """kmc_get_perm (Sect. "Simulation setup": particles sorted into bins every
    step).  The result is a permutation of 0..n-1; its c-bins (the oracle's
    keys) are grouped; inside every search cell the ids increase.  With search
    cells equal to the c-bins the permutation is unique -- c-bins in search
    order (x slowest), ids increasing -- and is compared with the one built
    from the oracle's keys, bit for bit, at the start and after steps."""
    _setup()
    import oracle
    import paper_1210_8084_gb300 as k
    name, geom, sub, prec = case
    n, dim, n_cells, lo, hi, bc, lam, dt, kind = GEOMS[geom]
    pos, vel = _state(geom, prec)
    cfg = _config(k, geom, prec)
    for d in range(3):
        cfg.sub_cells[d] = sub[d]
    sim = k.Simulation(cfg, pos, vel)
    info = sim.info()
    s = list(info.sub_cells)
    for step in range(3):
        perm = sim.perm()
        p, v = sim.state()
        assert np.array_equal(np.sort(perm), np.arange(n))
        P = _params(geom, prec)
        key, cidx = oracle.cell_keys(P, p.astype(np.float64))
        # search order of a c-bin: x slowest, the last position dimension fastest
        if dim == 3:
            corder = (cidx[:, 0] * n_cells[1] + cidx[:, 1]) * n_cells[2] + cidx[:, 2]
        else:
            corder = cidx[:, 0] * n_cells[1] + cidx[:, 1]
        if s == [1, 1, 1]:
            expect = np.lexsort((np.arange(n), corder))
            assert np.array_equal(perm, expect), step
        else:
            # sub-cells of a c-bin: the position's fraction of its c-bin, as the
            # search key takes it (x - lo) n / (hi - lo) in the state precision
            ft = np.float32 if prec == 32 else np.float64
            sc = np.zeros((n, 3), np.int64)
            for d in range(dim):
                t = (p[:, d].astype(ft) - ft(lo[d])) * ft(n_cells[d] / (hi[d] - lo[d]))
                c = np.clip(np.floor(t), 0, n_cells[d] - 1)
                fs = (t - c.astype(ft)) * ft(s[d])
                sc[:, d] = np.clip(np.floor(fs), 0, s[d] - 1).astype(np.int64)
                assert np.array_equal(c.astype(np.int64), cidx[:, d])
            g = [cidx[:, d] * s[d] + sc[:, d] for d in range(3)]
            M = [n_cells[d] * s[d] for d in range(3)]
            skey = (g[0] * M[1] + g[1]) * (M[2] if dim == 3 else 1) + (g[2] if dim == 3 else 0)
            expect = np.lexsort((np.arange(n), skey))
            assert np.array_equal(perm, expect), step
        sim.step(1)
    sim.close()


def test_batched_instance_matches_oracle():
    """An instance inside a batched run (instance-offset keys, one launch for
    all) against the oracle run on that instance alone: keys, closest
    candidates and pairs bit for bit, velocities to binary32 rounding, and
    per-c-bin moments within the bounds above."""
    _setup()
    import oracle
    import paper_1210_8084_gb300 as k
    from paper_1210_8084_gb300 import inputs
    ns = [9_000, 31_000, 4_500]
    lams = [1e-2, 1e-3, 1e-4]
    n_cells, lo, hi, bc, dt = (30, 1, 1), (0, 0, 0), (1, 1, 1), (WALL, PER, PER), 0.2 / 30
    P_, V_, insts = [], [], []
    for i, (n, lam) in enumerate(zip(ns, lams)):
        p, v = inputs.cast_state(*inputs.sod_tube(n, seed=300 + i), np.float32, lo, hi, bc)
        P_.append(p.astype(np.float64))
        V_.append(v.astype(np.float64))
        insts.append(dict(n=n, lam=lam, dt=dt, seed=40 + i))
    cfg = k.make_config(dim_pos=3, n_cells=n_cells, lo=lo, hi=hi, bc=bc, precision=32, instances=insts,
                        flags=k.KMC_FLAG_RECORD)
    sim = k.Simulation(cfg, np.concatenate(P_), np.concatenate(V_))
    keys = sim.cell_keys()
    sim.step(1, want_moments=1)
    best, partner = sim.partners()
    p1, v1 = sim.state()
    raw, der, glob = sim.moments()
    sim.close()
    i = 1
    off, n = ns[0], ns[1]
    P = oracle.make_params(3, n_cells, lo, hi, bc, R2=_oracle_R2(lams[i], n, 3, lo, hi), dt=dt, seed=40 + i, step=0,
                           decide32=True)
    ko, _ = oracle.cell_keys(P, P_[i])
    ob = oracle.best_partners(P, P_[i], V_[i])
    po, vo, W, paired = oracle.collide_move(P, P_[i], V_[i], ob)
    assert np.array_equal(keys[off:off + n], ko)
    assert np.array_equal(best[off:off + n], ob)
    assert np.array_equal(partner[off:off + n], paired)
    assert (paired >= 0).sum() > n // 20
    s0 = np.linalg.norm(V_[i], axis=1)
    scale = np.maximum(np.linalg.norm(vo, axis=1), np.where(paired >= 0, np.maximum(s0, s0[np.maximum(paired, 0)]), 0))
    assert (np.abs(v1[off:off + n] - vo).max(1) <= 1e-5 * np.maximum(scale, 1e-30)).all()
    rows = slice(n_cells[0] * i, n_cells[0] * (i + 1))
    raw_a, der_a, _ = oracle.moments(P, p1[off:off + n].astype(np.float64), v1[off:off + n].astype(np.float64), W)
    _check_raw(raw[rows], raw_a, P, p1[off:off + n].astype(np.float64), v1[off:off + n].astype(np.float64), 32, n)
    assert glob[i, 6] == (paired >= 0).sum() / 2


def test_bounded_scan_wait_times_out_and_recovers():
    """Failure detection without a GPU fault (the only device-side wait of a
    step is the key scan's look-back, bounded by a poll cap).  A test hook makes
    scan tile 1 withhold its status and lowers the cap to 64 polls: the tiles
    after it give up, the step ends, and kmc_sync reports KMC_ETIMEOUT instead
    of hanging.  Restoring the state clears the hold; the handle then steps
    exactly as a fresh one does."""
    _setup()
    import paper_1210_8084_gb300 as k
    pos, vel = _state("slab", 32)
    cfg = _config(k, "slab", 32)
    for d, s in enumerate((1, 40, 40)):   # 96,000 search cells: many scan tiles
        cfg.sub_cells[d] = s
    sim = k.Simulation(cfg, pos, vel)
    info = sim.info()
    assert info.n_scan_tiles >= 3
    p0, v0 = sim.state()
    k.kmc_test_hold_scan(sim.h, 1, 64)
    sim.step(1, want_moments=1)
    with pytest.raises(k.KmcError) as e:
        sim.sync()
    assert e.value.code == k.KMC_ETIMEOUT
    sim.set_state(p0, v0, step=0)
    sim.step(2, want_moments=1)
    p_a, v_a = sim.state()
    raw_a = sim.moments()[0]
    sim.close()
    ref = k.Simulation(cfg, pos, vel)
    ref.step(2, want_moments=1)
    p_b, v_b = ref.state()
    raw_b = ref.moments()[0]
    ref.close()
    assert np.array_equal(p_a, p_b) and np.array_equal(v_a, v_b)
    assert np.array_equal(raw_a, raw_b)


@pytest.mark.parametrize("prec", [32, 64])
@pytest.mark.parametrize("dim", [2, 3])
def test_radial_velocity_matches_oracle(prec, dim):
    """KMC_MOM_RADIAL (Eq. vel_r) after one step of a Noh inflow, about the
    corner the gas falls towards and about an off-corner centre: per c-bin
    Sum v . r_hat within the fixed-point bound plus the rounding of r_hat in the
    state precision (2^-20 or 2^-48 of Sum |v|), and v_r = Sum / N."""
    _setup()
    import oracle
    import paper_1210_8084_gb300 as k
    from paper_1210_8084_gb300 import inputs
    n, nc = 40_000, (16, 16, 16) if dim == 3 else (40, 40, 1)
    lo, hi, bc = (0, 0, 0), (1, 1, 1), (WALL, WALL, WALL)
    pos, vel = inputs.noh(n, seed=9, dim_pos=dim, v0=1.0, T0=0.01)
    if prec == 32:
        pos, vel = inputs.cast_state(pos, vel, np.float32, lo, hi, bc)
    pos, vel = pos.astype(np.float64), vel.astype(np.float64)
    for center in ((0.0, 0.0, 0.0), (0.3, 0.45, 0.55)):
        cfg = k.make_config(dim_pos=dim, n_cells=nc, lo=lo, hi=hi, bc=bc, lam=1e-3, dt=0.01, seed=2, precision=prec,
                            radial_center=center, flags=k.KMC_FLAG_RADIAL_MOMENT)
        sim = k.Simulation(cfg, pos, vel)
        sim.step(1, want_moments=1)
        p1, v1 = sim.state()
        rad = sim.radial()
        raw = sim.moments()[0]
        sim.close()
        p1, v1 = p1.astype(np.float64), v1.astype(np.float64)
        P = oracle.make_params(dim, nc, lo, hi, bc, R2=_oracle_R2(1e-3, n, dim, lo, hi), dt=0.01, seed=2,
                               decide32=prec == 32)
        ro = oracle.radial(P, p1, v1, center)
        N = raw[:, 0]
        vmax = np.linalg.norm(v1, axis=1).max() * (1 + 1e-6)
        abs_v = _bin_sum(P, p1, v1, np.linalg.norm(v1, axis=1))
        tol = N * n * vmax * 2.0 ** -61 + (2.0 ** -20 if prec == 32 else 2.0 ** -48) * abs_v
        assert np.all(np.abs(rad[:, 0] - ro[:, 0]) <= tol), center
        ok = N > 0
        assert np.all(np.abs(rad[ok, 1] - ro[ok, 1]) <= tol[ok] / N[ok] + 1e-15)
        assert np.all(rad[~ok] == 0)
        if center[0] == 0.0:
            # the cold inflow towards the corner: v_r close to -v0 away from the corner
            assert np.median(rad[ok, 1]) < -0.8
