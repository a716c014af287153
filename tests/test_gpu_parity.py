"""Parity of the CUDA path (through the C ABI) with the CPU oracle.

Integer results (cell keys, closest candidates, pairs) must match bit for
bit: in binary64 against the binary64 oracle, in binary32 against the
oracle's binary32 decision mode.  Post-collision velocities must agree to
1e-5 relative (binary32 state vs binary64 oracle) or 1e-12 (binary64 state),
positions to the corresponding rounding.  Every case starts from the same
seeded state on both sides.
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


def run_gpu_step(pos, vel, dim, n_cells, lo, hi, bc, lam, dt, seed, precision, step=0, sub_cells=(0, 0, 0),
                 nsteps=1, staged=False, occ=0.0, per_particle=False):
    import paper_1210_8084_gb300 as k
    flags = k.KMC_FLAG_RECORD | (k.KMC_FLAG_STAGED_SEARCH if staged else 0) | \
        (k.KMC_FLAG_NO_TILE_SEARCH if per_particle else 0)
    cfg = k.make_config(dim_pos=dim, n_cells=n_cells, lo=lo, hi=hi, bc=bc, lam=lam, dt=dt, seed=seed,
                        precision=precision, flags=flags, sub_cells=sub_cells, occupancy_target=occ)
    sim = k.Simulation(cfg, pos, vel)
    if step:
        p0, v0 = sim.state()
        sim.set_state(p0, v0, step=step)
    info = sim.info()
    keys = sim.cell_keys()
    sim.step(nsteps, want_moments=1)
    best, partner = sim.partners()
    p, v = sim.state()
    raw, der, glob = sim.moments()
    sim.close()
    return dict(info=info, keys=keys, best=best, partner=partner, pos=p, vel=v, raw=raw, der=der, glob=glob)


def oracle_R2(lam, n, dim, lo, hi, sigma=0.0):
    """The oracle's squared contact distance for n particles in the box (Eq. 7,
    Eq. reff_lambda with n = N / V over the position dimensions): computed on
    the oracle side, never taken from the device."""
    import oracle
    V = float(np.prod([hi[d] - lo[d] for d in range(dim)]))
    return oracle.contact_R2(lam, sigma, n / V)


def oracle_step(pos, vel, dim, n_cells, lo, hi, bc, R2, dt, seed, step, decide32):
    import oracle
    P = oracle.make_params(dim, n_cells, lo, hi, bc, R2=R2, dt=dt, seed=seed, step=step, decide32=decide32)
    key, _ = oracle.cell_keys(P, pos)
    best = oracle.best_partners(P, pos, vel)
    po, vo, W, paired = oracle.collide_move(P, pos, vel, best)
    raw, der, glob = oracle.moments(P, po, vo, W)
    return dict(P=P, keys=key, best=best, partner=paired, pos=po, vel=vo, W=W, raw=raw, der=der, glob=glob)


def compare_step(g, o, precision, pos0, vel0, dim):
    assert np.array_equal(g["keys"], o["keys"]), "cell keys"
    nb = (g["best"] != o["best"]).sum()
    assert nb == 0, f"{nb} closest candidates differ"
    assert np.array_equal(g["partner"], o["partner"]), "pairs"
    # post-collision velocities v_cm +- (g/2) n_hat are rounded at the scale of
    # the pair's incoming speeds: the error is relative to the largest of the
    # particle's outgoing speed and both incoming speeds; unpaired particles
    # keep their velocity exactly
    tol_v = 1e-12 if precision == 64 else 1e-5
    partner = np.asarray(o["partner"])
    paired = partner >= 0
    s0 = np.linalg.norm(vel0, axis=1)
    scale = np.linalg.norm(o["vel"], axis=1)
    scale[paired] = np.maximum(scale[paired], np.maximum(s0[paired], s0[partner[paired]]))
    err = np.abs(g["vel"] - o["vel"]).max(1)
    assert np.all(err[~paired] == 0), "unpaired velocities must be unchanged"
    dv = err[paired] / np.maximum(scale[paired], 1e-300)
    assert dv.size == 0 or dv.max() <= tol_v, f"velocity rel err {dv.max()}"
    tol_x = 1e-12 if precision == 64 else 4e-6
    assert np.abs(g["pos"][:, :dim] - o["pos"][:, :dim]).max() <= tol_x * max(1.0, np.abs(pos0).max())
    # moments: counts exact when every end position is binned the same way
    same_bins = np.array_equal(g["raw"][:, 0], o["raw"][:, 0])
    if precision == 64:
        assert same_bins
    rel = 1e-10 if precision == 64 else 1e-5
    e_g, e_o = g["glob"][0, 1], o["glob"][1]
    assert abs(e_g - e_o) <= rel * e_o
    assert g["glob"][0, 6] == len(np.nonzero(o["partner"] >= 0)[0]) / 2


CASES = [
    # name, n, dim, n_cells, lo, hi, bc, lam, dt, precision
    ("sod1d_fp64_200k", 200_000, 3, (200, 1, 1), (0, 0, 0), (1, 1, 1), (WALL, PER, PER), 1e-3, 1e-3, 64),
    ("sod1d_fp32_1M_k1e-3", 1_000_000, 3, (500, 1, 1), (0, 0, 0), (1, 1, 1), (WALL, PER, PER), 1e-3, 4e-4, 32),
    ("sod1d_fp32_1M_k1e-4", 1_000_000, 3, (500, 1, 1), (0, 0, 0), (1, 1, 1), (WALL, PER, PER), 1e-4, 4e-4, 32),
    ("sod1d_fp32_1M_k1", 1_000_000, 3, (500, 1, 1), (0, 0, 0), (1, 1, 1), (WALL, PER, PER), 1.0, 4e-4, 32),
    ("quad2d_fp32_300k", 300_000, 2, (96, 96, 1), (0, 0, 0), (1, 1, 1), (WALL, WALL, PER), 5e-4, 0.2 / 96, 32),
    ("sod3d_fp32_400k", 400_000, 3, (128, 8, 8), (0, 0, 0), (1, 1 / 16, 1 / 16), (WALL, PER, PER), 2e-4,
     0.2 / 128, 32),
    ("box3d_fp64_ragged", 12_345, 3, (5, 4, 3), (-1, 0, 2), (1, 0.5, 3), (PER, WALL, PER), 1e-2, 5e-3, 64),
    ("box2d_fp32_periodic_2cells", 3_001, 2, (2, 2, 1), (0, 0, 0), (1, 1, 1), (PER, PER, PER), 1e-2, 5e-3, 32),
    ("noh3d_fp32_walls", 60_000, 3, (16, 16, 16), (0, 0, 0), (1, 1, 1), (WALL, WALL, WALL), 1e-3, 0.02, 32),
]


def f32_state(pos, vel, lo, hi, bc):
    """The binary32 state both sides start from, held in float64."""
    from paper_1210_8084_gb300 import inputs
    p, v = inputs.cast_state(pos, vel, np.float32, lo, hi, bc)
    return p.astype(np.float64), v.astype(np.float64)


def make_inputs(name, n, dim, lo, hi):
    from paper_1210_8084_gb300 import inputs
    if name.startswith("quad"):
        return inputs.quadrants_2d(n, seed=3)
    if name.startswith("noh"):
        return inputs.noh(n, seed=3, dim_pos=dim, L=hi[0], v0=1.0, T0=0.01)
    if name.startswith("sod"):
        return inputs.sod_tube(n, seed=3, lo=lo, hi=hi)
    pos, vel = inputs.periodic_box(n, seed=3, lo=lo, hi=hi)
    if dim == 2:
        pos[:, 2] = 0.0
    return pos, vel


@pytest.mark.parametrize("mode", ["default", "per_particle", "staged"])
@pytest.mark.parametrize("case", CASES, ids=[c[0] for c in CASES])
def test_one_step_parity(case, mode):
    """One step from the same state.  default: one block per c-bin where the
    search grid is not subdivided, per-thread search elsewhere; per_particle:
    per-thread search everywhere; staged: shared-memory staged tiles (3-D
    subdivided grids where they fit).  All must match the oracle."""
    _setup()
    name, n, dim, n_cells, lo, hi, bc, lam, dt, prec = case
    pos, vel = make_inputs(name, n, dim, lo, hi)
    if prec == 32:
        pos, vel = f32_state(pos, vel, lo, hi, bc)
    seed = 11
    g = run_gpu_step(pos, vel, dim, n_cells, lo, hi, bc, lam, dt, seed, prec, staged=mode == "staged",
                     per_particle=mode == "per_particle")
    o = oracle_step(pos, vel, dim, n_cells, lo, hi, bc, oracle_R2(lam, n, dim, lo, hi), dt, seed, 0, prec == 32)
    assert (g["best"] >= 0).mean() > 0.02 or lam >= 1.0
    compare_step(g, o, prec, pos, vel, dim)


def test_contact_distance_matches_oracle_bitwise():
    _setup()
    import oracle
    pos, vel = make_inputs("sod", 5000, 3, (0, 0, 0), (1, 1, 1))
    for lam in (1e-4, 1e-3, 0.37, 1.0):
        g = run_gpu_step(pos, vel, 3, (10, 1, 1), (0, 0, 0), (1, 1, 1), (WALL, PER, PER), lam, 1e-3, 0, 64, nsteps=0)
        assert g["info"].R2 == oracle.contact_R2(lam, 0.0, 5000.0)


@pytest.mark.parametrize("sub", [(1, 1, 1), (1, 3, 2), (1, 9, 9), (1, 40, 40), (0, 0, 0)])
def test_search_grid_subdivision_does_not_change_results(sub):
    """Any subdivision of the c-bins into search cells returns the same
    closest candidates as the plain 3^D neighbourhood (the window adapts)."""
    _setup()
    pos, vel = make_inputs("sod", 60_000, 3, (0, 0, 0), (1, 1, 1))
    pos, vel = f32_state(pos, vel, (0, 0, 0), (1, 1, 1), (WALL, PER, PER))
    args = (3, (40, 1, 1), (0, 0, 0), (1, 1, 1), (WALL, PER, PER), 1e-3, 1e-3, 5)
    g = run_gpu_step(pos, vel, *args, precision=32, sub_cells=sub)
    R2 = oracle_R2(1e-3, len(pos), 3, (0, 0, 0), (1, 1, 1))
    o = oracle_step(pos, vel, 3, (40, 1, 1), (0, 0, 0), (1, 1, 1), (WALL, PER, PER), R2, 1e-3, 5, 0, True)
    assert np.array_equal(g["best"], o["best"])
    assert np.array_equal(g["partner"], o["partner"])


def test_multi_step_each_step_from_device_state():
    """Five steps: every device step equals the oracle step taken from the
    device's own state at that point (binary64 integers bit-exact)."""
    _setup()
    import paper_1210_8084_gb300 as k
    import oracle
    pos, vel = make_inputs("sod", 50_000, 3, (0, 0, 0), (1, 1, 1))
    cfg = k.make_config(dim_pos=3, n_cells=(50, 1, 1), bc=(WALL, PER, PER), lam=1e-3, dt=4e-3, seed=21,
                        precision=64, flags=k.KMC_FLAG_RECORD)
    sim = k.Simulation(cfg, pos, vel)
    R2 = oracle_R2(1e-3, len(pos), 3, (0, 0, 0), (1, 1, 1))
    for s in range(5):
        p0, v0 = sim.state()
        sim.step(1)
        best, partner = sim.partners()
        p1, v1 = sim.state()
        P = oracle.make_params(3, (50, 1, 1), (0, 0, 0), (1, 1, 1), (WALL, PER, PER), R2=R2, dt=4e-3, seed=21, step=s)
        bo = oracle.best_partners(P, p0, v0)
        po, vo, W, paired = oracle.collide_move(P, p0, v0, bo)
        assert np.array_equal(best, bo) and np.array_equal(partner, paired), f"step {s}"
        assert np.abs(v1 - vo).max() <= 1e-12 * np.abs(v0).max()
        assert sim.info().step == s + 1
    sim.close()


def test_checkpoint_resume_is_bit_identical():
    _setup()
    import paper_1210_8084_gb300 as k
    pos, vel = make_inputs("sod", 100_000, 3, (0, 0, 0), (1, 1, 1))
    pos, vel = f32_state(pos, vel, (0, 0, 0), (1, 1, 1), (WALL, PER, PER))
    cfg = k.make_config(dim_pos=3, n_cells=(100, 1, 1), bc=(WALL, PER, PER), lam=1e-3, dt=2e-3, seed=3,
                        precision=32)
    a = k.Simulation(cfg, pos, vel)
    a.step(6)
    pa, va = a.state()
    b = k.Simulation(cfg, pos, vel)
    b.step(3)
    pb, vb = b.state()
    step = b.info().step
    b.close()
    c = k.Simulation(cfg, pos, vel)
    c.set_state(pb, vb, step=step)
    c.step(3)
    pc, vc = c.state()
    assert np.array_equal(pa, pc) and np.array_equal(va, vc)
    a.close()
    c.close()


def test_batched_equals_plain_instances():
    """Instances of a batched run evolve exactly as separate runs."""
    _setup()
    import paper_1210_8084_gb300 as k
    from paper_1210_8084_gb300 import inputs
    ns = [7_000, 20_001, 3_333, 50_000]
    lams = [1e-3, 1e-1, 1e-4, 1.0]
    insts, P, V = [], [], []
    for i, (n, lam) in enumerate(zip(ns, lams)):
        p, v = f32_state(*inputs.sod_tube(n, seed=100 + i), (0, 0, 0), (1, 1, 1), (WALL, PER, PER))
        P.append(p)
        V.append(v)
        insts.append(dict(n=n, lam=lam, dt=5e-3, seed=1000 + i))
    base = dict(dim_pos=3, n_cells=(40, 1, 1), bc=(WALL, PER, PER), precision=32)
    batch = k.Simulation(k.make_config(**base, instances=insts), np.concatenate(P), np.concatenate(V))
    batch.step(8)
    pb, vb = batch.state()
    raw_b, der_b, glob_b = batch.moments()
    off = 0
    for i, inst in enumerate(insts):
        plain = k.Simulation(k.make_config(**base, lam=inst["lam"], dt=inst["dt"], seed=inst["seed"]), P[i], V[i])
        plain.step(8)
        pp, vp = plain.state()
        raw_p, der_p, glob_p = plain.moments()
        assert np.array_equal(pp, pb[off:off + ns[i]]), i
        assert np.array_equal(vp, vb[off:off + ns[i]]), i
        # moments: fixed-point sums do not depend on how particles are grouped,
        # so the instance's moments are those of the plain run bit for bit
        rows = slice(40 * i, 40 * (i + 1))
        assert np.array_equal(raw_p, raw_b[rows]), i
        assert np.array_equal(der_p, der_b[rows]), i
        assert np.array_equal(glob_p[0], glob_b[i]), i
        # the sort permutation of the instance: its particles in the same order
        perm_b = batch.perm()
        mine = perm_b[(perm_b >= off) & (perm_b < off + ns[i])] - off
        assert np.array_equal(mine, plain.perm()), i
        off += ns[i]
        plain.close()
    batch.close()


def test_batched_pruned_and_plain_tile_instances():
    """A batch whose instances take different tile searches (the pruned search on
    half c-bins where the contact distance is small, the plain tile search on
    c-bins where it is not) evolves each instance exactly as a separate run, and
    launches both tile kernels."""
    _setup()
    import paper_1210_8084_gb300 as k
    from paper_1210_8084_gb300 import inputs
    lo, hi, bc, cells = (0, 0, 0), (1, 0.5, 0.5), (WALL, PER, PER), (12, 6, 6)
    ns, lams = [40_000, 30_000, 20_000], [5e-3, 1e-4, 5e-2]
    insts, P, V = [], [], []
    for i, (n, lam) in enumerate(zip(ns, lams)):
        p, v = f32_state(*inputs.sod_tube(n, seed=200 + i, lo=lo, hi=hi), lo, hi, bc)
        P.append(p)
        V.append(v)
        insts.append(dict(n=n, lam=lam, dt=1e-2, seed=300 + i))
    base = dict(dim_pos=3, n_cells=cells, lo=lo, hi=hi, bc=bc, precision=32)
    batch = k.Simulation(k.make_config(**base, instances=insts), np.concatenate(P), np.concatenate(V))
    info = batch.info()
    assert info.tile_prune == 1
    assert info.kernels_per_step == 6   # plain tile search, pruned tile search, move, scan, two scatter passes
    batch.step(3)
    pb, vb = batch.state()
    raw_b = batch.moments()[0]
    off, nb = 0, int(np.prod(cells))
    for i, inst in enumerate(insts):
        plain = k.Simulation(k.make_config(**base, lam=inst["lam"], dt=inst["dt"], seed=inst["seed"]), P[i], V[i])
        assert plain.info().tile_prune == (0 if i == 1 else 1)
        plain.step(3)
        pp, vp = plain.state()
        assert np.array_equal(pp, pb[off:off + ns[i]]), i
        assert np.array_equal(vp, vb[off:off + ns[i]]), i
        assert np.array_equal(plain.moments()[0], raw_b[nb * i:nb * (i + 1)]), i
        off += ns[i]
        plain.close()
    batch.close()


@pytest.mark.parametrize("n", [0, 1, 2, 255, 257])
def test_tiny_and_ragged_sizes(n):
    _setup()
    import paper_1210_8084_gb300 as k
    rng = np.random.default_rng(n)
    pos = rng.random((n, 3))
    vel = rng.normal(0, 1, (n, 3))
    if n == 2:  # a head-on pair
        pos = np.array([[0.4, 0.5, 0.5], [0.6, 0.5, 0.5]])
        vel = np.array([[1.0, 0, 0], [-1.0, 0, 0]])
    cfg = k.make_config(dim_pos=3, n_cells=(3, 2, 1), bc=(WALL, PER, PER), sigma=0.5, dt=0.15, seed=1,
                        precision=64, flags=k.KMC_FLAG_RECORD)
    sim = k.Simulation(cfg, pos, vel)
    sim.step(2)
    p, v = sim.state()
    raw, der, glob = sim.moments()
    assert raw[:, 0].sum() == n
    if n == 2:
        best, partner = sim.partners()
        assert glob[0, 1] == pytest.approx(1.0, rel=1e-14)   # energy kept across the collision
        assert np.allclose(v.sum(0), 0.0, atol=1e-15)
    sim.close()


def test_invalid_particles_rejected():
    _setup()
    import paper_1210_8084_gb300 as k
    pos = np.full((10, 3), 0.5)
    vel = np.zeros((10, 3))
    cfg = k.make_config(dim_pos=3, n_cells=(2, 1, 1), lam=1e-3, dt=1e-3, precision=64)
    for bad in ("nan", "outside", "periodic_hi"):
        p = pos.copy()
        if bad == "nan":
            p[3, 1] = np.nan
        elif bad == "outside":
            p[4, 0] = 1.5
        else:
            p[5, 1] = 1.0   # periodic dims are [lo, hi)
        with pytest.raises(k.KmcError) as e:
            k.Simulation(cfg, p, vel)
        assert e.value.code == k.KMC_EINVAL


def test_energy_conservation_fp32():
    """Binary32 state: total energy drifts by < 1e-6 relative over 100 steps
    (binary64 per-bin sums)."""
    _setup()
    import paper_1210_8084_gb300 as k
    pos, vel = make_inputs("sod", 1_000_000, 3, (0, 0, 0), (1, 1, 1))
    pos, vel = f32_state(pos, vel, (0, 0, 0), (1, 1, 1), (WALL, PER, PER))
    cfg = k.make_config(dim_pos=3, n_cells=(500, 1, 1), bc=(WALL, PER, PER), lam=1e-3, dt=4e-4, seed=2,
                        precision=32)
    sim = k.Simulation(cfg, pos, vel)
    e0 = sim.moments()[2][0, 1]
    sim.step(100)
    e1 = sim.moments()[2][0, 1]
    sim.close()
    assert abs(e1 - e0) <= 1e-6 * e0, (e0, e1)


@pytest.mark.parametrize("precision", [32, 64])
@pytest.mark.parametrize("staged", [False, True])
def test_exact_tie_in_d2_goes_to_lower_id(precision, staged):
    """Two candidates at exactly the same distance of closest approach (mirror
    images in y of each other relative to particle 2).  Candidate 1 sorts
    before candidate 0 (lower y cell) but has the higher id: the closest
    candidate of particle 2 must be id 0 (R4), as in the oracle, and the
    following step must start from a clean tie list."""
    _setup()
    import oracle
    import paper_1210_8084_gb300 as k
    dt = 1e-3
    pos = np.array([[0.45, 0.5625, 0.5], [0.45, 0.4375, 0.5], [0.55, 0.5, 0.5]])
    vel = np.array([[200.0, -1.0, 0.0], [200.0, 1.0, 0.0], [0.0, 0.0, 0.0]])
    dtype = np.float32 if precision == 32 else np.float64
    pos, vel = pos.astype(dtype), vel.astype(dtype)
    flags = k.KMC_FLAG_RECORD | (k.KMC_FLAG_STAGED_SEARCH if staged else 0)
    cfg = k.make_config(dim_pos=3, n_cells=(4, 4, 4), bc=(PER, PER, PER), sigma=math.pi * 0.01, dt=dt, seed=3,
                        precision=precision, flags=flags)
    sim = k.Simulation(cfg, pos, vel)
    R2 = oracle_R2(0.0, 3, 3, (0, 0, 0), (1, 1, 1), sigma=math.pi * 0.01)
    sim.step(1)
    best, partner = sim.partners()
    p1, v1 = sim.state()
    sim.step(1)
    best2, partner2 = sim.partners()
    sim.close()
    assert list(best) == [2, 2, 0]
    assert list(partner) == [2, -1, 0]
    P = oracle.make_params(3, (4, 4, 4), (0, 0, 0), (1, 1, 1), (PER, PER, PER), R2=R2, dt=dt, seed=3, step=0,
                           decide32=precision == 32)
    assert list(oracle.best_partners(P, pos.astype(np.float64), vel.astype(np.float64))) == [2, 2, 0]
    P.step = 1
    assert np.array_equal(best2, oracle.best_partners(P, p1.astype(np.float64), v1.astype(np.float64)))


TILE_CASES = [
    # name, n, dim, n_cells, lo, hi, bc, lam, dt, precision (unsubdivided grids: the tile search)
    ("cubic3d_fp32_walls", 60_000, 3, (20, 6, 6), (0, 0, 0), (1, 0.3, 0.3), (WALL, PER, PER), 1e-3, 0.01, 32),
    ("cubic3d_fp64", 30_000, 3, (16, 5, 5), (0, 0, 0), (1, 5 / 16, 5 / 16), (WALL, PER, PER), 1e-3, 0.0125, 64),
    ("square2d_fp32_dense", 200_000, 2, (40, 40, 1), (0, 0, 0), (1, 1, 1), (WALL, WALL, PER), 5e-4, 0.005, 32),
    ("periodic3d_fp32_3cells", 20_000, 3, (3, 3, 4), (0, 0, 0), (1, 1, 1), (PER, PER, PER), 1e-3, 0.02, 32),
    ("tiny_cells_fp32", 7_777, 3, (30, 30, 4), (0, 0, 0), (1, 1, 0.2), (PER, PER, WALL), 1e-3, 0.003, 32),
    # the 3-D Sod benchmark's geometry at small N: ~208 per dense c-bin, R = 0.11 and v_th dt = 0.2 c-bin widths
    ("sod3d_fp32_narrow_contact", 120_000, 3, (16, 8, 8), (0, 0, 0), (1, 0.5, 0.5), (WALL, PER, PER), 0.0139,
     0.0125, 32),
    # 2-D with a contact distance of a third of a c-bin (the pruned search in 2-D), walls on all sides
    ("square2d_fp32_narrow", 200_000, 2, (40, 40, 1), (0, 0, 0), (1, 1, 1), (WALL, WALL, PER), 0.02, 0.005, 32),
    # 2-D periodic in y (images in the pruned search's rows)
    ("slab2d_fp32_periodic_narrow", 100_000, 2, (20, 12, 1), (0, 0, 0), (1, 0.6, 1), (WALL, PER, PER), 0.02, 0.01,
     32),
]


@pytest.mark.parametrize("case", TILE_CASES, ids=[c[0] for c in TILE_CASES])
def test_tile_search_matches_oracle_and_per_particle_search(case):
    """Grids whose search cells are the c-bins (forced with sub_cells = 1):
    the one-block-per-cell search gives the oracle's closest candidates and
    pairs bit for bit, and the same keys as the per-thread search, for dense
    and nearly empty cells, periodic windows that wrap (3 cells) and walls."""
    _setup()
    name, n, dim, n_cells, lo, hi, bc, lam, dt, prec = case
    pos, vel = make_inputs(name, n, dim, lo, hi)
    if prec == 32:
        pos, vel = f32_state(pos, vel, lo, hi, bc)
    seed = 5
    sub = (1, 1, 1)
    g = run_gpu_step(pos, vel, dim, n_cells, lo, hi, bc, lam, dt, seed, prec, sub_cells=sub)
    d = run_gpu_step(pos, vel, dim, n_cells, lo, hi, bc, lam, dt, seed, prec, sub_cells=sub, per_particle=True)
    o = oracle_step(pos, vel, dim, n_cells, lo, hi, bc, oracle_R2(lam, n, dim, lo, hi), dt, seed, 0, prec == 32)
    assert list(g["info"].sub_cells) == [1, 1, 1]
    assert (g["best"] >= 0).mean() > 0.05
    compare_step(g, o, prec, pos, vel, dim)
    assert np.array_equal(g["best"], d["best"]) and np.array_equal(g["partner"], d["partner"])
    assert np.array_equal(g["pos"], d["pos"]) and np.array_equal(g["vel"], d["vel"])


def test_autotune_picks_a_setup_with_identical_results():
    """kmc_autotune only times set-ups (subdivision, tile or per-particle
    search, staged tiles); a handle built from its choice gives the same
    closest candidates, pairs and state as the default handle."""
    _setup()
    import paper_1210_8084_gb300 as k
    from paper_1210_8084_gb300 import inputs
    for n_cells, hi in (((200, 1, 1), (1, 1, 1)), ((40, 8, 8), (1, 0.2, 0.2))):
        pos, vel = inputs.sod_tube(100_000, seed=4, hi=hi)
        pos, vel = inputs.cast_state(pos, vel, np.float32, (0, 0, 0), hi, (WALL, PER, PER))
        cfg = k.make_config(dim_pos=3, n_cells=n_cells, hi=hi, bc=(WALL, PER, PER), lam=1e-3, dt=0.2 / n_cells[0],
                            seed=9, precision=32, flags=k.KMC_FLAG_RECORD)
        best, ms = k.kmc_autotune(cfg, len(pos), pos, vel, k.KMC_WHERE_HOST, 2)
        assert ms > 0 and best.flags & k.KMC_FLAG_RECORD
        out = []
        for c in (cfg, best):
            sim = k.Simulation(c, pos, vel)
            sim.step(3)
            out.append((sim.partners(), sim.state()))
            sim.close()
        (b0, p0), (s0, v0) = out[0]
        (b1, p1), (s1, v1) = out[1]
        assert np.array_equal(b0, b1) and np.array_equal(p0, p1)
        assert np.array_equal(s0, s1) and np.array_equal(v0, v1)


@pytest.mark.parametrize("prec", [32, 64])
def test_adaptive_timestep_matches_oracle(prec):
    """KMC_FLAG_ADAPTIVE_DT (Sect. "Simulation setup": dt = dx / v_max(t)).
    Before every step the device's timestep equals the oracle's dx / v_max of
    the device state bit for bit (binary32 decisions use it rounded to
    binary32 on both sides), the elapsed time is the sum of the steps, and the
    step's closest candidates, pairs and virial pressure match the oracle."""
    _setup()
    import oracle
    import paper_1210_8084_gb300 as k
    from paper_1210_8084_gb300 import inputs
    n, n_cells, lo, hi, bc = 100_000, (100, 1, 1), (0, 0, 0), (1, 1, 1), (WALL, PER, PER)
    pos, vel = inputs.sod_tube(n, seed=21)
    if prec == 32:
        pos, vel = f32_state(pos, vel, lo, hi, bc)
    cfg = k.make_config(dim_pos=3, n_cells=n_cells, lo=lo, hi=hi, bc=bc, lam=1e-3, dt=1.0, seed=3, precision=prec,
                        flags=k.KMC_FLAG_RECORD | k.KMC_FLAG_ADAPTIVE_DT)
    sim = k.Simulation(cfg, pos, vel)
    t = 0.0
    for s in range(4):
        p, v = sim.state()
        p, v = p.astype(np.float64), v.astype(np.float64)
        info = sim.info()
        P = oracle.make_params(3, n_cells, lo, hi, bc, R2=oracle_R2(1e-3, n, 3, lo, hi), dt=1.0, seed=3, step=s,
                               decide32=prec == 32)
        dt = oracle.adaptive_dt(P, v, 1.0)
        assert info.dt == dt, (s, info.dt, dt)
        assert info.time == t
        # binary32: |v|^2 is rounded to binary32 before the binary64 root and quotient
        assert dt == pytest.approx(0.01 / np.linalg.norm(v, axis=1).max(), rel=1e-12 if prec == 64 else 1e-6)
        P.dt = dt
        sim.step(1, want_moments=1)
        best, partner = sim.partners()
        ob = oracle.best_partners(P, p, v)
        assert np.array_equal(best, ob), s
        paired = oracle.collide_move(P, p, v, ob)[3]
        assert np.array_equal(partner, paired), s
        t += dt
        # p_vir = Sum W / (2 d V_c dt) with the dt of the step that produced W
        raw, der, glob = sim.moments()
        assert np.allclose(der[:, 6], raw[:, 7] / (2 * 3 * 0.01 * dt), rtol=1e-12, atol=0)
    assert sim.info().time == t
    sim.close()


@pytest.mark.parametrize("prec", [32, 64])
def test_velocity2d_one_step_parity(prec):
    """KMC_FLAG_VELOCITY_2D (the paper's 2-D runs): one step against the
    oracle with 2-D velocities -- closest candidates and pairs bit for bit,
    velocities stay in the plane, temperature with two degrees of freedom."""
    _setup()
    import oracle
    import paper_1210_8084_gb300 as k
    from paper_1210_8084_gb300 import inputs
    n, n_cells, lo, hi, bc = 150_000, (60, 30, 1), (0, 0, 0), (1, 0.5, 1), (WALL, PER, PER)
    pos, vel = inputs.sod_tube(n, seed=41, hi=hi, dim_pos=2, vel_dim=2)
    if prec == 32:
        pos, vel = f32_state(pos, vel, lo, hi, bc)
    dt = 0.2 / 60
    cfg = k.make_config(dim_pos=2, n_cells=n_cells, lo=lo, hi=hi, bc=bc, lam=1e-3, dt=dt, seed=8, precision=prec,
                        flags=k.KMC_FLAG_RECORD | k.KMC_FLAG_VELOCITY_2D)
    sim = k.Simulation(cfg, pos, vel)
    info = sim.info()
    keys = sim.cell_keys()
    sim.step(1, want_moments=1)
    best, partner = sim.partners()
    p, v = sim.state()
    raw, der, glob = sim.moments()
    sim.close()
    g = dict(info=info, keys=keys, best=best, partner=partner, pos=p, vel=v, raw=raw, der=der, glob=glob)
    P = oracle.make_params(2, n_cells, lo, hi, bc, R2=oracle_R2(1e-3, n, 2, lo, hi), dt=dt, seed=8, step=0,
                           decide32=prec == 32, vel_dim=2)
    key, _ = oracle.cell_keys(P, pos)
    ob = oracle.best_partners(P, pos, vel)
    po, vo, W, paired = oracle.collide_move(P, pos, vel, ob)
    oraw, oder, oglob = oracle.moments(P, po, vo, W)
    o = dict(P=P, keys=key, best=ob, partner=paired, pos=po, vel=vo, W=W, raw=oraw, der=oder, glob=oglob)
    assert (best >= 0).mean() > 0.05
    compare_step(g, o, prec, pos, vel, 2)
    assert np.all(v[:, 2] == 0)
    ok = raw[:, 0] > 100
    assert np.allclose(der[ok, 4], oder[ok, 4], rtol=1e-10 if prec == 64 else 1e-4)   # T = c2 / 2


def test_velocity2d_rejects_out_of_plane_input():
    _setup()
    import paper_1210_8084_gb300 as k
    pos = np.array([[0.5, 0.5, 0.0], [0.25, 0.25, 0.0]], np.float32)
    vel = np.array([[1.0, 0.0, 0.0], [0.0, 1.0, 0.1]], np.float32)
    cfg = k.make_config(dim_pos=2, n_cells=(4, 4, 1), bc=(PER, PER, PER), lam=1e-2, dt=1e-3, seed=1, precision=32,
                        flags=k.KMC_FLAG_VELOCITY_2D)
    with pytest.raises(k.KmcError):
        k.Simulation(cfg, pos, vel)


@pytest.mark.parametrize("prec", [32, 64])
def test_absorbing_walls_match_oracle(prec):
    """KMC_BC_ABSORB (Sect. "Sedov test"): over several steps the device
    removes the same particles as the oracle (NaN state), keeps them out of the
    search and the moments, and the other particles' closest candidates and
    pairs stay bit for bit those of the oracle."""
    _setup()
    import oracle
    import paper_1210_8084_gb300 as k
    from paper_1210_8084_gb300 import inputs
    ABS = k.KMC_BC_ABSORB
    n, n_cells, lo, hi, bc = 80_000, (20, 20, 20), (0, 0, 0), (1, 1, 1), (ABS, ABS, ABS)
    pos, vel = inputs.periodic_box(n, seed=52, T=1.0)
    if prec == 32:
        pos, vel = f32_state(pos, vel, lo, hi, (1, 1, 1))
    dt = 0.02
    cfg = k.make_config(dim_pos=3, n_cells=n_cells, lo=lo, hi=hi, bc=bc, lam=1e-3, dt=dt, seed=4, precision=prec,
                        flags=k.KMC_FLAG_RECORD)
    sim = k.Simulation(cfg, pos, vel)
    R2 = oracle_R2(1e-3, n, 3, lo, hi)
    for s in range(4):
        p, v = sim.state()
        p, v = p.astype(np.float64), v.astype(np.float64)
        P = oracle.make_params(3, n_cells, lo, hi, bc, R2=R2, dt=dt, seed=4, step=s, decide32=prec == 32)
        ob = oracle.best_partners(P, p, v)
        po, vo, W, paired = oracle.collide_move(P, p, v, ob)
        sim.step(1, want_moments=1)
        best, partner = sim.partners()
        p1, v1 = sim.state()
        raw, der, glob = sim.moments()
        assert np.array_equal(best, ob), s
        assert np.array_equal(partner, paired), s
        gone_d, gone_o = np.isnan(p1[:, 0]), np.isnan(po[:, 0])
        diff = gone_d != gone_o
        if prec == 64:
            assert not diff.any(), s
        else:
            # removal is decided on the end-of-step position, which the binary32
            # state rounds: a mismatch may only occur where the side that kept
            # the particle has it within rounding of an absorbing face
            kept = np.where(gone_d[diff][:, None], po[diff], p1[diff].astype(np.float64))
            dist = np.minimum(np.abs(kept), np.abs(1.0 - kept)).min(1)
            assert diff.sum() <= 3 and np.all(dist < 1e-5), (s, diff.sum(), dist)
        assert glob[0, 0] == np.isfinite(p1[:, 0]).sum()
    assert np.isnan(p1[:, 0]).sum() > 1000
    sim.close()


def test_graph_resident_step_loop_equals_kernel_by_kernel():
    """kmc_step runs all its steps in one CUDA graph (a conditional while node
    driven by a device-side step counter).  Calls of 3 + 4 steps, one of 7, and
    7 steps launched kernel by kernel (KMC_FLAG_NO_GRAPH) give the same state,
    moments and step counter bit for bit; a batched handle too."""
    _setup()
    import paper_1210_8084_gb300 as k
    from paper_1210_8084_gb300 import inputs
    pos, vel = f32_state(*inputs.sod_tube(80_000, seed=31), (0, 0, 0), (1, 1, 1), (WALL, PER, PER))
    base = dict(dim_pos=3, n_cells=(80, 1, 1), bc=(WALL, PER, PER), lam=1e-3, dt=0.2 / 80, seed=17, precision=32)
    insts = [dict(n=30_000, lam=1e-3, dt=0.0025, seed=1), dict(n=50_000, lam=1e-2, dt=0.0025, seed=2)]
    for kw in (base, dict(dim_pos=3, n_cells=(80, 1, 1), bc=(WALL, PER, PER), precision=32, instances=insts)):
        out = []
        for flags, calls in ((0, (3, 4)), (0, (7,)), (k.KMC_FLAG_NO_GRAPH, (7,))):
            sim = k.Simulation(k.make_config(**kw, flags=flags), pos, vel)
            for c in calls:
                sim.step(c, want_moments=1)
            info = sim.info()
            assert info.step == 7
            assert info.graph_mode == (0 if flags else 2)
            out.append((sim.state(), sim.moments()))
            sim.close()
        for (s, m) in out[1:]:
            assert np.array_equal(s[0], out[0][0][0]) and np.array_equal(s[1], out[0][0][1])
            for a, b in zip(m, out[0][1]):
                assert np.array_equal(a, b)


@pytest.mark.parametrize("prec", [32, 64])
@pytest.mark.parametrize("dim", [2, 3])
def test_dsmc_variant_matches_oracle(prec, dim):
    """KMC_FLAG_DSMC, the random-partner comparison variant (Sect. "Direct
    Simulation Monte Carlo Technique", Bird's no-time-counter scheme): two
    steps from the same state on both sides.  The collisions are computed in
    binary64 on both sides from the same draws, the cell's particles in id
    order, so the accepted pairs are the same: the number of collided
    particles matches exactly and the end velocities agree to 1e-12 (binary64)
    or to one binary32 rounding (binary32, most of them bit for bit)."""
    _setup()
    import oracle
    import paper_1210_8084_gb300 as k
    from paper_1210_8084_gb300 import inputs
    if dim == 3:
        n, n_cells, lo, hi, bc = 60_000, (60, 1, 1), (0, 0, 0), (1, 1, 1), (WALL, PER, PER)
        pos, vel = inputs.sod_tube(n, seed=13)
        lam, dt = 1e-3, 0.2 / 60
    else:
        n, n_cells, lo, hi, bc = 40_000, (20, 20, 1), (0, 0, 0), (1, 1, 1), (WALL, WALL, PER)
        pos, vel = inputs.sod_tube(n, seed=13, dim_pos=2, vel_dim=2)
        lam, dt = 1e-3, 0.2 / 20
    if prec == 32:
        pos, vel = f32_state(pos, vel, lo, hi, bc)
    flags = k.KMC_FLAG_DSMC | (k.KMC_FLAG_VELOCITY_2D if dim == 2 else 0)
    cfg = k.make_config(dim_pos=dim, n_cells=n_cells, lo=lo, hi=hi, bc=bc, lam=lam, dt=dt, seed=23, precision=prec,
                        flags=flags)
    sim = k.Simulation(cfg, pos, vel)
    assert list(sim.info().sub_cells)[:dim] == [1] * dim
    P = oracle.make_params(dim, n_cells, lo, hi, bc, R2=oracle_R2(lam, n, dim, lo, hi), dt=dt, seed=23,
                           decide32=prec == 32, vel_dim=dim)
    p, v = pos, vel
    for s in range(2):
        sim.step(1, want_moments=1)
        pd, vd = sim.state()
        glob = sim.moments()[2]
        P.step = s
        p, v, collided, acc = oracle.dsmc_step(P, p, v)
        assert acc > n // 50
        assert glob[0, 6] * 2 == collided.sum(), (s, glob[0, 6] * 2, collided.sum())
        scale = np.linalg.norm(v, axis=1)[:, None] + 1e-300
        err = np.abs(vd - v) / scale
        if prec == 64:
            assert err.max() <= 1e-12, (s, err.max())
        else:
            assert err.max() <= 2.0 ** -22 and (err == 0).mean() > 0.999, (s, err.max(), (err == 0).mean())
        tol_x = 1e-12 if prec == 64 else 4e-6
        assert np.abs(pd[:, :dim] - p[:, :dim]).max() <= tol_x
        p, v = pd.astype(np.float64), vd.astype(np.float64)   # the next step from the device state
    sim.close()


@pytest.mark.parametrize("case", [c for c in TILE_CASES if c[9] == 32], ids=[c[0] for c in TILE_CASES if c[9] == 32])
def test_tile_pruning_changes_speed_only(case):
    """The binary32 tile search skips candidate clusters whose swept boxes stay
    out of the contact distance of a warp's homes: three steps with and without
    the pruning give bit-identical closest candidates, pairs and states, and in
    dense c-bins much wider than the contact distance the pruned search counts
    fewer pair tests than the plain one's (C_p - 1) / 2 per particle."""
    _setup()
    import paper_1210_8084_gb300 as k
    name, n, dim, n_cells, lo, hi, bc, lam, dt, prec = case
    pos, vel = make_inputs(name, n, dim, lo, hi)
    pos, vel = f32_state(pos, vel, lo, hi, bc)
    out = []
    # pruned (half c-bin search cells) where the contact distance is at most half a
    # c-bin and every periodic dimension has 6 c-bins or more
    expect = name in ("cubic3d_fp32_walls", "sod3d_fp32_narrow_contact", "square2d_fp32_narrow",
                      "slab2d_fp32_periodic_narrow")
    for flags in (k.KMC_FLAG_RECORD, k.KMC_FLAG_RECORD | k.KMC_FLAG_NO_TILE_PRUNE):
        cfg = k.make_config(dim_pos=dim, n_cells=n_cells, lo=lo, hi=hi, bc=bc, lam=lam, dt=dt, seed=9,
                            precision=32, flags=flags)
        sim = k.Simulation(cfg, pos, vel)
        info = sim.info()
        if flags & k.KMC_FLAG_NO_TILE_PRUNE:
            assert info.tile_prune == 0
        else:
            assert info.tile_prune == int(expect)
            if expect:
                assert list(info.sub_cells)[:dim] == [2] * dim
            pruned = info.tile_prune
        cand = sim.window_size()
        sim.step(3)
        best, partner = sim.partners()
        p1, v1 = sim.state()
        out.append((best, partner, p1, v1, sim.tile_tests(), cand))
        sim.close()
    (b0, q0, p0, w0, t0, c0), (b1, q1, p1, w1, t1, _) = out
    assert (b0 >= 0).mean() > 0.05
    assert np.array_equal(b0, b1) and np.array_equal(q0, q1)
    assert np.array_equal(p0, p1) and np.array_equal(w0, w1)
    assert t1 == 0.0
    assert (t0 > 0) == bool(pruned)
    width = min((hi[d] - lo[d]) / n_cells[d] for d in range(dim))
    if n / np.prod(n_cells[:dim]) >= 50 and np.sqrt(info.R2) < 0.25 * width:
        # dense c-bins and a contact distance well inside one: fewer tests than
        # the plain search's (C_p - 1) / 2 per particle-step (window of the first step)
        assert t0 < 3 * n * (c0 - 1) / 2


def test_tile_search_far_from_origin():
    """Coordinates near 100 (the rounding margin of the pruned tile search grows
    with the coordinates' magnitude): closest candidates and pairs equal the
    oracle's binary32 decisions, with and without the pruning.  (The end-of-step
    state is not compared with the binary64 oracle here: at |x| ~ 100 a binary32
    position that ends within an ulp of a wall or face may fold or wrap
    differently from the binary64 one.)"""
    _setup()
    import paper_1210_8084_gb300 as k
    n, dim, n_cells, lo, hi, bc, lam, dt = 60_000, 3, (20, 6, 6), (100, -50, 7), (101, -49.7, 7.3), \
        (WALL, PER, PER), 1e-3, 0.01
    pos, vel = make_inputs("offset", n, dim, lo, hi)
    pos, vel = f32_state(pos, vel, lo, hi, bc)
    o = oracle_step(pos, vel, dim, n_cells, lo, hi, bc, oracle_R2(lam, n, dim, lo, hi), dt, 5, 0, True)
    assert (o["best"] >= 0).mean() > 0.05
    for flags in (k.KMC_FLAG_RECORD, k.KMC_FLAG_RECORD | k.KMC_FLAG_NO_TILE_PRUNE):
        cfg = k.make_config(dim_pos=dim, n_cells=n_cells, lo=lo, hi=hi, bc=bc, lam=lam, dt=dt, seed=5,
                            precision=32, flags=flags)
        sim = k.Simulation(cfg, pos, vel)
        assert sim.info().tile_prune == (0 if flags & k.KMC_FLAG_NO_TILE_PRUNE else 1)
        sim.step(1)
        best, partner = sim.partners()
        sim.close()
        assert np.array_equal(best, o["best"]) and np.array_equal(partner, o["partner"])


@pytest.mark.parametrize("prec,tt,cap,split", [(32, 64, 64, 1), (32, 128, 768, 1), (32, 256, 6144, 1),
                                               (64, 128, 3072, 1), (64, 64, 100, 1), (32, 256, 1536, 2),
                                               (32, 128, 64, 3), (32, 256, 768, 8),
                                               (32, 96, 1536, 1), (64, 224, 768, 1)])
def test_tile_search_parameters_do_not_change_results(prec, tt, cap, split):
    """Threads per c-bin block, staging capacity and the number of blocks that
    share a c-bin's window (the autotuner's choices; binary32: the pruned
    search, binary64: the plain tile search) change speed only: the
    closest candidates and pairs equal the oracle's, from a capacity far below
    one neighbourhood (many staging chunks) to one above it, and with up to 8
    blocks per c-bin (some of them then without candidates)."""
    _setup()
    import paper_1210_8084_gb300 as k
    name, n, dim, n_cells, lo, hi, bc, lam, dt, _ = TILE_CASES[0]
    pos, vel = make_inputs(name, n, dim, lo, hi)
    if prec == 32:
        pos, vel = f32_state(pos, vel, lo, hi, bc)
    cfg = k.make_config(dim_pos=dim, n_cells=n_cells, lo=lo, hi=hi, bc=bc, lam=lam, dt=dt, seed=5, precision=prec,
                        flags=k.KMC_FLAG_RECORD, tile_threads=tt, tile_cap=cap, tile_split=split)
    sim = k.Simulation(cfg, pos, vel)
    info = sim.info()
    assert (info.tile_threads, info.tile_cap, info.tile_split) == (tt, cap, split)
    assert info.tile_prune == (prec == 32)   # binary32: the pruned search on half c-bins
    sim.step(1)
    best, partner = sim.partners()
    sim.close()
    o = oracle_step(pos, vel, dim, n_cells, lo, hi, bc, oracle_R2(lam, n, dim, lo, hi), dt, 5, 0, prec == 32)
    assert (best >= 0).mean() > 0.05
    assert np.array_equal(best, o["best"]) and np.array_equal(partner, o["partner"])
