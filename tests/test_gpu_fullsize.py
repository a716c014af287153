"""Parity at the full sizes of the workloads, in the benchmark's launch set-up.

The benchmark's configuration (same config fields, library-chosen search
grid, graph replay with moments) runs a few steps on the full state; then one
device step is checked against the oracle on samples the oracle can compute
exactly on their own: every particle of a sampled c-bin.  The closest
candidate of a particle depends on the c-bins within one of its own, and its
partner's choice on those within two, so the oracle's step on the particles
of the c-bins within two of the sampled one (global geometry, global contact
distance, global ids for the random keys) decides the sampled particles'
pairs exactly as the whole system does.  Sampled c-bins: both walls, the
initial density step, the dense and the dilute side (and for the 2-D
quadrants the corners and the quadrant boundaries).

Checked on samples: the velocities of unpaired particles bit for bit (free
flight, mirrored at a wall), post-collision velocities to 1e-5 of the pair's
speed scale (a different partner or a missed pair shows as an O(1) error),
positions to binary32 rounding.  Checked on the whole
state (properties at any size): every cell key equals the oracle's binary32
key of the device's own positions, the per-c-bin counts of the moments equal
the counts of those keys, and kinetic energy is conserved (elastic
collisions, specular walls).
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _setup():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__ as g
    g.build()


def _near(cidx, t, n_cells, bc, reach):
    """Particles whose c-bin is within `reach` of c-bin t in every dimension
    (cyclic distance in periodic dimensions)."""
    ok = np.ones(cidx.shape[0], dtype=bool)
    for d in range(3):
        n = n_cells[d]
        if n == 1:
            continue
        diff = np.abs(cidx[:, d] - t[d])
        if bc[d] == 0:
            diff = np.minimum(diff, n - diff)
        ok &= diff <= reach
    return ok


def _oracle_cell(P, pos, vel, cidx, t, n_cells, bc):
    """The oracle's step for every particle of c-bin t, from the particles of
    the c-bins within two of it.  Returns (ids, pos, vel, paired) of c-bin t."""
    import oracle
    sub = np.flatnonzero(_near(cidx, t, n_cells, bc, 2))      # increasing ids
    best = oracle.best_partners(P, pos[sub], vel[sub])
    po, vo, _, paired = oracle.collide_move(P, pos[sub], vel[sub], best, ids=sub)
    own = _near(cidx[sub], t, n_cells, bc, 0)
    partner = np.where(paired >= 0, sub[np.maximum(paired, 0)], -1)
    return sub[own], po[own], vo[own], partner[own]


def _run(workload, cells, steps_before=2):
    _setup()
    import oracle
    import paper_1210_8084_gb300 as k
    from paper_1210_8084_gb300 import inputs

    w = dict(inputs.WORKLOADS[workload])
    n, dim, n_cells, bc = w["n"], w["dim_pos"], tuple(w["n_cells"]), tuple(w["bc"])
    pos, vel = inputs.make_state(w)
    pos, vel = inputs.cast_state(pos, vel, np.float32, w["lo"], w["hi"], bc)
    cfg = k.make_config(dim_pos=dim, n_cells=n_cells, lo=w["lo"], hi=w["hi"], bc=bc, lam=w["lam"], dt=w["dt"],
                        seed=w["seed"], precision=w["precision"], occupancy_target=0.0)
    sim = k.Simulation(cfg, pos, vel)
    del pos, vel
    # contact distance on the oracle side (Eq. 7, Eq. reff_lambda; n = N / V)
    V = float(np.prod([w["hi"][d] - w["lo"][d] for d in range(dim)]))
    R2 = oracle.contact_R2(w["lam"], 0.0, n / V)
    sim.step(steps_before, want_moments=1)
    p0, v0 = sim.state()
    e0 = sim.moments()[2][0, 1]
    sim.step(1, want_moments=1)
    p1, v1 = sim.state()
    keys1 = sim.cell_keys()
    raw1, _, glob1 = sim.moments()
    sim.close()

    P = oracle.make_params(dim, n_cells, w["lo"], w["hi"], bc, R2=R2, dt=w["dt"], seed=w["seed"],
                           step=steps_before, decide32=True)
    # whole state: keys of the device's positions, counts per c-bin, energy
    okey, _ = oracle.cell_keys(P, p1.astype(np.float64))
    assert np.array_equal(keys1, okey), f"{int((keys1 != okey).sum())} cell keys differ"
    assert np.array_equal(raw1[:, 0], np.bincount(okey, minlength=raw1.shape[0]).astype(np.float64))
    assert abs(glob1[0, 1] - e0) <= 1e-6 * e0
    assert abs(glob1[0, 0] - n) == 0

    # samples: every particle of the chosen c-bins
    p0d, v0d = p0.astype(np.float64), v0.astype(np.float64)
    _, cidx = oracle.cell_keys(P, p0d)
    checked = paired_seen = 0
    for t in cells:
        ids, po, vo, partner = _oracle_cell(P, p0d, v0d, cidx, t, n_cells, bc)
        assert ids.size > 0, f"empty sample c-bin {t}"
        paired = partner >= 0
        gv = v1[ids].astype(np.float64)
        scale = np.linalg.norm(vo, axis=1)
        s_own = np.linalg.norm(v0d[ids[paired]], axis=1)
        s_par = np.linalg.norm(v0d[partner[paired]], axis=1)
        scale[paired] = np.maximum(scale[paired], np.maximum(s_own, s_par))
        err = np.abs(gv - vo).max(1) / np.maximum(scale, 1e-300)
        # a pairing that differs shows as an O(1) velocity error: a particle the
        # device left unpaired keeps (or mirrors at a wall) its velocity
        assert np.all(err[~paired] == 0), f"c-bin {t}: {int((err[~paired] != 0).sum())} unpaired velocities differ"
        assert err.max() <= 1e-5, f"c-bin {t}: velocity rel err {err.max()}"
        assert np.abs(p1[ids, :dim].astype(np.float64) - po[:, :dim]).max() <= 4e-6
        checked += ids.size
        paired_seen += int(paired.sum())
    assert paired_seen > 0.02 * checked
    return checked


def test_sod_tube_16M_sampled_cbins():
    """The benchmark's workload: 16M particles, 2000 slab c-bins, lambda/L = 1e-3."""
    cells = [(0, 0, 0), (500, 0, 0), (999, 0, 0), (1000, 0, 0), (1500, 0, 0), (1999, 0, 0)]
    assert _run("sod1d_fp32_16M", cells) > 30_000


def test_quadrants_64M_sampled_cbins():
    """2-D four-quadrant problem: 64M particles, 512 x 512 c-bins (tile search)."""
    cells = [(0, 0, 0), (511, 511, 0), (0, 511, 0), (255, 255, 0), (256, 256, 0), (255, 256, 0),
             (128, 384, 0), (400, 100, 0)]
    assert _run("quadrant2d_fp32_64M", cells) > 1_500


def test_sod_3d_16M_sampled_cbins():
    """3-D Sod tube with the c-bin occupancy of the 512M case: 512 x 16 x 16 c-bins."""
    cells = [(0, 0, 0), (255, 7, 8), (256, 0, 15), (511, 15, 15), (100, 3, 12), (400, 12, 3)]
    assert _run("sod3d_fp32_16M", cells) > 500
