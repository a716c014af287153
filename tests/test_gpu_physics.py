"""Physics of the device path over full runs.

* Sod shock tube in the paper's geometry (Sect. "Sod test": cubic c-bins,
  about 20 particles per c-bin): 1024 x 32 x 32 c-bins over 1 x 1/32 x 1/32,
  21M particles, lambda/L = 1e-3, t = 0.1.  Relative L1 distance of n, p, T to
  the exact Riemann solution (gamma = 5/3) within 2 %; the star state (the
  plateau between rarefaction and contact) within 2 %.
* Sod shock tube with slab c-bins at 16M particles (2000 c-bins, lambda/L = 1e-3, t = 0.1):
  relative L1 distance of n, p, T to the exact Riemann solution (Sect. "Sod
  test"; gamma = 5/3).  Measured 3.4 %, 4.0 %, 4.9 % (the 2 % aimed at is not
  reached: with one c-bin across y and z the candidates of a particle lie
  mostly beside it, the closest-approach choice favours pairs approaching
  sideways, and x-momentum is exchanged more slowly than the nominal lambda
  suggests); the bounds below guard that behaviour.
* The batched ensemble (256 slab Sod tubes, N and lambda log-uniform): L1 of
  n, p, T to the exact solution for the instances with lambda/L <= 1e-3.
* Ensemble means of the device path and of the CPU oracle over independent
  seeds agree per output bin within 3 standard errors.
* A mono-energetic gas relaxes to the Maxwell speed law (Sect. "Equilibration
  and Speed-up").
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


def _profiles(raw, nb, n_left_density):
    """Coarse-grain per-c-bin raw sums into nb output bins: (n/n_l, u, p/p_l, T)."""
    k = raw.shape[0] // nb
    R = raw.reshape(nb, k, 8).sum(1)
    N = R[:, 0]
    u = R[:, 1] / N
    c2 = (R[:, 4] + R[:, 5] + R[:, 6]) / N - (R[:, 1:4] ** 2).sum(1) / N ** 2
    T = c2 / 3.0
    dens = N * nb
    return dens / n_left_density, u, dens * T / n_left_density, T


def _profiles_x(raw, ncx, nb, n_left_density):
    """As _profiles, after summing c-bins over y and z (c-bin rows are x fastest)."""
    rx = raw.reshape(raw.shape[0] // ncx, ncx, 8).sum(0)
    return _profiles(rx, nb, n_left_density)


def test_sod_3d_cubic_bins_within_two_percent():
    _setup()
    import paper_1210_8084_gb300 as k
    from paper_1210_8084_gb300 import inputs
    from analytic import riemann
    ncx, ppc, steps = 1024, 20, 512
    n_cells = (ncx, 32, 32)
    hi = (1.0, 1 / 32, 1 / 32)
    n = ppc * ncx * 32 * 32
    dt = 0.2 / ncx
    bc = (WALL, PER, PER)
    pos, vel = inputs.sod_tube(n, seed=5, hi=hi)
    pos, vel = inputs.cast_state(pos, vel, np.float32, (0, 0, 0), hi, bc)
    sim = k.Simulation(k.make_config(dim_pos=3, n_cells=n_cells, hi=hi, bc=bc, lam=1e-3, dt=dt, seed=5,
                                     precision=32), pos, vel)
    e0 = sim.moments()[2][0, 1]
    sim.step(steps, want_moments=1)
    raw, der, glob = sim.moments()
    sim.close()
    t = steps * dt
    nb = 256
    n_l = n * 8 / 9 / 0.5
    dn, u, p, T = _profiles_x(raw, ncx, nb, n_l)
    ex = riemann.sod_profile(np.linspace(0, 1, nb + 1), t, 0.5, 1.0, 1.0)
    l1 = {name: float(np.abs(q - qe).sum() / np.abs(qe).sum())
          for name, q, qe in (("n", dn, ex[:, 0]), ("u", u, ex[:, 1]), ("p", p, ex[:, 2]), ("T", T, ex[:, 3]))}
    print("Sod (cubic c-bins) L1:", l1)
    assert l1["n"] <= 0.02 and l1["p"] <= 0.02 and l1["T"] <= 0.02, l1
    assert l1["u"] <= 0.08, l1
    # star state on the left of the contact: x in [0.51, 0.54]
    xc = (np.arange(nb) + 0.5) / nb
    star = (xc > 0.51) & (xc < 0.54)
    for q, qe in ((dn, ex[:, 0]), (u, ex[:, 1]), (p, ex[:, 2]), (T, ex[:, 3])):
        assert abs(q[star].mean() / qe[star].mean() - 1) < 0.02
    assert abs(glob[0, 1] / e0 - 1) < 1e-6
    assert glob[0, 0] == n


def test_sod_tube_l1_against_exact_riemann():
    _setup()
    import paper_1210_8084_gb300 as k
    from paper_1210_8084_gb300 import inputs
    from analytic import riemann
    n, nc, steps = 16_000_000, 2000, 1000
    dt = 0.2 / nc
    pos, vel = inputs.sod_tube(n, seed=5)
    pos, vel = inputs.cast_state(pos, vel, np.float32, (0, 0, 0), (1, 1, 1), (WALL, PER, PER))
    cfg = k.make_config(dim_pos=3, n_cells=(nc, 1, 1), bc=(WALL, PER, PER), lam=1e-3, dt=dt, seed=5, precision=32)
    sim = k.Simulation(cfg, pos, vel)
    e0 = sim.moments()[2][0, 1]
    sim.step(steps, want_moments=1)
    raw, der, glob = sim.moments()
    sim.close()
    t = steps * dt
    nb = 200
    n_l = n * 8 / 9 / 0.5
    dn, u, p, T = _profiles(raw, nb, n_l)
    ex = riemann.sod_profile(np.linspace(0, 1, nb + 1), t, 0.5, 1.0, 1.0)
    l1 = {name: float(np.abs(q - qe).sum() / np.abs(qe).sum())
          for name, q, qe in (("n", dn, ex[:, 0]), ("u", u, ex[:, 1]), ("p", p, ex[:, 2]), ("T", T, ex[:, 3]))}
    print("Sod L1:", l1)
    assert l1["n"] <= 0.045 and l1["p"] <= 0.05 and l1["T"] <= 0.06, l1
    assert l1["u"] <= 0.30, l1
    # undisturbed states far from the waves
    assert np.abs(dn[:60] - 1.0).max() < 0.02 and np.abs(dn[150:] - 0.125).max() < 0.01
    assert abs(glob[0, 1] / e0 - 1) < 1e-6          # energy, walls included
    assert glob[0, 0] == n


def test_batched_ensemble_l1_against_exact_riemann():
    """The batched ensemble of the benchmark (256 Sod tubes, N log-uniform in
    [50k, 2M], lambda/L log-uniform in [1e-4, 1], 200 slab c-bins each) run to
    t = 0.1 in one batched handle: the relative L1 distance of n, p, T to the
    exact Riemann solution for every instance with lambda/L <= 1e-3.  Batched
    and plain runs give bit-identical instance states (tested separately), so
    these are the L1 errors of both."""
    _setup()
    import paper_1210_8084_gb300 as k
    from paper_1210_8084_gb300 import inputs
    from analytic import riemann
    w = dict(inputs.WORKLOADS["sod1d_batched_256"])
    ns, lams = inputs.log_uniform_instances(w["n_instances"], seed=w["seed"], n_range=w["n_range"],
                                            lam_range=w["lam_range"])
    nc = w["n_cells"][0]
    P, V, insts = [], [], []
    for i in range(len(ns)):
        p, v = inputs.sod_tube(int(ns[i]), seed=i)
        p, v = inputs.cast_state(p, v, np.float32, w["lo"], w["hi"], w["bc"])
        P.append(p)
        V.append(v)
        insts.append(dict(n=int(ns[i]), lam=float(lams[i]), dt=w["dt"], seed=i))
    cfg = k.make_config(dim_pos=3, n_cells=w["n_cells"], lo=w["lo"], hi=w["hi"], bc=w["bc"], precision=32,
                        instances=insts)
    sim = k.Simulation(cfg, np.concatenate(P), np.concatenate(V))
    del P, V
    steps = int(round(0.1 / w["dt"]))
    sim.step(steps, want_moments=1)
    raw, _, glob = sim.moments()
    sim.close()
    t = steps * w["dt"]
    ex = riemann.sod_profile(np.linspace(0, 1, nc + 1), t, 0.5, 1.0, 1.0)
    rows = []
    for i in np.flatnonzero(lams <= 1e-3):
        dn, u, pp, T = _profiles(raw[nc * i:nc * (i + 1)], nc, ns[i] * 8 / 9 / 0.5)
        l1 = [float(np.abs(q - qe).sum() / np.abs(qe).sum()) for q, qe in ((dn, ex[:, 0]), (pp, ex[:, 2]),
                                                                         (T, ex[:, 3]))]
        rows.append((int(ns[i]), float(lams[i]), *l1))
        assert glob[i, 0] == ns[i]
    rows = np.array(rows)
    for r in rows:
        print("N %8d  lambda/L %.2e  L1 n %.3f  p %.3f  T %.3f" % tuple(r))
    med = np.median(rows[:, 2:], axis=0)
    print("instances:", len(rows), "median L1 n, p, T:", med, "max:", rows[:, 2:].max(0))
    # measured: median 4.9 %, 6.1 %, 6.6 %; worst 7.1 %, 9.0 %, 9.6 % (the smallest instances); the error
    # falls with N (counting noise of 200 output bins on top of the slab geometry's bias): 3.1-3.7 % in n
    # above 1M particles
    assert len(rows) >= 40
    assert np.all(med <= [0.06, 0.075, 0.08]), med
    assert np.all(rows[:, 2:].max(0) <= [0.09, 0.115, 0.12]), rows[:, 2:].max(0)
    big = rows[:, 0] >= 1_000_000
    assert big.sum() >= 5 and rows[big, 2].max() <= 0.045, rows[big]


def test_ensemble_means_match_oracle():
    """16 seeds per side of a small Sod tube (binary64 device path): per output
    bin and field (n, u, T) the two ensemble means differ by at most 3 combined
    standard errors, except for at most 2 of the 75 checks (0.27 % expected)."""
    _setup()
    import oracle
    import paper_1210_8084_gb300 as k
    from paper_1210_8084_gb300 import inputs
    n, nc, steps, R = 10_000, 25, 25, 16
    dt = 0.2 / nc
    lam = 1e-3
    nb = 25
    gpu, cpu = [], []
    for seed in range(R):
        pos, vel = inputs.sod_tube(n, seed=100 + seed)
        cfg = k.make_config(dim_pos=3, n_cells=(nc, 1, 1), bc=(WALL, PER, PER), lam=lam, dt=dt, seed=seed,
                            precision=64)
        sim = k.Simulation(cfg, pos, vel)
        R2 = oracle.contact_R2(lam, 0.0, float(n))
        sim.step(steps, want_moments=1)
        gpu.append(sim.moments()[0])
        sim.close()
        P = oracle.make_params(3, (nc, 1, 1), (0, 0, 0), (1, 1, 1), (WALL, PER, PER), R2=R2, dt=dt, seed=seed)
        p, v = pos, vel
        for s in range(steps):
            P.step = s
            p, v, best, paired, raw, der, glob, npairs = oracle.step(P, p, v)
        cpu.append(raw)
    n_l = n * 8 / 9 / 0.5
    fg = np.array([_profiles(r, nb, n_l) for r in gpu])   # R x 4 x nb
    fc = np.array([_profiles(r, nb, n_l) for r in cpu])
    outside = 0
    for f in (0, 1, 3):
        mg, mc = fg[:, f].mean(0), fc[:, f].mean(0)
        se = np.sqrt(fg[:, f].var(0, ddof=1) / R + fc[:, f].var(0, ddof=1) / R)
        outside += int((np.abs(mg - mc) > 3 * se + 1e-12).sum())
    assert outside <= 2, outside


def _profiles_p(raw, nb, dt, dim=3):
    """Coarse-grain per-c-bin raw sums of a unit box into nb output bins:
    n, u_x, T and p = n T + Sum W / (2 d V dt) (kinetic and collisional parts,
    Eqs. stress, 18, 19)."""
    k = raw.shape[0] // nb
    R = raw.reshape(nb, k, 8).sum(1)
    N = R[:, 0]
    u = R[:, 1] / N
    c2 = (R[:, 4] + R[:, 5] + R[:, 6]) / N - (R[:, 1:4] ** 2).sum(1) / N ** 2
    T = c2 / 3.0
    V = 1.0 / nb
    dens = N / V
    return np.array([dens, u, T, dens * T + R[:, 7] / (2 * dim * V * dt)])


def test_ensemble_means_match_oracle_fp32_config1_reduction():
    """The 16M-particle slab Sod tube (2000 c-bins, lambda/L = 1e-3, dt =
    0.2 dx) reduced to 1M particles on the same c-bins: binary32 device path
    against the binary64 oracle, 16 seeds per side from the same rounded
    states, 3 steps (the oracle's share of the test: about 4 s per step on 16
    cores).  Per output bin (100 bins of 20 c-bins) and field n, u, T and p
    (kinetic plus collisional) the ensemble means differ by more than 3
    combined standard errors in at most 1 % of the 400 checks (0.27 % expected
    by chance)."""
    _setup()
    import oracle
    import paper_1210_8084_gb300 as k
    from paper_1210_8084_gb300 import inputs
    n, nc, steps, R, nb = 1_000_000, 2000, 3, 16, 100
    dt, lam = 0.2 / nc, 1e-3
    lo, hi, bc = (0, 0, 0), (1, 1, 1), (WALL, PER, PER)
    R2 = oracle.contact_R2(lam, 0.0, float(n))
    gpu, cpu = [], []
    for seed in range(R):
        pos, vel = inputs.cast_state(*inputs.sod_tube(n, seed=500 + seed), np.float32, lo, hi, bc)
        cfg = k.make_config(dim_pos=3, n_cells=(nc, 1, 1), bc=bc, lam=lam, dt=dt, seed=seed, precision=32)
        sim = k.Simulation(cfg, pos, vel)
        sim.step(steps, want_moments=1)
        gpu.append(_profiles_p(sim.moments()[0], nb, dt))
        sim.close()
        P = oracle.make_params(3, (nc, 1, 1), lo, hi, bc, R2=R2, dt=dt, seed=seed)
        p, v = pos.astype(np.float64), vel.astype(np.float64)
        for s in range(steps):
            P.step = s
            p, v, best, paired, raw, der, glob, npairs = oracle.step(P, p, v)
        cpu.append(_profiles_p(raw, nb, dt))
    fg, fc = np.array(gpu), np.array(cpu)   # R x 4 x nb
    mg, mc = fg.mean(0), fc.mean(0)
    se = np.sqrt(fg.var(0, ddof=1) / R + fc.var(0, ddof=1) / R)
    outside = int((np.abs(mg - mc) > 3 * se + 1e-12).sum())
    assert outside <= 4, outside
    # the collisional part is present and the collisions are comparable
    assert np.abs(fc[:, 3] - fc[:, 0] * fc[:, 2]).max() > 0


def test_dsmc_variant_against_exact_riemann_and_poca():
    """The random-partner comparison variant (KMC_FLAG_DSMC; Sect. "Direct
    Simulation Monte Carlo Technique") and the paper's method on the same slab
    Sod tube (4M particles, 2000 c-bins, lambda/L = 1e-3, t = 0.1): relative L1
    of n, p, T against the exact Riemann solution for both.  With collision
    cells half a mean free path wide the random-partner scheme is a consistent
    Boltzmann solver here; the slab geometry penalises the closest-approach
    search (its candidates lie mostly beside a particle, design notes R19).
    The numbers are printed; the bounds guard both."""
    _setup()
    import paper_1210_8084_gb300 as k
    from paper_1210_8084_gb300 import inputs
    from analytic import riemann
    n, nc, lam = 4_000_000, 2000, 1e-3
    dt = 0.2 / nc
    steps = int(round(0.1 / dt))
    pos, vel = inputs.cast_state(*inputs.sod_tube(n, seed=77), np.float32, (0, 0, 0), (1, 1, 1), (WALL, PER, PER))
    nb = 200
    ex = riemann.sod_profile(np.linspace(0, 1, nb + 1), steps * dt, 0.5, 1.0, 1.0)
    out = {}
    for name, flags in (("dsmc", k.KMC_FLAG_DSMC), ("poca", 0)):
        sim = k.Simulation(k.make_config(dim_pos=3, n_cells=(nc, 1, 1), bc=(WALL, PER, PER), lam=lam, dt=dt, seed=5,
                                         precision=32, flags=flags), pos, vel)
        e0 = sim.moments()[2][0, 1]
        sim.step(steps, want_moments=1)
        raw, _, glob = sim.moments()
        sim.close()
        dn, u, pp, T = _profiles(raw, nb, n * 8 / 9 / 0.5)
        out[name] = [float(np.abs(q - qe).sum() / np.abs(qe).sum()) for q, qe in ((dn, ex[:, 0]), (pp, ex[:, 2]),
                                                                                (T, ex[:, 3]))]
        assert abs(glob[0, 1] / e0 - 1) < 1e-5
        print(name, "L1 n, p, T:", ["%.4f" % x for x in out[name]])
    assert max(out["dsmc"]) < 0.03, out
    assert max(out["poca"]) < 0.065, out


def test_mono_energetic_gas_relaxes_to_maxwell_on_device():
    _setup()
    from scipy import stats
    import paper_1210_8084_gb300 as k
    from paper_1210_8084_gb300 import inputs
    n, v_in = 1_000_000, 10.0
    pos, vel = inputs.periodic_box(n, seed=8, v_in=v_in)
    pos, vel = inputs.cast_state(pos, vel, np.float32, (0, 0, 0), (1, 1, 1), (PER, PER, PER))
    cfg = k.make_config(dim_pos=3, n_cells=(40, 40, 40), bc=(PER, PER, PER), lam=1e-3 / 40, dt=(1 / 40) / 60 * 2,
                        seed=8, precision=32)
    sim = k.Simulation(cfg, pos, vel)
    sim.step(60, want_moments=1)
    p, v = sim.state()
    glob = sim.moments()[2]
    sim.close()
    T = v_in ** 2 / 3
    speed = np.linalg.norm(v.astype(np.float64), axis=1)
    ks = stats.kstest(speed[::50] / math.sqrt(T), stats.chi(3).cdf)
    assert ks.pvalue > 1e-3, ks
    assert glob[0, 1] == pytest.approx(0.5 * n * v_in ** 2, rel=1e-5)


def test_noh_spherical_implosion_against_exact_solution():
    """3-D spherical Noh implosion (Sect. "Noh test"), gamma = 5/3: inside the
    shock the gas is at rest with density 64 n0 and temperature v0^2 / 3; the
    shock sits at v0 t / 3; the infall ahead of it has density n0 (1 + v0 t / r)^2."""
    _setup()
    import paper_1210_8084_gb300 as k
    from paper_1210_8084_gb300 import inputs
    from analytic import noh
    n, nc, v0 = 4_000_000, 80, 1.0
    dt = 0.2 / nc / v0
    steps = 120
    pos, vel = inputs.noh(n, seed=6, L=1.0, v0=v0, T0=1e-6)
    wall3 = (1, 1, 1)
    pos, vel = inputs.cast_state(pos, vel, np.float32, (0, 0, 0), (1, 1, 1), wall3)
    sim = k.Simulation(k.make_config(dim_pos=3, n_cells=(nc, nc, nc), bc=wall3, lam=1e-3, dt=dt, seed=6,
                                     precision=32, flags=k.KMC_FLAG_RADIAL_MOMENT), pos, vel)
    e0 = sim.moments()[2][0, 1]
    sim.step(steps, want_moments=1)
    raw, der, glob = sim.moments()
    rad = sim.radial()   # Eq. vel_r about the corner the gas falls towards
    sim.close()
    t = steps * dt
    g = 5.0 / 3.0
    rs = noh.shock_radius(t, v0, g)
    c = (np.arange(nc) + 0.5) / nc
    X, Y, Z = np.meshgrid(c, c, c, indexing="ij")
    r = np.sqrt(X ** 2 + Y ** 2 + Z ** 2).transpose(2, 1, 0).ravel()   # rows: c_x fastest
    N = raw[:, 0]
    n0 = n / 1.0
    dens = N * nc ** 3
    u = raw[:, 1:4] / np.maximum(N, 1)[:, None]
    c2 = raw[:, 4:7].sum(1) / np.maximum(N, 1) - (u ** 2).sum(1)
    inner = r < 0.6 * rs
    ahead = (r > 1.6 * rs) & (r < 2.4 * rs)
    n_in = dens[inner].sum() / inner.sum()
    T_in = (raw[inner, 4:7].sum() - (raw[inner, 1:4].sum(0) ** 2).sum() / N[inner].sum()) / N[inner].sum() / 3
    n_ahead = dens[ahead].sum() / noh.profile(r[ahead], t, v0, n0, g, 3)[0].sum()
    print(f"Noh: n_in/n0 {n_in / n0:.2f} (64), T_in {T_in:.3f} ({(g - 1) * v0 ** 2 / 2:.3f}), n_ahead/exact {n_ahead:.3f}")
    assert abs(n_in / n0 / noh.shocked_density(1.0, g, 3) - 1) < 0.15
    assert abs(T_in / ((g - 1) * 0.5 * v0 ** 2) - 1) < 0.15
    assert abs(n_ahead - 1) < 0.1
    # radial velocity (Eq. vel_r): at rest inside the shock, -v0 in the infall ahead of it
    vr_in = rad[inner, 0].sum() / N[inner].sum()
    vr_ahead = rad[ahead, 0].sum() / N[ahead].sum()
    print(f"Noh: v_r inside {vr_in:.4f} (0), ahead {vr_ahead:.4f} ({-v0})")
    assert abs(vr_in) < 0.05 * v0
    assert abs(vr_ahead / -v0 - 1) < 0.05
    # shock position: the density falls below half of the plateau between 0.8 and 1.25 r_s
    shells = np.linspace(0.0, 2 * rs, 41)
    idx = np.digitize(r, shells) - 1
    prof = np.array([dens[idx == i].mean() if np.any(idx == i) else np.nan for i in range(40)])
    mid = 0.5 * (shells[1:] + shells[:-1])
    half = mid[np.nanargmax(prof < 0.5 * n_in * (1 + 1e-9))] if np.any(prof < 0.5 * n_in) else np.inf
    assert 0.8 * rs < half < 1.25 * rs, (half, rs)
    assert abs(glob[0, 1] / e0 - 1) < 1e-5


def test_sod_2d_with_2d_velocities_matches_gamma_2():
    """The paper's 2-D Sod set-up: square c-bins (2000 x 500 over 1 x 1/4, 20
    per c-bin), velocities in the plane (f = 2, gamma = 2), lambda/L = 1e-3,
    t = 0.1, against the exact Riemann solution with gamma = 2: relative L1 of
    n, p, T within 2.5 % and the star state within 2 % (with 3-D velocities
    the star velocity sits 2.5 % low)."""
    _setup()
    import paper_1210_8084_gb300 as k
    from paper_1210_8084_gb300 import inputs
    from analytic import riemann
    ncx, ncy, ppc, steps = 2000, 500, 20, 1000
    hi = (1.0, 0.25, 1.0)
    n = ppc * ncx * ncy
    dt = 0.2 / ncx
    bc = (WALL, PER, PER)
    pos, vel = inputs.sod_tube(n, seed=5, hi=hi, dim_pos=2, vel_dim=2)
    pos, vel = inputs.cast_state(pos, vel, np.float32, (0, 0, 0), hi, bc)
    sim = k.Simulation(k.make_config(dim_pos=2, n_cells=(ncx, ncy, 1), hi=hi, bc=bc, lam=1e-3, dt=dt, seed=5,
                                     precision=32, flags=k.KMC_FLAG_VELOCITY_2D), pos, vel)
    sim.step(steps, want_moments=1)
    raw, der, glob = sim.moments()
    sim.close()
    t = steps * dt
    nb = 200
    rx = raw.reshape(ncy, ncx, 8).sum(0)
    R = rx.reshape(nb, ncx // nb, 8).sum(1)
    N = R[:, 0]
    u = R[:, 1] / N
    c2 = (R[:, 4] + R[:, 5]) / N - (R[:, 1] ** 2 + R[:, 2] ** 2) / N ** 2
    T = c2 / 2.0
    n_l = n * 8 / 9 / 0.5
    dn = N * nb / n_l
    p = dn * T
    ex = riemann.sod_profile(np.linspace(0, 1, nb + 1), t, 0.5, 1.0, 1.0, gamma=2.0)
    l1 = {name: float(np.abs(q - qe).sum() / np.abs(qe).sum())
          for name, q, qe in (("n", dn, ex[:, 0]), ("u", u, ex[:, 1]), ("p", p, ex[:, 2]), ("T", T, ex[:, 3]))}
    xc = (np.arange(nb) + 0.5) / nb
    star = (xc > 0.51) & (xc < 0.54)
    stat = {name: float(q[star].mean() / qe[star].mean() - 1)
            for name, q, qe in (("n", dn, ex[:, 0]), ("u", u, ex[:, 1]), ("p", p, ex[:, 2]), ("T", T, ex[:, 3]))}
    print("Sod 2-D velocities L1:", l1, "star:", stat)
    assert l1["n"] <= 0.025 and l1["p"] <= 0.025 and l1["T"] <= 0.025, l1
    assert all(abs(v) < 0.02 for v in stat.values()), stat


def test_sedov_blast_radius_grows_as_t_to_two_fifths():
    """3-D Sedov-Taylor blast (Sect. "Sedov test"): absorbing walls, adaptive
    timestep, energy deposited as speed v_blast inside 2 c-bins of the centre.
    The shock (the radius of the density peak) grows as (E t^2 / n0)^(1/5):
    between two times its radius scales as (t2 / t1)^(2/5), whatever the
    constant alpha; the peak is compressed above 1.8 n0 (4 n0 for an
    infinitely thin shock); the peak sits at the similarity solution's radius
    (E t^2 / (alpha n0))^(1/5), alpha from oracle/sedov.py."""
    _setup()
    import paper_1210_8084_gb300 as k
    from paper_1210_8084_gb300 import inputs
    n, nc = 8_000_000, 100
    A = k.KMC_BC_ABSORB
    pos, vel = inputs.sedov(n, seed=7, r_blast=2.0 / nc, v_blast=85.0)
    pos, vel = inputs.cast_state(pos, vel, np.float32, (0, 0, 0), (1, 1, 1), (1, 1, 1))
    sim = k.Simulation(k.make_config(dim_pos=3, n_cells=(nc, nc, nc), bc=(A, A, A), lam=1e-3, dt=1.0, seed=7,
                                     precision=32, flags=k.KMC_FLAG_ADAPTIVE_DT), pos, vel)
    c = (np.arange(nc) + 0.5) / nc - 0.5
    X, Y, Z = np.meshgrid(c, c, c, indexing="ij")
    r = np.sqrt(X ** 2 + Y ** 2 + Z ** 2).ravel()
    shells = np.arange(0.0, 0.5, 1.0 / nc)
    idx = np.digitize(r, shells) - 1
    n0 = float(n)

    def peak():
        raw = sim.moments()[0]
        dens = raw[:, 0] * nc ** 3 / n0
        prof = np.array([dens[idx == i].mean() for i in range(len(shells) - 1)])
        i = int(np.argmax(prof[3:])) + 3
        return 0.5 * (shells[i] + shells[i + 1]), prof[i]

    out = []
    for t_goal in (0.05, 0.1):
        while sim.info().time < t_goal:
            sim.step(25, want_moments=1)
        t = sim.info().time
        rp, npk = peak()
        out.append((t, rp, npk))
    glob = sim.moments()[2]
    sim.close()
    (t1, r1, n1), (t2, r2, n2) = out
    from analytic import sedov
    E = 0.5 * float((vel.astype(np.float64) ** 2).sum())
    al = sedov.alpha(3, 5.0 / 3.0)
    rs1, rs2 = (sedov.shock_radius(E, n0, t, alpha_value=al) for t in (t1, t2))
    print(f"Sedov: t {t1:.4f} r {r1:.3f} (exact {rs1:.3f}) peak {n1:.2f}; t {t2:.4f} r {r2:.3f} "
          f"(exact {rs2:.3f}) peak {n2:.2f}; live {glob[0, 0]:.0f}")
    assert abs((r2 / r1) / (t2 / t1) ** 0.4 - 1) < 0.08
    # the density peak sits at the similarity solution's shock radius (within a few c-bins)
    assert abs(r1 / rs1 - 1) < 0.08 and abs(r2 / rs2 - 1) < 0.08
    assert n1 > 1.8 and n2 > 1.8
    assert 0.1 < r1 < r2 < 0.45


def test_noh_cylindrical_2d_reaches_nine_times_n0():
    """The paper's 2-D cylindrical Noh test with 2-D velocities (gamma = 2):
    the gas inside the shock at rest with density 9 n0 (the value the paper
    reports its runs approach) and temperature v0^2 / 2, the shock at v0 t / 2,
    the infall ahead of it at n0 (1 + v0 t / r)."""
    _setup()
    import paper_1210_8084_gb300 as k
    from paper_1210_8084_gb300 import inputs
    from analytic import noh
    n, nc, v0 = 5_000_000, 500, 1.0
    dt = 0.2 / nc / v0
    steps = 750
    pos, vel = inputs.noh(n, seed=9, dim_pos=2, L=1.0, v0=v0, T0=1e-6, vel_dim=2)
    bc = (1, 1, 0)
    pos, vel = inputs.cast_state(pos, vel, np.float32, (0, 0, 0), (1, 1, 1), bc)
    sim = k.Simulation(k.make_config(dim_pos=2, n_cells=(nc, nc, 1), bc=bc, lam=1e-3, dt=dt, seed=9, precision=32,
                                     flags=k.KMC_FLAG_VELOCITY_2D | k.KMC_FLAG_RADIAL_MOMENT), pos, vel)
    sim.step(steps, want_moments=1)
    raw = sim.moments()[0]
    rad = sim.radial()   # Eq. vel_r about the corner (the cylinder axis)
    sim.close()
    t = steps * dt
    g = 2.0
    rs = noh.shock_radius(t, v0, g)
    c = (np.arange(nc) + 0.5) / nc
    X, Y = np.meshgrid(c, c, indexing="xy")      # rows: c_x fastest
    r = np.sqrt(X ** 2 + Y ** 2).ravel()
    N = raw[:, 0]
    dens = N * nc ** 2 / float(n)
    inner = r < 0.6 * rs
    ahead = (r > 1.6 * rs) & (r < 2.4 * rs)
    Nin = N[inner].sum()
    c2 = (raw[inner, 4:6].sum() - (raw[inner, 1:3].sum(0) ** 2).sum() / Nin) / Nin
    T_in = c2 / 2.0
    n_in = dens[inner].mean()
    n_ahead = dens[ahead].sum() / noh.profile(r[ahead], t, v0, 1.0, g, 2)[0].sum()
    print(f"Noh 2-D: n_in/n0 {n_in:.2f} (9), T_in {T_in:.3f} (0.5), n_ahead/exact {n_ahead:.3f}")
    assert abs(n_in / noh.shocked_density(1.0, g, 2) - 1) < 0.1
    assert abs(T_in / ((g - 1) * 0.5 * v0 ** 2) - 1) < 0.1
    assert abs(n_ahead - 1) < 0.05
    vr_in = rad[inner, 0].sum() / N[inner].sum()
    vr_ahead = rad[ahead, 0].sum() / N[ahead].sum()
    print(f"Noh 2-D: v_r inside {vr_in:.4f} (0), ahead {vr_ahead:.4f} ({-v0})")
    assert abs(vr_in) < 0.05 * v0
    assert abs(vr_ahead / -v0 - 1) < 0.05
