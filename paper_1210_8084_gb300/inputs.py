"""Seeded synthetic initial states and workload definitions.

This module holds no arithmetic of the method: it only draws initial
conditions (uniform positions, Maxwellian or mono-energetic velocities) with
numpy's PCG64 and describes the benchmark workloads.  Both the CUDA path and
the CPU oracle are fed from here.

Recipes (units m = 1, k_B = 1, v_th = sqrt(T_left / m) = 1):
  * Sod tube (Sect. "Sod test", Eq. np_sod): box split at x = split, left and
    right halves with number-density ratio 8 : 1 and pressure ratio 10 : 1, so
    T_left = 1 and T_right = 0.8; particle counts follow density x volume
    (N_left = round(8 N / 9) for equal halves); positions uniform in each half;
    each velocity component N(0, T); bulk velocity 0.
  * Four-quadrant 2-D Riemann problem: quadrant densities 1, 0.5, 0.25, 0.125
    counter-clockwise from (x > 1/2, y > 1/2), counts proportional to density,
    all at rest with T = 1; 3-D velocities, z = 0.
  * Homogeneous periodic box: uniform positions, Maxwellian (T) or
    mono-energetic (|v| = v_in, isotropic directions, Sect. "Equilibration").
  * Noh implosion (Sect. "Noh test"): uniform density, radial inflow v0 towards
    the corner at the origin, cold (T0 << v0^2), reflective walls.
  * Sedov-Taylor blast (Sect. "Sedov test"): uniform density, speed v0 in
    random directions, v_blast inside r_blast of the centre, absorbing walls.
"""
import math
import os
from concurrent.futures import ThreadPoolExecutor

import numpy as np

WALL = 1
PERIODIC = 0


def _rng(seed, stream):
    return np.random.Generator(np.random.PCG64(np.random.SeedSequence([int(seed), int(stream)])))


# Above this many particles a Sod tube is drawn in blocks of CHUNK particles,
# block k from its own stream (seed, stream, k), on all host cores; smaller
# tubes keep the single-stream recipe.
CHUNKED_ABOVE = 1 << 25
CHUNK = 1 << 22


def _sod_tube_chunked(n, seed, lo, hi, split, rho, p, dim_pos, vel_dim, dtype):
    vol_l = (split - lo[0]) / (hi[0] - lo[0])
    w_l, w_r = rho[0] * vol_l, rho[1] * (1.0 - vol_l)
    n_l = int(round(n * w_l / (w_l + w_r)))
    T = (p[0] / rho[0], p[1] / rho[1])
    pos = np.empty((n, 3), dtype=dtype)
    vel = np.empty((n, 3), dtype=dtype)

    def block(k):
        a, b = k * CHUNK, min(n, (k + 1) * CHUNK)
        idx = np.arange(a, b)
        left = idx < n_l
        g = np.random.Generator(np.random.PCG64(np.random.SeedSequence([int(seed), 1, k])))
        x = np.where(left, g.uniform(lo[0], split, b - a), g.uniform(split, hi[0], b - a))
        x = np.clip(x, lo[0], hi[0])
        P = np.empty((b - a, 3))
        P[:, 0] = x
        for d in (1, 2):
            y = g.uniform(lo[d], hi[d], b - a)
            P[:, d] = np.where(y >= hi[d], lo[d], y)
        if dim_pos == 2:
            P[:, 2] = 0.0
        gv = np.random.Generator(np.random.PCG64(np.random.SeedSequence([int(seed), 2, k])))
        V = gv.normal(0.0, 1.0, (b - a, 3)) * np.where(left, math.sqrt(T[0]), math.sqrt(T[1]))[:, None]
        if vel_dim == 2:
            V[:, 2] = 0.0
        Pc = P.astype(dtype)
        for d in (1, 2):   # a periodic coordinate that rounds up to hi is the point lo
            Pc[:, d] = np.where(Pc[:, d] >= dtype(hi[d]), dtype(lo[d]), Pc[:, d])
        pos[a:b] = Pc
        vel[a:b] = V.astype(dtype)

    n_blocks = (n + CHUNK - 1) // CHUNK
    with ThreadPoolExecutor(max_workers=min(n_blocks, os.cpu_count() or 1)) as ex:
        list(ex.map(block, range(n_blocks)))
    return pos, vel


def sod_tube(n, seed=0, lo=(0.0, 0.0, 0.0), hi=(1.0, 1.0, 1.0), split=0.5, rho=(1.0, 0.125), p=(1.0, 0.1),
             dim_pos=3, vel_dim=3, dtype=np.float64):
    """(pos, vel) arrays of shape (n, 3), left particles first, in dtype
    (rounded from binary64 as cast_state rounds, y and z periodic).
    vel_dim = 2: velocities in the (x, y) plane (v_z = 0).  Tubes of more than
    CHUNKED_ABOVE particles are drawn in independent blocks in parallel."""
    if n > CHUNKED_ABOVE:
        return _sod_tube_chunked(n, seed, np.asarray(lo, dtype=np.float64), np.asarray(hi, dtype=np.float64),
                                 split, rho, p, dim_pos, vel_dim, dtype)
    if dtype is not np.float64:
        pos, vel = sod_tube(n, seed, lo, hi, split, rho, p, dim_pos, vel_dim)
        return cast_state(pos, vel, dtype, lo, hi, (WALL, PERIODIC, PERIODIC))
    lo = np.asarray(lo, dtype=np.float64)
    hi = np.asarray(hi, dtype=np.float64)
    vol_l = (split - lo[0]) / (hi[0] - lo[0])
    vol_r = 1.0 - vol_l
    w_l = rho[0] * vol_l
    w_r = rho[1] * vol_r
    n_l = int(round(n * w_l / (w_l + w_r)))
    n_r = n - n_l
    T = (p[0] / rho[0], p[1] / rho[1])
    g = _rng(seed, 1)
    pos = np.empty((n, 3))
    vel = np.empty((n, 3))
    for (a, b, m, k) in ((0, n_l, lo[0], split), (n_l, n, split, hi[0])):
        cnt = b - a
        pos[a:b, 0] = g.uniform(m, k, cnt)
        for d in (1, 2):
            pos[a:b, d] = g.uniform(lo[d], hi[d], cnt)
    # guard the open upper end of periodic dimensions and the split point
    pos[:, 0] = np.clip(pos[:, 0], lo[0], hi[0])
    for d in (1, 2):
        pos[:, d] = np.where(pos[:, d] >= hi[d], lo[d], pos[:, d])
    if dim_pos == 2:
        pos[:, 2] = 0.0
    gv = _rng(seed, 2)
    vel[:n_l] = gv.normal(0.0, math.sqrt(T[0]), (n_l, 3))
    vel[n_l:] = gv.normal(0.0, math.sqrt(T[1]), (n_r, 3))
    if vel_dim == 2:
        vel[:, 2] = 0.0
    return pos, vel


def quadrants_2d(n, seed=0, densities=(1.0, 0.5, 0.25, 0.125), T=1.0):
    """Unit square, quadrant order Q1 (x>1/2,y>1/2), Q2 (x<1/2,y>1/2), Q3, Q4."""
    w = np.asarray(densities, dtype=np.float64)
    counts = np.floor(n * w / w.sum()).astype(np.int64)
    counts[0] += n - counts.sum()
    corners = [(0.5, 0.5), (0.0, 0.5), (0.0, 0.0), (0.5, 0.0)]
    g = _rng(seed, 1)
    pos = np.zeros((n, 3))
    a = 0
    for (cx, cy), c in zip(corners, counts):
        pos[a:a + c, 0] = g.uniform(cx, cx + 0.5, c)
        pos[a:a + c, 1] = g.uniform(cy, cy + 0.5, c)
        a += c
    vel = _rng(seed, 2).normal(0.0, math.sqrt(T), (n, 3))
    return pos, vel


def periodic_box(n, seed=0, lo=(0.0, 0.0, 0.0), hi=(1.0, 1.0, 1.0), T=1.0, v_in=None, vel_dim=3):
    """Uniform positions; Maxwellian (per-component variance T) or
    mono-energetic (|v| = v_in) velocities, isotropic in vel_dim components."""
    g = _rng(seed, 1)
    lo = np.asarray(lo, dtype=np.float64)
    hi = np.asarray(hi, dtype=np.float64)
    pos = lo + (hi - lo) * g.random((n, 3))
    pos = np.where(pos >= hi, lo, pos)
    gv = _rng(seed, 2)
    if v_in is None:
        vel = gv.normal(0.0, math.sqrt(T), (n, 3))
        if vel_dim == 2:
            vel[:, 2] = 0.0
    else:
        d = gv.normal(0.0, 1.0, (n, 3))
        if vel_dim == 2:
            d[:, 2] = 0.0
        d /= np.linalg.norm(d, axis=1, keepdims=True)
        vel = v_in * d
    return pos, vel


def noh(n, seed=0, dim_pos=3, L=1.0, v0=1.0, T0=1e-6, vel_dim=3):
    """Noh implosion (Sect. "Noh test"): uniform positions in [0, L]^dim with
    the origin at the corner (walls at 0 are the symmetry planes), velocity
    -v0 r_hat towards the origin in the position dimensions plus a small
    Maxwellian spread of temperature T0 per component ("zero pressure");
    vel_dim = 2: velocities in the (x, y) plane."""
    g = _rng(seed, 1)
    pos = np.zeros((n, 3))
    pos[:, :dim_pos] = L * g.random((n, dim_pos))
    pos = np.minimum(pos, L)
    r = np.linalg.norm(pos[:, :dim_pos], axis=1, keepdims=True)
    rhat = np.zeros((n, 3))
    rhat[:, :dim_pos] = pos[:, :dim_pos] / np.maximum(r, 1e-300)
    vel = -v0 * rhat + _rng(seed, 2).normal(0.0, math.sqrt(T0), (n, 3))
    if vel_dim == 2:
        vel[:, 2] = 0.0
    return pos, vel


def sedov(n, seed=0, dim_pos=3, L=1.0, v0=1e-3, r_blast=0.02, v_blast=85.0):
    """Sedov-Taylor blast (Sect. "Sedov test"): uniform positions in [0, L]^dim,
    velocities of magnitude v0 in random directions, except |v| = v_blast
    inside r_blast of the centre (the energy deposition)."""
    g = _rng(seed, 1)
    pos = np.zeros((n, 3))
    pos[:, :dim_pos] = L * g.random((n, dim_pos))
    pos = np.minimum(pos, L)
    d = _rng(seed, 2).normal(0.0, 1.0, (n, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    r = np.linalg.norm(pos[:, :dim_pos] - 0.5 * L, axis=1)
    speed = np.where(r <= r_blast, v_blast, v0)
    return pos, speed[:, None] * d


def cast_state(pos, vel, dtype, lo, hi, bc):
    """Round a state to the working precision; a periodic coordinate that
    rounds up to the upper face is the same point as the lower face."""
    pos = np.ascontiguousarray(pos, dtype=dtype).copy()
    vel = np.ascontiguousarray(vel, dtype=dtype)
    for d in range(3):
        if bc[d] == PERIODIC:
            h = dtype(hi[d])
            pos[:, d] = np.where(pos[:, d] >= h, dtype(lo[d]), pos[:, d])
    return pos, vel


def log_uniform_instances(n_instances, seed=0, n_range=(50_000, 2_000_000), lam_range=(1e-4, 1.0)):
    """Per-instance particle counts and mean free paths, log-uniform."""
    g = _rng(seed, 3)
    ns = np.exp(g.uniform(math.log(n_range[0]), math.log(n_range[1]), n_instances)).astype(np.int64)
    lams = np.exp(g.uniform(math.log(lam_range[0]), math.log(lam_range[1]), n_instances))
    return ns, lams


# Workloads: the shapes of the paper's shock-tube / Riemann set-ups scaled to
# one GB300.  dt = 0.2 * cell width / v_th with v_th = 1.
WORKLOADS = {
    "sod1d_fp64_200k": dict(
        kind="sod", n=200_000, dim_pos=3, n_cells=(200, 1, 1), lo=(0, 0, 0), hi=(1, 1, 1),
        bc=(WALL, PERIODIC, PERIODIC), lam=1e-3, dt=0.2 / 200, steps=200, precision=64, seed=0),
    "sod1d_fp32_16M": dict(
        kind="sod", n=16_000_000, dim_pos=3, n_cells=(2000, 1, 1), lo=(0, 0, 0), hi=(1, 1, 1),
        bc=(WALL, PERIODIC, PERIODIC), lam=1e-3, lam_sweep=(1e-4, 1e-3, 1e-2, 1e-1, 1.0),
        dt=0.2 / 2000, steps=1000, precision=32, seed=0),
    "quadrant2d_fp32_64M": dict(
        kind="quadrants", n=64_000_000, dim_pos=2, n_cells=(512, 512, 1), lo=(0, 0, 0), hi=(1, 1, 1),
        bc=(WALL, WALL, PERIODIC), lam=5e-4, dt=0.2 / 512, steps=500, precision=32, seed=0),
    "sod1d_batched_256": dict(
        kind="batched_sod", n_instances=256, n_range=(50_000, 2_000_000), lam_range=(1e-4, 1.0),
        dim_pos=3, n_cells=(200, 1, 1), lo=(0, 0, 0), hi=(1, 1, 1), bc=(WALL, PERIODIC, PERIODIC),
        dt=0.2 / 200, steps=400, precision=32, seed=0),
    "sod3d_fp32_16M": dict(     # the 512M case's cubic c-bins and occupancy (~122 per c-bin) on 16M particles
        kind="sod", n=16_000_000, dim_pos=3, n_cells=(512, 16, 16), lo=(0, 0, 0), hi=(1, 1 / 32, 1 / 32),
        bc=(WALL, PERIODIC, PERIODIC), lam=2e-4, dt=0.2 / 512, steps=300, precision=32, seed=0),
    "sod3d_fp32_512M": dict(
        kind="sod", n=512_000_000, dim_pos=3, n_cells=(1024, 64, 64), lo=(0, 0, 0), hi=(1, 1 / 16, 1 / 16),
        bc=(WALL, PERIODIC, PERIODIC), lam=2e-4, dt=0.2 / 1024, steps=300, precision=32, seed=0),
}


def make_state(w, n=None, seed=None, dtype=np.float64):
    """Initial (pos, vel) of a workload dict (optionally resized), in dtype
    (rounded as cast_state rounds)."""
    n = w["n"] if n is None else n
    seed = w["seed"] if seed is None else seed
    if w["kind"] == "sod":
        return sod_tube(n, seed, lo=w["lo"], hi=w["hi"], dim_pos=w["dim_pos"], dtype=dtype)
    if dtype is not np.float64:
        return cast_state(*make_state(w, n, seed), dtype, w["lo"], w["hi"], w["bc"])
    if w["kind"] == "quadrants":
        return quadrants_2d(n, seed)
    raise ValueError(w["kind"])
