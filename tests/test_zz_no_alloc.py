"""The closest-candidate search that allocates nothing.

Some callers may not allocate device memory themselves or through this
library: a host framework that owns all device memory through its own pool,
code running under a fixed device-memory budget, or a loop where cudaMalloc's
implicit device synchronisation is not acceptable.  For them
kmc_find_partners_noalloc keeps every scratch buffer in one fixed device array
of the library.  This checks, through the C ABI, that two calls in a row give
exactly the closest candidates the allocating handle path gives
(kmc_init + one kmc_step with KMC_FLAG_RECORD + kmc_get_partners) for the same
states: integer results, so bit for bit.  The file sorts last so a run that
stops at the first failure has already run every other test.
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


def _handle_best(k, cfg_kwargs, pos, vel):
    kw = dict(cfg_kwargs)
    kw["flags"] = kw.get("flags", 0) | k.KMC_FLAG_RECORD
    cfg = k.make_config(**kw)
    sim = k.Simulation(cfg, pos, vel)
    sim.step(1)
    best, _ = sim.partners()
    sim.close()
    return best


def _state(inputs, n, seed, dim, cells, dtype):
    if dim == 2:
        pos, vel = inputs.quadrants_2d(n, seed=seed)
        return inputs.cast_state(pos, vel, dtype, (0, 0, 0), (1, 1, 1), (1, 1, 0))
    pos, vel = inputs.sod_tube(n, seed=seed)
    return inputs.cast_state(pos, vel, dtype, (0, 0, 0), (1, 1, 1), (1, 0, 0))


def test_noalloc_search_matches_allocating_path_on_two_calls():
    _setup()
    import torch
    import paper_1210_8084_gb300 as k
    from paper_1210_8084_gb300 import inputs

    W, P = k.KMC_BC_WALL, k.KMC_BC_PERIODIC
    cases = [
        # (n, lambda, c-bins, seed, precision, dim, sub_cells, flags): consecutive calls on the
        # shared array, smaller after larger, so leftovers of a call would show
        (60_000, 1e-3, (60, 1, 1), 1, 32, 3, (0, 0, 0), 0),
        (23_457, 1e-2, (25, 1, 1), 2, 32, 3, (0, 0, 0), 0),
        (40_000, 1e-3, (40, 1, 1), 3, 64, 3, (0, 0, 0), 0),
        (50_000, 1e-3, (50, 1, 1), 4, 32, 3, (1, 8, 8), 0),
        (30_000, 5e-4, (30, 30, 1), 5, 32, 2, (0, 0, 0), 0),
        (30_000, 1e-3, (30, 1, 1), 6, 32, 3, (0, 0, 0), k.KMC_FLAG_ADAPTIVE_DT),
        # at the particle limit in binary64 (the largest carving of the array), subdivided
        (k.KMC_STATIC_MAX_PARTICLES, 1e-3, (256, 1, 1), 7, 64, 3, (1, 16, 16), 0),
        (1_001, 1e-2, (10, 1, 1), 8, 64, 3, (0, 0, 0), 0),
    ]
    for n, lam, cells, seed, prec, dim, sub, flags in cases:
        dtype = np.float32 if prec == 32 else np.float64
        pos, vel = _state(inputs, n, seed, dim, cells, dtype)
        bc = (W, W, P) if dim == 2 else (W, P, P)
        kw = dict(dim_pos=dim, n_cells=cells, bc=bc, lam=lam, dt=0.2 / cells[0], seed=seed, precision=prec,
                  sub_cells=sub, flags=flags)
        ref = _handle_best(k, kw, pos, vel)

        cfg = k.make_config(**kw)
        pos_d = torch.from_numpy(pos).cuda()
        vel_d = torch.from_numpy(vel).cuda()
        for call in range(2):
            best_d = torch.full((n,), -7, dtype=torch.int32, device="cuda")
            torch.cuda.synchronize()
            rc = k.kmc_find_partners_noalloc(cfg, n, pos_d, vel_d, best_d)
            assert rc == k.KMC_OK, (n, rc)
            torch.cuda.synchronize()
            got = best_d.cpu().numpy()
            assert (ref >= 0).sum() > n // 20, (n, (ref >= 0).sum())
            assert np.array_equal(got, ref), (n, prec, dim, sub, flags, call)


def test_noalloc_rejects_sizes_beyond_its_array():
    _setup()
    import paper_1210_8084_gb300 as k
    cfg = k.make_config(dim_pos=3, n_cells=(10, 1, 1), lam=1e-3, dt=1e-3, precision=32)
    rc = k.kmc_find_partners_noalloc(cfg, k.KMC_STATIC_MAX_PARTICLES + 1, 1, 1, 1)
    assert rc == k.KMC_ERANGE
    big = k.make_config(dim_pos=3, n_cells=(2000, 1, 1), lam=1e-3, dt=1e-3, precision=32, sub_cells=(1, 100, 100))
    rc = k.kmc_find_partners_noalloc(big, 10, 1, 1, 1)
    assert rc == k.KMC_ERANGE


def test_noalloc_checks_the_configuration_as_kmc_init_does():
    _setup()
    import paper_1210_8084_gb300 as k
    bad = [
        k.make_config(dim_pos=3, n_cells=(10, 1, 1), lam=1e-3, dt=1e-3, flags=1 << 9),
        k.make_config(dim_pos=3, n_cells=(10, 1, 1), lam=1e-3, dt=1e-3, flags=k.KMC_FLAG_VELOCITY_2D),
        k.make_config(dim_pos=3, n_cells=(10, 1, 1), sigma=float("inf"), dt=1e-3),
        k.make_config(dim_pos=3, n_cells=(10, 1, 1), lam=1e-3, dt=0.0),
        k.make_config(dim_pos=3, n_cells=(10, 1, 1), lam=1e-3, dt=1e-3, bc=(3, 0, 0)),
    ]
    for cfg in bad:
        assert k.kmc_find_partners_noalloc(cfg, 10, 1, 1, 1) == k.KMC_EINVAL
