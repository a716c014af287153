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
    cfg = k.make_config(**cfg_kwargs, flags=k.KMC_FLAG_RECORD)
    sim = k.Simulation(cfg, pos, vel)
    sim.step(1)
    best, _ = sim.partners()
    sim.close()
    return best


def test_noalloc_search_matches_allocating_path_on_two_calls():
    _setup()
    import torch
    import paper_1210_8084_gb300 as k
    from paper_1210_8084_gb300 import inputs

    cases = [
        # (n, lambda, c-bins, seed, precision): the second call is smaller, so
        # leftovers of the first call in the shared array would show
        (60_000, 1e-3, (60, 1, 1), 1, 32),
        (23_457, 1e-2, (25, 1, 1), 2, 32),
    ]
    for n, lam, cells, seed, prec in cases:
        dtype = np.float32 if prec == 32 else np.float64
        pos, vel = inputs.sod_tube(n, seed=seed)
        pos, vel = inputs.cast_state(pos, vel, dtype, (0, 0, 0), (1, 1, 1), (1, 0, 0))
        kw = dict(dim_pos=3, n_cells=cells, bc=(k.KMC_BC_WALL, k.KMC_BC_PERIODIC, k.KMC_BC_PERIODIC),
                  lam=lam, dt=0.2 / cells[0], seed=seed, precision=prec)
        ref = _handle_best(k, kw, pos, vel)

        cfg = k.make_config(**kw)
        pos_d = torch.from_numpy(pos).cuda()
        vel_d = torch.from_numpy(vel).cuda()
        best_d = torch.full((n,), -7, dtype=torch.int32, device="cuda")
        torch.cuda.synchronize()
        rc = k.kmc_find_partners_noalloc(cfg, n, pos_d, vel_d, best_d)
        assert rc == k.KMC_OK
        torch.cuda.synchronize()
        got = best_d.cpu().numpy()
        assert (ref >= 0).sum() > n // 20
        assert np.array_equal(got, ref)


def test_noalloc_rejects_sizes_beyond_its_array():
    _setup()
    import paper_1210_8084_gb300 as k
    cfg = k.make_config(dim_pos=3, n_cells=(10, 1, 1), lam=1e-3, dt=1e-3, precision=32)
    rc = k.kmc_find_partners_noalloc(cfg, k.KMC_STATIC_MAX_PARTICLES + 1, 1, 1, 1)
    assert rc == k.KMC_ERANGE
    big = k.make_config(dim_pos=3, n_cells=(2000, 1, 1), lam=1e-3, dt=1e-3, precision=32, sub_cells=(1, 100, 100))
    rc = k.kmc_find_partners_noalloc(big, 10, 1, 1, 1)
    assert rc == k.KMC_ERANGE
