"""CPU oracle of the kinetic Monte Carlo step (test infrastructure only).

Only the test-suite, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  It wraps ``kmc_oracle.c`` (plain C,
FP64, optional binary32 decisions) through ctypes.  It shares no code with the
CUDA library.  (The exact solutions of the test problems live in ``analytic``.)
"""
import ctypes
import os

import numpy as np

from . import build as _build

_HERE = os.path.dirname(os.path.abspath(__file__))
_lib = None


class Params(ctypes.Structure):
    _fields_ = [
        ("dim", ctypes.c_int),
        ("n_cells", ctypes.c_int * 3),
        ("lo", ctypes.c_double * 3),
        ("hi", ctypes.c_double * 3),
        ("bc", ctypes.c_int * 3),
        ("R2", ctypes.c_double),
        ("dt", ctypes.c_double),
        ("seed", ctypes.c_uint64),
        ("step", ctypes.c_uint32),
        ("decide32", ctypes.c_int),
        ("vel_dim", ctypes.c_int),
    ]


def lib():
    global _lib
    if _lib is None:
        path = _build.build()
        L = ctypes.CDLL(path)
        P = ctypes.POINTER(Params)
        dp = ctypes.POINTER(ctypes.c_double)
        ip = ctypes.POINTER(ctypes.c_int32)
        up = ctypes.POINTER(ctypes.c_uint32)
        i64 = ctypes.c_int64
        L.orc_philox4x32_10.argtypes = [up, up, up]
        L.orc_philox4x32_10.restype = None
        L.orc_contact_R2.argtypes = [ctypes.c_double, ctypes.c_double, ctypes.c_double]
        L.orc_contact_R2.restype = ctypes.c_double
        L.orc_set_threads.argtypes = [ctypes.c_int]
        L.orc_set_threads.restype = ctypes.c_int
        L.orc_adaptive_dt.argtypes = [P, i64, dp, ctypes.c_double]
        L.orc_adaptive_dt.restype = ctypes.c_double
        L.orc_cell_keys.argtypes = [P, i64, dp, ip, ip]
        L.orc_cell_keys.restype = None
        L.orc_pair_test.argtypes = [P, dp, dp, dp, dp, dp]
        L.orc_pair_test.restype = ctypes.c_int
        for name in ("orc_best_partners", "orc_best_partners_brute"):
            f = getattr(L, name)
            f.argtypes = [P, i64, dp, dp, ip]
            f.restype = i64
        L.orc_candidate_count.argtypes = [P, i64, dp]
        L.orc_candidate_count.restype = i64
        L.orc_mutual_pairs.argtypes = [i64, ip, ip]
        L.orc_mutual_pairs.restype = i64
        L.orc_collide_move.argtypes = [P, i64, dp, dp, ip, dp, dp, dp, ip]
        L.orc_collide_move.restype = None
        L.orc_collide_move_ids.argtypes = [P, i64, dp, dp, ip, ctypes.c_void_p, dp, dp, dp, ip]
        L.orc_collide_move_ids.restype = None
        L.orc_moments.argtypes = [P, i64, dp, dp, dp, dp, dp, dp]
        L.orc_moments.restype = None
        L.orc_dsmc_collide.argtypes = [P, i64, dp, dp, ip]
        L.orc_dsmc_collide.restype = i64
        L.orc_radial.argtypes = [P, i64, dp, dp, dp, dp]
        L.orc_radial.restype = None
        L.orc_step.argtypes = [P, i64, dp, dp, ip, ip, dp, dp, dp]
        L.orc_step.restype = i64
        _lib = L
    return _lib


def _d(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double)) if a is not None else None


def _i(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)) if a is not None else None


def make_params(dim, n_cells, lo, hi, bc, R2, dt, seed=0, step=0, decide32=False, vel_dim=3):
    p = Params()
    p.dim = int(dim)
    for d in range(3):
        p.n_cells[d] = int(n_cells[d]) if d < len(n_cells) else 1
        p.lo[d] = float(lo[d]) if d < len(lo) else 0.0
        p.hi[d] = float(hi[d]) if d < len(hi) else 1.0
        p.bc[d] = int(bc[d]) if d < len(bc) else 0
    p.R2 = float(R2)
    p.dt = float(dt)
    p.seed = int(seed) & 0xFFFFFFFFFFFFFFFF
    p.step = int(step) & 0xFFFFFFFF
    p.decide32 = 1 if decide32 else 0
    p.vel_dim = int(vel_dim)
    return p


def philox4x32_10(ctr, key):
    c = np.ascontiguousarray(ctr, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    out = np.zeros(4, dtype=np.uint32)
    up = ctypes.POINTER(ctypes.c_uint32)
    lib().orc_philox4x32_10(c.ctypes.data_as(up), k.ctypes.data_as(up), out.ctypes.data_as(up))
    return out


def contact_R2(lam, sigma, nbar):
    return lib().orc_contact_R2(float(lam), float(sigma), float(nbar))


def set_threads(n):
    """OpenMP threads of the oracle's loops (n <= 0: unchanged); returns the number in use."""
    return int(lib().orc_set_threads(int(n)))


def adaptive_dt(P, vel, dt_rest=0.0):
    """dx_min / v_max of the state (Sect. "Simulation setup"); dt_rest when at rest."""
    vel = np.ascontiguousarray(vel, dtype=np.float64).reshape(-1, 3)
    return lib().orc_adaptive_dt(ctypes.byref(P), vel.shape[0], _d(vel), float(dt_rest))


def _state(pos, vel=None):
    pos = np.ascontiguousarray(pos, dtype=np.float64).reshape(-1, 3)
    if vel is None:
        return pos
    vel = np.ascontiguousarray(vel, dtype=np.float64).reshape(-1, 3)
    return pos, vel


def cell_keys(P, pos):
    pos = _state(pos)
    n = pos.shape[0]
    key = np.zeros(n, dtype=np.int32)
    cidx = np.zeros((n, 3), dtype=np.int32)
    lib().orc_cell_keys(ctypes.byref(P), n, _d(pos), _i(key), _i(cidx))
    return key, cidx


def pair_test(P, ri, vi, rj, vj):
    arrs = [np.ascontiguousarray(x, dtype=np.float64).reshape(3) for x in (ri, vi, rj, vj)]
    q = np.zeros(5)
    ok = lib().orc_pair_test(ctypes.byref(P), *[_d(a) for a in arrs], _d(q))
    return bool(ok), q


def best_partners(P, pos, vel, brute=False):
    pos, vel = _state(pos, vel)
    n = pos.shape[0]
    best = np.full(n, -1, dtype=np.int32)
    f = lib().orc_best_partners_brute if brute else lib().orc_best_partners
    f(ctypes.byref(P), n, _d(pos), _d(vel), _i(best))
    return best


def candidate_count(P, pos):
    pos = _state(pos)
    return int(lib().orc_candidate_count(ctypes.byref(P), pos.shape[0], _d(pos)))


def mutual_pairs(best):
    best = np.ascontiguousarray(best, dtype=np.int32)
    n = best.shape[0]
    out = np.zeros(2 * max(n, 1), dtype=np.int32)
    m = lib().orc_mutual_pairs(n, _i(best), _i(out))
    return out[: 2 * m].reshape(m, 2)


def collide_move(P, pos, vel, best, ids=None):
    """Scatter, move and walls.  ids (increasing int64 global identities of the
    entries) key the pairs' random directions when the state is a subset of a
    larger system; None means ids = arange(n)."""
    pos, vel = _state(pos, vel)
    n = pos.shape[0]
    best = np.ascontiguousarray(best, dtype=np.int32)
    po = np.zeros_like(pos)
    vo = np.zeros_like(vel)
    W = np.zeros(n)
    paired = np.zeros(n, dtype=np.int32)
    if ids is None:
        lib().orc_collide_move(ctypes.byref(P), n, _d(pos), _d(vel), _i(best), _d(po), _d(vo), _d(W), _i(paired))
    else:
        ids = np.ascontiguousarray(ids, dtype=np.int64)
        if ids.shape != (n,) or (n > 1 and not np.all(np.diff(ids) > 0)):
            raise ValueError("ids must be n strictly increasing identities")
        lib().orc_collide_move_ids(ctypes.byref(P), n, _d(pos), _d(vel), _i(best),
                                   ids.ctypes.data_as(ctypes.c_void_p), _d(po), _d(vo), _d(W), _i(paired))
    return po, vo, W, paired


def n_bins(P):
    C = P.n_cells[0] * P.n_cells[1]
    if P.dim == 3:
        C *= P.n_cells[2]
    return C


def moments(P, pos, vel, virial=None):
    pos, vel = _state(pos, vel)
    n = pos.shape[0]
    C = n_bins(P)
    raw = np.zeros((C, 8))
    der = np.zeros((C, 8))
    glob = np.zeros(8)
    W = None if virial is None else np.ascontiguousarray(virial, dtype=np.float64)
    lib().orc_moments(ctypes.byref(P), n, _d(pos), _d(vel), _d(W), _d(raw), _d(der), _d(glob))
    return raw, der, glob


def dsmc_collide(P, pos, vel):
    """DSMC comparison variant (random partners in a c-bin): returns
    (new velocities, collided flags, accepted collisions); inputs unchanged."""
    pos, vel = _state(pos, vel)
    v = vel.copy()
    n = pos.shape[0]
    collided = np.zeros(n, dtype=np.int32)
    acc = lib().orc_dsmc_collide(ctypes.byref(P), n, _d(pos), _d(v), _i(collided))
    return v, collided, int(acc)


def dsmc_step(P, pos, vel):
    """One step of the DSMC variant: collisions, then free flight and walls.
    Returns (pos, vel, collided, accepted)."""
    v, collided, acc = dsmc_collide(P, pos, vel)
    po, vo, _, _ = collide_move(P, pos, v, np.full(len(v), -1, dtype=np.int32))
    return po, vo, collided, acc


def radial(P, pos, vel, center=(0.0, 0.0, 0.0)):
    """Per-c-bin [Sum v . r_hat, v_r] (Eq. vel_r) about `center`."""
    pos, vel = _state(pos, vel)
    c = np.ascontiguousarray(center, dtype=np.float64).reshape(3)
    out = np.zeros((n_bins(P), 2))
    lib().orc_radial(ctypes.byref(P), pos.shape[0], _d(pos), _d(vel), _d(c), _d(out))
    return out


def step(P, pos, vel):
    """One full step.  Returns (pos, vel, best, paired, raw, derived, glob, npairs);
    the inputs are not modified."""
    pos, vel = _state(pos, vel)
    pos = pos.copy()
    vel = vel.copy()
    n = pos.shape[0]
    C = n_bins(P)
    best = np.zeros(n, dtype=np.int32)
    paired = np.zeros(n, dtype=np.int32)
    raw = np.zeros((C, 8))
    der = np.zeros((C, 8))
    glob = np.zeros(8)
    npairs = lib().orc_step(ctypes.byref(P), n, _d(pos), _d(vel), _i(best), _i(paired), _d(raw), _d(der), _d(glob))
    return pos, vel, best, paired, raw, der, glob, int(npairs)
