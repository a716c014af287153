"""Python binding of the sm_103a kinetic Monte Carlo library (libkmc.so).

Argument marshalling only: every step of the method runs in the CUDA kernels
behind the C ABI of ``include/kmc.h``.  The names mirror that header
(``kmc_init``, ``kmc_step``, ``kmc_moments``, ``kmc_free`` and the getters).
Host arrays are numpy arrays; device arrays are anything with a
``data_ptr()`` (torch tensors), passed with ``where=KMC_WHERE_DEVICE``.

The library is loaded on the first call into it (or by ``load()``), not at
import, so that the input generators in ``inputs`` can be used without it; a
missing ``libkmc.so`` raises ``ImportError`` at that point (build it with
``python -c "import __graft_entry__ as g; g.build()"``): there is no fallback.
"""
import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libkmc.so")

KMC_OK = 0
KMC_EINVAL = -1
KMC_ENOMEM = -2
KMC_ECUDA = -3
KMC_ETIMEOUT = -4
KMC_ERANGE = -5
KMC_ESTATE = -6
KMC_WHERE_HOST = 0
KMC_WHERE_DEVICE = 1
KMC_BC_PERIODIC = 0
KMC_BC_WALL = 1
KMC_BC_ABSORB = 2
KMC_FLAG_RECORD = 1
KMC_FLAG_NO_GRAPH = 2
KMC_FLAG_STAGED_SEARCH = 4
KMC_FLAG_NO_TILE_SEARCH = 8
KMC_FLAG_ADAPTIVE_DT = 16
KMC_FLAG_VELOCITY_2D = 32
KMC_FLAG_DSMC = 64
KMC_FLAG_RADIAL_MOMENT = 128
KMC_FLAG_NO_TILE_PRUNE = 256
KMC_MOM_RAW = 1
KMC_MOM_DERIVED = 2
KMC_MOM_GLOBAL = 4
KMC_MOM_RADIAL = 8
KMC_NPHASES = 7
PHASES = ("search", "tile", "move", "scan", "scatter", "moments", "finalize")

ABI_FUNCTIONS = (
    "kmc_init", "kmc_step", "kmc_moments", "kmc_moments_size", "kmc_free", "kmc_sync",
    "kmc_last_error", "kmc_get_info", "kmc_get_state", "kmc_set_state", "kmc_get_cell_keys",
    "kmc_get_partners", "kmc_step_profiled", "kmc_find_partners_noalloc", "kmc_window_size", "kmc_autotune",
    "kmc_get_perm", "kmc_test_hold_scan", "kmc_tile_tests",
)
KMC_STATIC_MAX_PARTICLES = 262144


class KmcInstance(ctypes.Structure):
    _fields_ = [
        ("n_particles", ctypes.c_int64),
        ("lambda_", ctypes.c_double),
        ("sigma", ctypes.c_double),
        ("dt", ctypes.c_double),
        ("seed", ctypes.c_uint64),
    ]


class KmcConfig(ctypes.Structure):
    _fields_ = [
        ("dim_pos", ctypes.c_int),
        ("n_cells", ctypes.c_int * 3),
        ("lo", ctypes.c_double * 3),
        ("hi", ctypes.c_double * 3),
        ("bc", ctypes.c_int * 3),
        ("lambda_", ctypes.c_double),
        ("sigma", ctypes.c_double),
        ("dt", ctypes.c_double),
        ("seed", ctypes.c_uint64),
        ("precision", ctypes.c_int),
        ("n_instances", ctypes.c_int),
        ("instances", ctypes.POINTER(KmcInstance)),
        ("stream", ctypes.c_void_p),
        ("sub_cells", ctypes.c_int * 3),
        ("occupancy_target", ctypes.c_double),
        ("flags", ctypes.c_int),
        ("radial_center", ctypes.c_double * 3),
        ("tile_threads", ctypes.c_int),
        ("tile_cap", ctypes.c_int),
        ("tile_split", ctypes.c_int),
    ]


class KmcInfo(ctypes.Structure):
    _fields_ = [
        ("n_particles", ctypes.c_int64),
        ("n_bins", ctypes.c_int64),
        ("n_search_cells", ctypes.c_int64),
        ("n_instances", ctypes.c_int),
        ("precision", ctypes.c_int),
        ("step", ctypes.c_uint32),
        ("sub_cells", ctypes.c_int * 3),
        ("R2", ctypes.c_double),
        ("sigma", ctypes.c_double),
        ("dt", ctypes.c_double),
        ("vmax", ctypes.c_double),
        ("window", ctypes.c_int * 3),
        ("bytes_device", ctypes.c_int64),
        ("stage_tiles", ctypes.c_int64),
        ("tile_rows", ctypes.c_int),
        ("stage_cap", ctypes.c_int),
        ("time", ctypes.c_double),
        ("n_scan_tiles", ctypes.c_int),
        ("kernels_per_step", ctypes.c_int),
        ("kernels_moments", ctypes.c_int),
        ("tile_threads", ctypes.c_int),
        ("tile_cap", ctypes.c_int),
        ("tile_split", ctypes.c_int),
        ("graph_mode", ctypes.c_int),
        ("tile_prune", ctypes.c_int),
    ]


class KmcError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"kmc error {code}: {msg}")
        self.code = code


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError(
            f"{LIB_PATH} is missing: build it with `python -c \"import __graft_entry__ as g; g.build()\"`"
        )
    L = ctypes.CDLL(LIB_PATH)
    H = ctypes.c_void_p
    vp = ctypes.c_void_p
    L.kmc_init.argtypes = [ctypes.POINTER(KmcConfig), ctypes.c_int64, vp, vp, ctypes.c_int, ctypes.POINTER(H)]
    L.kmc_init.restype = ctypes.c_int
    L.kmc_step.argtypes = [H, ctypes.c_int, ctypes.c_int]
    L.kmc_step.restype = ctypes.c_int
    L.kmc_moments.argtypes = [H, vp, ctypes.c_int, ctypes.c_int]
    L.kmc_moments.restype = ctypes.c_int
    L.kmc_moments_size.argtypes = [H, ctypes.c_int]
    L.kmc_moments_size.restype = ctypes.c_int64
    L.kmc_free.argtypes = [H]
    L.kmc_free.restype = None
    L.kmc_sync.argtypes = [H]
    L.kmc_sync.restype = ctypes.c_int
    L.kmc_last_error.argtypes = [H]
    L.kmc_last_error.restype = ctypes.c_char_p
    L.kmc_get_info.argtypes = [H, ctypes.POINTER(KmcInfo)]
    L.kmc_get_info.restype = ctypes.c_int
    L.kmc_get_state.argtypes = [H, vp, vp, ctypes.c_int]
    L.kmc_get_state.restype = ctypes.c_int
    L.kmc_set_state.argtypes = [H, vp, vp, ctypes.c_int, ctypes.c_uint32]
    L.kmc_set_state.restype = ctypes.c_int
    L.kmc_get_cell_keys.argtypes = [H, vp, ctypes.c_int]
    L.kmc_get_cell_keys.restype = ctypes.c_int
    L.kmc_get_partners.argtypes = [H, vp, vp, ctypes.c_int]
    L.kmc_get_partners.restype = ctypes.c_int
    L.kmc_get_perm.argtypes = [H, vp, ctypes.c_int]
    L.kmc_get_perm.restype = ctypes.c_int
    L.kmc_test_hold_scan.argtypes = [H, ctypes.c_int, ctypes.c_uint32]
    L.kmc_test_hold_scan.restype = ctypes.c_int
    L.kmc_step_profiled.argtypes = [H, ctypes.c_int, ctypes.c_int, ctypes.POINTER(ctypes.c_double)]
    L.kmc_step_profiled.restype = ctypes.c_int
    L.kmc_window_size.argtypes = [H, ctypes.POINTER(ctypes.c_double)]
    L.kmc_window_size.restype = ctypes.c_int
    L.kmc_tile_tests.argtypes = [H, ctypes.POINTER(ctypes.c_double)]
    L.kmc_tile_tests.restype = ctypes.c_int
    L.kmc_find_partners_noalloc.argtypes = [ctypes.POINTER(KmcConfig), ctypes.c_int64, vp, vp, vp]
    L.kmc_find_partners_noalloc.restype = ctypes.c_int
    L.kmc_autotune.argtypes = [ctypes.POINTER(KmcConfig), ctypes.c_int64, vp, vp, ctypes.c_int, ctypes.c_int,
                               ctypes.POINTER(KmcConfig), ctypes.POINTER(ctypes.c_double)]
    L.kmc_autotune.restype = ctypes.c_int
    return L


_lib = None


def load():
    """Load libkmc.so (once) and return the ctypes handle."""
    global _lib
    if _lib is None:
        _lib = _load()
    return _lib


def __getattr__(name):
    # `lib` is the loaded library, created on first access
    if name == "lib":
        return load()
    raise AttributeError(f"module {__name__!r} has no attribute {name!r}")


def _ptr(a):
    """Raw address of a numpy array (host) or a tensor-like with data_ptr()."""
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        if not a.flags["C_CONTIGUOUS"]:
            raise ValueError("array must be C-contiguous")
        return a.ctypes.data
    if hasattr(a, "data_ptr"):
        if hasattr(a, "is_contiguous") and not a.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return a.data_ptr()
    if isinstance(a, int):
        return a
    raise TypeError(f"cannot take the address of {type(a)}")


def _check(rc, h=None):
    if rc != KMC_OK:
        msg = load().kmc_last_error(h)
        raise KmcError(rc, msg.decode() if msg else "")
    return rc


def make_config(dim_pos=3, n_cells=(1, 1, 1), lo=(0.0, 0.0, 0.0), hi=(1.0, 1.0, 1.0),
                bc=(KMC_BC_WALL, KMC_BC_PERIODIC, KMC_BC_PERIODIC), lam=1e-3, sigma=0.0, dt=1e-3,
                seed=0, precision=32, instances=None, stream=None, sub_cells=(0, 0, 0),
                occupancy_target=0.0, flags=0, radial_center=(0.0, 0.0, 0.0), tile_threads=0, tile_cap=0,
                tile_split=0):
    """Fill a KmcConfig.  `instances` is a list of dicts with keys n, lam, sigma, dt, seed;
    the returned object keeps the instance array alive."""
    c = KmcConfig()
    c.dim_pos = int(dim_pos)
    for d in range(3):
        c.n_cells[d] = int(n_cells[d]) if d < len(n_cells) else 1
        c.lo[d] = float(lo[d]) if d < len(lo) else 0.0
        c.hi[d] = float(hi[d]) if d < len(hi) else 1.0
        c.bc[d] = int(bc[d]) if d < len(bc) else KMC_BC_PERIODIC
        c.sub_cells[d] = int(sub_cells[d]) if d < len(sub_cells) else 0
        c.radial_center[d] = float(radial_center[d]) if d < len(radial_center) else 0.0
    c.lambda_ = float(lam)
    c.sigma = float(sigma)
    c.dt = float(dt)
    c.seed = int(seed) & 0xFFFFFFFFFFFFFFFF
    c.precision = int(precision)
    c.stream = stream
    c.occupancy_target = float(occupancy_target)
    c.flags = int(flags)
    c.tile_threads = int(tile_threads)
    c.tile_cap = int(tile_cap)
    c.tile_split = int(tile_split)
    if instances:
        arr = (KmcInstance * len(instances))()
        for i, inst in enumerate(instances):
            arr[i].n_particles = int(inst["n"])
            arr[i].lambda_ = float(inst.get("lam", 0.0))
            arr[i].sigma = float(inst.get("sigma", 0.0))
            arr[i].dt = float(inst["dt"])
            arr[i].seed = int(inst.get("seed", 0)) & 0xFFFFFFFFFFFFFFFF
        c.n_instances = len(instances)
        c.instances = ctypes.cast(arr, ctypes.POINTER(KmcInstance))
        c._keep = arr
    else:
        c.n_instances = 0
    return c


# ------------------------------------------------------------- the C ABI names

def kmc_init(cfg, n, pos, vel, where=KMC_WHERE_HOST):
    h = ctypes.c_void_p()
    _check(load().kmc_init(ctypes.byref(cfg), int(n), _ptr(pos), _ptr(vel), int(where), ctypes.byref(h)))
    return h


def kmc_step(h, nsteps=1, want_moments=1):
    return _check(load().kmc_step(h, int(nsteps), int(want_moments)), h)


def kmc_moments(h, out, where=KMC_WHERE_HOST, fields_mask=KMC_MOM_RAW | KMC_MOM_DERIVED | KMC_MOM_GLOBAL):
    return _check(load().kmc_moments(h, _ptr(out), int(where), int(fields_mask)), h)


def kmc_step_profiled(h, nsteps=1, want_moments=1):
    """Returns a dict phase -> summed device milliseconds, plus 'total'."""
    ms = (ctypes.c_double * (KMC_NPHASES + 1))()
    _check(load().kmc_step_profiled(h, int(nsteps), int(want_moments), ms), h)
    out = {name: ms[i] for i, name in enumerate(PHASES)}
    out["total"] = ms[KMC_NPHASES]
    return out


def kmc_window_size(h):
    """Mean candidates examined per particle by the search of the current state."""
    v = ctypes.c_double()
    _check(load().kmc_window_size(h, ctypes.byref(v)), h)
    return v.value


def kmc_tile_tests(h):
    """Pair tests made by the pruned binary32 tile search since kmc_init."""
    v = ctypes.c_double()
    _check(load().kmc_tile_tests(h, ctypes.byref(v)), h)
    return v.value


def kmc_find_partners_noalloc(cfg, n, pos, vel, best):
    """Closest candidate of every particle of a device-resident state, with no
    allocation (scratch in the library's fixed device array).  pos, vel, best
    are device arrays; returns the C status code (KMC_OK on success)."""
    return int(load().kmc_find_partners_noalloc(ctypes.byref(cfg), int(n), _ptr(pos), _ptr(vel), _ptr(best)))


def kmc_autotune(cfg, n, pos, vel, where=KMC_WHERE_HOST, trial_steps=3):
    """Fastest search set-up for cfg on this state (same results for every
    set-up): returns (config to pass to kmc_init, milliseconds per step)."""
    best = KmcConfig()
    ms = ctypes.c_double()
    _check(load().kmc_autotune(ctypes.byref(cfg), int(n), _ptr(pos), _ptr(vel), int(where), int(trial_steps),
                            ctypes.byref(best), ctypes.byref(ms)))
    if hasattr(cfg, "_keep"):
        best._keep = cfg._keep   # the instance array the copy points to
    return best, ms.value


def kmc_moments_size(h, fields_mask):
    return int(load().kmc_moments_size(h, int(fields_mask)))


def kmc_free(h):
    load().kmc_free(h)


def kmc_sync(h):
    return _check(load().kmc_sync(h), h)


def kmc_last_error(h=None):
    m = load().kmc_last_error(h)
    return m.decode() if m else ""


def kmc_get_info(h):
    info = KmcInfo()
    _check(load().kmc_get_info(h, ctypes.byref(info)), h)
    return info


def kmc_get_state(h, pos, vel, where=KMC_WHERE_HOST):
    return _check(load().kmc_get_state(h, _ptr(pos), _ptr(vel), int(where)), h)


def kmc_set_state(h, pos, vel, where=KMC_WHERE_HOST, step=0):
    return _check(load().kmc_set_state(h, _ptr(pos), _ptr(vel), int(where), int(step)), h)


def kmc_get_cell_keys(h, keys, where=KMC_WHERE_HOST):
    return _check(load().kmc_get_cell_keys(h, _ptr(keys), int(where)), h)


def kmc_get_partners(h, best, partner, where=KMC_WHERE_HOST):
    return _check(load().kmc_get_partners(h, _ptr(best), _ptr(partner), int(where)), h)


def kmc_get_perm(h, perm, where=KMC_WHERE_HOST):
    return _check(load().kmc_get_perm(h, _ptr(perm), int(where)), h)


def kmc_test_hold_scan(h, tile, spin_cap):
    """Test hook of the bounded device wait (see include/kmc.h)."""
    return _check(load().kmc_test_hold_scan(h, int(tile), int(spin_cap)), h)


# --------------------------------------------------------- convenience wrapper

class Simulation:
    """Owns one handle; host-side numpy in/out around the C ABI calls."""

    def __init__(self, cfg, pos, vel, where=KMC_WHERE_HOST):
        self.cfg = cfg
        self.dtype = np.float32 if cfg.precision == 32 else np.float64
        if where == KMC_WHERE_HOST:
            pos = np.ascontiguousarray(pos, dtype=self.dtype).reshape(-1, 3)
            vel = np.ascontiguousarray(vel, dtype=self.dtype).reshape(-1, 3)
            n = pos.shape[0]
        else:
            n = pos.shape[0]
        self.n = n
        self.h = kmc_init(cfg, n, pos, vel, where)
        info = kmc_get_info(self.h)
        self.n_bins = info.n_bins
        self.n_instances = info.n_instances

    def close(self):
        if self.h is not None:
            kmc_free(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def step(self, nsteps=1, want_moments=1):
        kmc_step(self.h, nsteps, want_moments)

    def step_profiled(self, nsteps=1, want_moments=1):
        return kmc_step_profiled(self.h, nsteps, want_moments)

    def sync(self):
        kmc_sync(self.h)

    def info(self):
        return kmc_get_info(self.h)

    def window_size(self):
        return kmc_window_size(self.h)

    def tile_tests(self):
        return kmc_tile_tests(self.h)

    def state(self):
        pos = np.zeros((self.n, 3), dtype=self.dtype)
        vel = np.zeros((self.n, 3), dtype=self.dtype)
        kmc_get_state(self.h, pos, vel)
        return pos, vel

    def set_state(self, pos, vel, step=0):
        pos = np.ascontiguousarray(pos, dtype=self.dtype).reshape(-1, 3)
        vel = np.ascontiguousarray(vel, dtype=self.dtype).reshape(-1, 3)
        kmc_set_state(self.h, pos, vel, KMC_WHERE_HOST, step)

    def cell_keys(self):
        k = np.zeros(self.n, dtype=np.int32)
        kmc_get_cell_keys(self.h, k)
        return k

    def perm(self):
        p = np.zeros(self.n, dtype=np.int32)
        kmc_get_perm(self.h, p)
        return p

    def partners(self):
        best = np.zeros(self.n, dtype=np.int32)
        partner = np.zeros(self.n, dtype=np.int32)
        kmc_get_partners(self.h, best, partner)
        return best, partner

    def radial(self):
        """[bins, 2]: Sum v.r_hat and the radial velocity v_r per c-bin (Eq. vel_r)."""
        out = np.zeros(kmc_moments_size(self.h, KMC_MOM_RADIAL), dtype=np.float64)
        kmc_moments(self.h, out, KMC_WHERE_HOST, KMC_MOM_RADIAL)
        return out.reshape(-1, 2)

    def moments(self):
        """(raw [bins, 8], derived [bins, 8], glob [instances, 8])"""
        mask = KMC_MOM_RAW | KMC_MOM_DERIVED | KMC_MOM_GLOBAL
        out = np.zeros(kmc_moments_size(self.h, mask), dtype=np.float64)
        kmc_moments(self.h, out, KMC_WHERE_HOST, mask)
        nb = self.n_bins
        raw = out[: 8 * nb].reshape(nb, 8)
        der = out[8 * nb: 16 * nb].reshape(nb, 8)
        glob = out[16 * nb:].reshape(-1, 8)
        return raw, der, glob
