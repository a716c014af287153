"""Pins of the CPU oracle against what the paper and the mathematics fix.

Each test checks the oracle against something other than itself: published
known answers, an independent library routine, brute force over tiny inputs,
dense sampling of the relative trajectory, closed forms of free flight in a
walled box, or conservation laws.  A plausible slip (dropped term, wrong sign
or index, transposed operand) in the oracle fails at least one of them.
"""
import math
import os

import numpy as np
import pytest

import oracle
from paper_1210_8084_gb300 import inputs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def params(**kw):
    d = dict(dim=3, n_cells=(3, 3, 3), lo=(0, 0, 0), hi=(1, 1, 1), bc=(1, 0, 0), R2=0.01, dt=0.05,
             seed=0, step=0, decide32=False)
    d.update(kw)
    return oracle.make_params(**d)


# ----------------------------------------------------------------- Philox

def test_philox_known_answers():
    """Philox4x32-10 known-answer vectors (Salmon et al., SC'11 / Random123)."""
    rows = [ln.split() for ln in open(os.path.join(GOLDEN, "philox4x32_10_kat.txt")) if ln[0] != "#"]
    assert len(rows) == 3
    for r in rows:
        v = [int(x, 16) for x in r]
        out = oracle.philox4x32_10(v[0:4], v[4:6])
        assert [int(x) for x in out] == v[6:10]


def test_philox_matches_triton_library():
    """Cross-check against triton's Philox4x32 (CPU interpreter) on random counters/keys."""
    pytest.importorskip("triton")
    import subprocess
    import sys
    code = r'''
import os, sys
os.environ["TRITON_INTERPRET"] = "1"
import numpy as np, torch, triton, triton.language as tl
@triton.jit
def k(out_ptr, c_ptr, k_ptr, N: tl.constexpr):
    i = tl.arange(0, N)
    c0 = tl.load(c_ptr + 0 + i*4).to(tl.uint32); c1 = tl.load(c_ptr + 1 + i*4).to(tl.uint32)
    c2 = tl.load(c_ptr + 2 + i*4).to(tl.uint32); c3 = tl.load(c_ptr + 3 + i*4).to(tl.uint32)
    k0 = tl.load(k_ptr + 0 + i*2).to(tl.uint32); k1 = tl.load(k_ptr + 1 + i*2).to(tl.uint32)
    a, b, c, d = tl.random.philox_impl(c0, c1, c2, c3, k0, k1, 10)
    tl.store(out_ptr + 0 + i*4, a.to(tl.int64) & 0xffffffff); tl.store(out_ptr + 1 + i*4, b.to(tl.int64) & 0xffffffff)
    tl.store(out_ptr + 2 + i*4, c.to(tl.int64) & 0xffffffff); tl.store(out_ptr + 3 + i*4, d.to(tl.int64) & 0xffffffff)
rng = np.random.default_rng(7)
C = rng.integers(0, 2**32, (16, 4)); K = rng.integers(0, 2**32, (16, 2))
out = torch.zeros(64, dtype=torch.int64)
k[(1,)](out, torch.tensor(C.ravel()), torch.tensor(K.ravel()), 16)
for r in range(16):
    print(*C[r], *K[r], *[int(x) for x in out[4*r:4*r+4]])
'''
    res = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, timeout=600)
    if res.returncode != 0:
        pytest.skip("triton interpreter unavailable: " + res.stderr[-200:])
    for line in res.stdout.strip().splitlines():
        v = [int(x) for x in line.split()]
        assert [int(x) for x in oracle.philox4x32_10(v[0:4], v[4:6])] == v[6:10]


# ------------------------------------------------------- derived constants

def test_contact_distance_inverts_eq7_and_reff():
    """lambda = 1/(4 pi r_eff^2 n) with r_eff = R/2 (Eq. reff_lambda); sigma = 4 pi r_eff^2 (Eq. 7)."""
    for lam, nbar in [(1e-3, 2e5), (5e-4, 6.4e7), (1.0, 1.6e7), (2e-4, 512e6 / (1 / 256))]:
        R2 = oracle.contact_R2(lam, 0.0, nbar)
        r_eff = math.sqrt(R2) / 2.0
        assert 1.0 / (4 * math.pi * r_eff ** 2 * nbar) == pytest.approx(lam, rel=1e-13)
    # sigma given directly: contact radius of two spheres of cross-section sigma = pi R^2
    assert oracle.contact_R2(123.0, 0.5, 1.0) == pytest.approx(0.5 / math.pi, rel=1e-15)
    # free streaming (lambda -> inf): no contact distance
    assert oracle.contact_R2(math.inf, 0.0, 1e6) == 0.0


# -------------------------------------------------------------------- keys

@pytest.mark.parametrize("decide32", [False, True])
def test_cell_keys_membership(decide32):
    """Each particle lies in the c-bin its key names; key = c_x + n_x (c_y + n_y c_z)."""
    rng = np.random.default_rng(1)
    n_cells = (7, 5, 3)
    lo = np.array([-1.0, 0.5, 2.0])
    hi = np.array([2.5, 1.0, 3.75])
    P = params(n_cells=n_cells, lo=lo, hi=hi, decide32=decide32)
    pos = lo + (hi - lo) * rng.random((5000, 3))
    pos[:5] = lo            # lower faces
    pos[5:10] = hi          # upper faces clamp into the last bin
    key, cidx = oracle.cell_keys(P, pos)
    dx = (hi - lo) / np.array(n_cells)
    tol = 1e-6 if decide32 else 1e-12
    for d in range(3):
        c = cidx[:, d]
        assert (c >= 0).all() and (c < n_cells[d]).all()
        assert (pos[:, d] >= lo[d] + c * dx[d] - tol).all()
        assert (pos[:, d] <= lo[d] + (c + 1) * dx[d] + tol).all()
    assert (cidx[5:10] == np.array(n_cells) - 1).all()
    assert (cidx[:5] == 0).all()
    assert (key == cidx[:, 0] + n_cells[0] * (cidx[:, 1] + n_cells[1] * cidx[:, 2])).all()
    P2 = params(dim=2, n_cells=(7, 5, 1), lo=lo, hi=hi, decide32=decide32)
    key2, cidx2 = oracle.cell_keys(P2, pos)
    assert (key2 == cidx2[:, 0] + 7 * cidx2[:, 1]).all() and (cidx2[:, 2] == 0).all()


# ------------------------------------------------------- PoCA pair algebra

def _trajectory_min(dr, dv, t_lo, t_hi, samples=20001):
    """min over t of |dr + dv t|^2 by dense sampling plus golden-section refinement."""
    t = np.linspace(t_lo, t_hi, samples)
    d2 = ((dr[None, :] + t[:, None] * dv[None, :]) ** 2).sum(1)
    k = int(np.argmin(d2))
    a = t[max(k - 1, 0)]
    b = t[min(k + 1, samples - 1)]
    gr = (math.sqrt(5) - 1) / 2
    f = lambda s: float(((dr + s * dv) ** 2).sum())
    c, d = b - gr * (b - a), a + gr * (b - a)
    for _ in range(100):
        if f(c) < f(d):
            b = d
        else:
            a = c
        c, d = b - gr * (b - a), a + gr * (b - a)
    tm = 0.5 * (a + b)
    return tm, f(tm)


@pytest.mark.parametrize("decide32", [False, True])
def test_poca_against_sampled_trajectory(decide32):
    """criterion 1 <=> closest approach inside (0, dt); criterion 2 <=> d_min <= R;
    d2 equals the sampled minimum distance squared (Eqs. 5-6, 8-9, 12)."""
    rng = np.random.default_rng(2)
    dt, R2 = 0.3, 0.04
    P = params(dim=3, n_cells=(1, 1, 1), lo=(-10, -10, -10), hi=(10, 10, 10), bc=(1, 1, 1), R2=R2, dt=dt,
               decide32=decide32)
    checked = 0
    for _ in range(400):
        ri = rng.normal(0, 0.3, 3)
        rj = rng.normal(0, 0.3, 3)
        vi = rng.normal(0, 1, 3)
        vj = rng.normal(0, 1, 3)
        ok, q = oracle.pair_test(P, ri, vi, rj, vj)
        dr, dv = ri - rj, vi - vj
        t_all, d2_all = _trajectory_min(dr, dv, -50.0, 50.0)
        # the closest approach of the infinite line and its distance
        assert q[4] == pytest.approx(d2_all, rel=1e-5 if decide32 else 1e-9, abs=1e-6 if decide32 else 1e-12)
        inside = 0.0 < t_all < dt
        close = d2_all <= R2
        margin_t = min(abs(t_all), abs(t_all - dt))
        if margin_t < 1e-4 or abs(d2_all - R2) < 1e-4:
            continue  # too near a threshold for a sampled reference
        assert ok == (inside and close)
        checked += 1
    assert checked > 300


def test_real_overlap_times_match_numpy_roots():
    """Criterion 2 reads Eq. collision_time2 as the discriminant of Eq. collision_time:
    the overlap times are real exactly when numpy.roots finds real roots."""
    rng = np.random.default_rng(3)
    R2 = 0.25
    P = params(dim=3, n_cells=(1, 1, 1), lo=(-10, -10, -10), hi=(10, 10, 10), bc=(1, 1, 1), R2=R2, dt=1e3)
    n_real = 0
    for _ in range(500):
        ri, rj = rng.normal(0, 0.4, (2, 3))
        vi, vj = rng.normal(0, 1, (2, 3))
        dr, dv = ri - rj, vi - vj
        _, q = oracle.pair_test(P, ri, vi, rj, vj)
        a, b, r2, disc = q[0], q[1], q[2], q[3]
        roots = np.roots([b, 2 * a, r2 - R2])
        real = bool(np.all(np.abs(np.imag(roots)) < 1e-9 * (1 + np.abs(np.real(roots)))))
        if abs(disc) < 1e-9:
            continue
        assert real == (disc >= 0)
        if real:
            n_real += 1
            # both roots are overlap times: |dr + dv t_o| = R
            for t in np.real(roots):
                assert np.linalg.norm(dr + dv * t) == pytest.approx(math.sqrt(R2), rel=1e-7)
    assert n_real > 100


def test_minimum_image_in_periodic_dimension():
    """A pair across a periodic face is tested with the short separation."""
    P = params(dim=3, n_cells=(1, 1, 1), lo=(0, 0, 0), hi=(1, 1, 1), bc=(0, 1, 1), R2=1e-4, dt=0.1)
    ri, rj = np.array([0.98, 0.5, 0.5]), np.array([0.02, 0.5, 0.5])
    vi, vj = np.array([1.0, 0, 0]), np.array([-1.0, 0, 0])   # approaching through x = 1 == 0
    ok, q = oracle.pair_test(P, ri, vi, rj, vj)
    assert ok and q[0] == pytest.approx(-0.04 * 2.0)
    P_wall = params(dim=3, n_cells=(1, 1, 1), lo=(0, 0, 0), hi=(1, 1, 1), bc=(1, 1, 1), R2=1e-4, dt=0.1)
    ok2, _ = oracle.pair_test(P_wall, ri, vi, rj, vj)
    assert not ok2  # through a wall they recede


# ------------------------------------------- best partner (criterion 3)

def _numpy_best(P, pos, vel):
    """Independent brute force in float64 numpy: all pairs, neighbourhood by
    cell-index distance, the three criteria, argmin of d_min^2, ties to lower id."""
    dim = P.dim
    n_cells = np.array(P.n_cells[:dim])
    lo = np.array(P.lo[:dim])
    hi = np.array(P.hi[:dim])
    L = hi - lo
    per = np.array([P.bc[d] == 0 for d in range(dim)])
    c = np.clip(np.floor((pos[:, :dim] - lo) * (n_cells / L)).astype(int), 0, n_cells - 1)
    n = pos.shape[0]
    best = np.full(n, -1)
    for i in range(n):
        dr = pos[i, :dim] - pos[:, :dim]
        dr = np.where(per & (dr > L / 2), dr - L, dr)
        dr = np.where(per & (dr < -L / 2), dr + L, dr)
        dc = np.abs(c[i] - c)
        dc = np.where(per, np.minimum(dc, n_cells - dc), dc)
        nb = (dc <= 1).all(1)
        dv = vel[i, :dim] - vel[:, :dim]
        a = (dr * dv).sum(1)
        b = (dv * dv).sum(1)
        r2 = (dr * dr).sum(1)
        with np.errstate(divide="ignore", invalid="ignore"):
            d2 = r2 - a * a / b
        ok = nb & (b > 0) & (a < 0) & (a + b * P.dt > 0) & (a * a - b * (r2 - P.R2) >= 0)
        ok[i] = False
        if ok.any():
            idx = np.nonzero(ok)[0]
            best[i] = idx[np.lexsort((idx, d2[idx]))[0]]
    return best


@pytest.mark.parametrize("dim,n_cells,bc", [
    (3, (1, 1, 1), (1, 0, 0)), (3, (2, 2, 2), (0, 0, 0)), (3, (3, 3, 3), (1, 0, 0)),
    (3, (5, 2, 3), (1, 1, 0)), (2, (5, 5, 1), (1, 1, 0)), (2, (2, 3, 1), (0, 0, 0)),
])
def test_best_partner_brute_force(dim, n_cells, bc):
    rng = np.random.default_rng(sum(n_cells) + dim)
    n = 64
    pos = rng.random((n, 3))
    vel = rng.normal(0, 1, (n, 3))
    P = params(dim=dim, n_cells=n_cells, bc=bc, R2=0.02, dt=0.2)
    best = oracle.best_partners(P, pos, vel)
    brute = oracle.best_partners(P, pos, vel, brute=True)
    ref = _numpy_best(P, pos, vel)
    assert (best == brute).all()
    assert (best == ref).all()
    assert (best >= 0).sum() > 5


def test_tie_breaks_to_lower_id():
    """Two candidates at the same closest-approach distance: the lower id wins."""
    P = params(dim=3, n_cells=(1, 1, 1), lo=(-5, -5, -5), hi=(5, 5, 5), bc=(1, 1, 1), R2=1.0, dt=10.0)
    pos = np.array([[0.0, 0, 0], [1.0, 0.2, 0], [-1.0, -0.2, 0]])
    vel = np.array([[0.0, 0, 0], [-1.0, 0, 0], [1.0, 0, 0]])
    best = oracle.best_partners(P, pos, vel)
    assert best[0] == 1


def test_mutual_pairs_invariants():
    rng = np.random.default_rng(5)
    pos = rng.random((3000, 3))
    vel = rng.normal(0, 1, (3000, 3))
    P = params(n_cells=(6, 6, 6), R2=0.005, dt=0.05)
    best = oracle.best_partners(P, pos, vel)
    pairs = oracle.mutual_pairs(best)
    flat = pairs.ravel()
    assert len(np.unique(flat)) == flat.size            # nobody in two pairs
    assert (pairs[:, 0] < pairs[:, 1]).all()
    assert (best[pairs[:, 0]] == pairs[:, 1]).all() and (best[pairs[:, 1]] == pairs[:, 0]).all()
    expected = {(i, int(best[i])) for i in range(3000) if best[i] > i and best[best[i]] == i}
    assert expected == {tuple(p) for p in pairs.tolist()}


# ------------------------------------------------- scattering and motion

def test_cm_scattering_conserves_and_keeps_relative_speed():
    rng = np.random.default_rng(6)
    n = 4000
    pos = rng.random((n, 3))
    vel = rng.normal(0, 1, (n, 3))
    P = params(n_cells=(8, 8, 8), bc=(0, 0, 0), R2=0.004, dt=0.05, seed=12345, step=7)  # no wall folds
    best = oracle.best_partners(P, pos, vel)
    po, vo, W, paired = oracle.collide_move(P, pos, vel, best)
    pairs = oracle.mutual_pairs(best)
    assert len(pairs) > 200
    i, j = pairs[:, 0], pairs[:, 1]
    eps = np.finfo(float).eps
    mom_in = vel[i] + vel[j]
    mom_out = vo[i] + vo[j]
    scale = np.linalg.norm(vel[i], axis=1) + np.linalg.norm(vel[j], axis=1)
    assert (np.abs(mom_out - mom_in).max(1) <= 8 * eps * scale).all()
    e_in = (vel[i] ** 2).sum(1) + (vel[j] ** 2).sum(1)
    e_out = (vo[i] ** 2).sum(1) + (vo[j] ** 2).sum(1)
    assert (np.abs(e_out - e_in) <= 16 * eps * e_in).all()
    g_in = np.linalg.norm(vel[i] - vel[j], axis=1)
    g_out = np.linalg.norm(vo[i] - vo[j], axis=1)
    assert np.allclose(g_out, g_in, rtol=1e-12)
    # outgoing relative directions are isotropic
    nh = (vo[i] - vo[j]) / g_out[:, None]
    m = len(pairs)
    assert np.abs(nh.mean(0)).max() < 4 / math.sqrt(3 * m)
    assert np.abs((nh ** 2).mean(0) - 1 / 3).max() < 4 * math.sqrt(4 / 45 / m)
    # unpaired particles keep their velocity; paired[] is symmetric
    un = paired < 0
    assert np.array_equal(vo[un], vel[un])
    assert (paired[i] == j).all() and (paired[j] == i).all()


def test_split_move_meets_at_closest_approach():
    """Eq. 13: both partners sit at their point of closest approach at t_poca,
    so the end-of-step separation is r_rel(t_poca) + (v_i' - v_j')(dt - t_poca)."""
    rng = np.random.default_rng(8)
    n = 2000
    pos = 0.25 + 0.5 * rng.random((n, 3))
    vel = rng.normal(0, 1, (n, 3))
    P = params(n_cells=(4, 4, 4), bc=(1, 1, 1), R2=0.003, dt=0.02)
    best = oracle.best_partners(P, pos, vel)
    po, vo, W, paired = oracle.collide_move(P, pos, vel, best)
    pairs = oracle.mutual_pairs(best)
    i, j = pairs[:, 0], pairs[:, 1]
    dr, dv = pos[i] - pos[j], vel[i] - vel[j]
    tp = -(dr * dv).sum(1) / (dv * dv).sum(1)
    assert ((tp > 0) & (tp < P.dt)).all()
    rp = dr + dv * tp[:, None]
    expect = rp + (vo[i] - vo[j]) * (P.dt - tp)[:, None]
    assert np.allclose(po[i] - po[j], expect, atol=1e-13)
    # virial: r_ij(t_poca) . dp_i, and each partner sees the same value
    assert np.allclose(W[i], (rp * (vo[i] - vel[i])).sum(1), atol=1e-14)
    assert np.allclose(W[i], W[j], atol=1e-14)


def test_free_streaming_reflecting_box_closed_form():
    """lambda -> inf (free streaming, Sect. "Study of non-equilibrium systems"):
    positions follow the triangle wave of x0 + v t in a walled box, speeds
    are conserved exactly and only the normal component flips."""
    rng = np.random.default_rng(9)
    n = 500
    lo = np.array([0.0, -0.5, 1.0])
    hi = np.array([1.0, 0.5, 1.5])
    pos = lo + (hi - lo) * rng.random((n, 3))
    vel = rng.normal(0, 3, (n, 3))
    P = params(dim=3, n_cells=(4, 4, 4), lo=lo, hi=hi, bc=(1, 1, 1), R2=0.0, dt=0.013)
    p, v = pos.copy(), vel.copy()
    steps = 57
    for s in range(steps):
        p, v, best, paired, raw, der, glob, npairs = oracle.step(P, p, v)
        assert npairs == 0
    t = steps * P.dt
    L = hi - lo
    u = np.mod(pos - lo + vel * t, 2 * L)
    x_exact = lo + np.where(u <= L, u, 2 * L - u)
    assert np.allclose(p, x_exact, atol=1e-11)
    assert np.array_equal(np.abs(v), np.abs(vel))


def test_periodic_wrap_closed_form():
    rng = np.random.default_rng(10)
    n = 300
    pos = rng.random((n, 3))
    vel = rng.normal(0, 2, (n, 3))
    P = params(n_cells=(3, 3, 3), bc=(0, 0, 0), R2=0.0, dt=0.01)
    p, v = pos.copy(), vel.copy()
    for _ in range(40):
        p, v = oracle.step(P, p, v)[:2]
    assert np.allclose(p, np.mod(pos + vel * 0.4, 1.0), atol=1e-12)
    assert np.array_equal(v, vel)


# ---------------------------------------------------------------- moments

def test_moments_special_cases():
    """Known states: six particles per bin moving +-c along the axes on top of a
    drift u give n = N/V, bulk velocity u, T = c^2/3, p_kin = n T (Eqs. 15, 18, 19)."""
    P = params(dim=3, n_cells=(2, 1, 1), lo=(0, 0, 0), hi=(2, 1, 1), bc=(1, 0, 0), R2=0.0, dt=0.1)
    c, u = 2.0, np.array([0.3, -0.1, 0.7])
    axes = np.concatenate([np.eye(3), -np.eye(3)])
    pos = np.concatenate([np.full((6, 3), 0.5), np.array([[1.5, 0.5, 0.5]] * 6)])
    vel = np.concatenate([u + c * axes, -u + 2 * c * axes])
    raw, der, glob = oracle.moments(P, pos, vel, np.zeros(12))
    assert der[0, 0] == pytest.approx(6.0) and der[1, 0] == pytest.approx(6.0)
    assert np.allclose(der[0, 1:4], u) and np.allclose(der[1, 1:4], -u)
    assert der[0, 4] == pytest.approx(c * c / 3) and der[1, 4] == pytest.approx(4 * c * c / 3)
    assert der[0, 5] == pytest.approx(6.0 * c * c / 3)
    assert glob[0] == 12 and glob[1] == pytest.approx(0.5 * (vel ** 2).sum())
    assert np.allclose(glob[2:5], vel.sum(0), atol=1e-14)


def test_virial_pressure_vanishes_on_average():
    """Isotropic scattering: <r_ij(t_poca) . dp_i> = 0 because r_ij(t_poca) is
    perpendicular to v_rel (Eq. stress, collisional part)."""
    pos, vel = inputs.periodic_box(20000, seed=3, T=1.0)
    P = params(n_cells=(10, 10, 10), bc=(0, 0, 0), R2=oracle.contact_R2(1e-3, 0, 20000), dt=0.02)
    best = oracle.best_partners(P, pos, vel)
    _, _, W, paired = oracle.collide_move(P, pos, vel, best)
    Wp = W[paired >= 0]
    assert len(Wp) > 5000
    assert abs(Wp.mean()) < 4 * Wp.std() / math.sqrt(len(Wp))


# ------------------------------------------------------- physics of the gas

def test_mono_energetic_gas_relaxes_to_maxwell():
    """Sect. "Equilibration and Speed-up": |v| = v_in with random directions
    reaches the Maxwell-Boltzmann speed law at small lambda within tens of steps."""
    from scipy import stats
    n = 20000
    v_in = 10.0
    pos, vel = inputs.periodic_box(n, seed=11, v_in=v_in)
    dx = 0.1
    P = params(n_cells=(10, 10, 10), bc=(0, 0, 0), R2=oracle.contact_R2(1e-3 * dx, 0, n), dt=dx / 60 * 2)
    e0 = 0.5 * (vel ** 2).sum()
    fracs = []
    p, v = pos, vel
    for s in range(40):
        P.step = s
        p, v, best, paired, raw, der, glob, npairs = oracle.step(P, p, v)
        fracs.append(2 * npairs / n)
    assert glob[1] == pytest.approx(e0, rel=1e-12)      # energy conserved every step
    T = v_in ** 2 / 3
    speed = np.linalg.norm(v, axis=1)
    ks = stats.kstest(speed / math.sqrt(T), stats.chi(3).cdf)
    assert ks.pvalue > 1e-3, ks
    assert 0.3 < np.mean(fracs) < 0.7   # about half of the particles scatter per step


def _equilibration_fractions(R2_of_lam, lams_dx, steps=4):
    """Pairs per particle and step in the paper's 2-D equilibration set-up
    (Sect. "Equilibration and Speed-up": 20 particles per c-bin of width
    dx = 0.004, |v| = 10 in random in-plane directions, dt = dx / 60), here on
    40 x 40 periodic c-bins."""
    dx, nc, ppc = 0.004, 40, 20
    L = nc * dx
    n = nc * nc * ppc
    out = []
    for lam_dx in lams_dx:
        pos, vel = inputs.periodic_box(n, seed=1, lo=(0, 0, 0), hi=(L, L, 1), v_in=10.0, vel_dim=2)
        pos[:, 2] = 0.0
        fr = []
        for k in range(steps):
            P = oracle.make_params(2, (nc, nc, 1), (0, 0, 0), (L, L, 1), (0, 0, 0), R2=R2_of_lam(lam_dx * dx, n / L ** 2),
                                   dt=dx / 60, seed=3, step=k, vel_dim=2)
            pos, vel, _, _, _, _, _, npairs = oracle.step(P, pos, vel)
            fr.append(2 * npairs / n)
        out.append(float(np.mean(fr)))
    return out


def test_collision_fraction_of_the_equilibration_setup():
    """The paper prints about 50 %, 25 % and 3 % of the particles scattering
    per step for lambda = 1e-3, 1 and 10 dx in its 2-D equilibration runs
    (parity unpinned for the exact values: the figures are approximate).
    With the contact distance of Eq. reff_lambda taken literally in 2-D (the
    reading the library follows, n = N / area) the reach R = 63, 2 and 0.6 dx
    covers every approaching neighbour and the fraction saturates near 57 %
    at all three lambda.  With the 2-D mean free path lambda = 1 / (n 2R) the
    printed trend returns (57 %, 18 %, 2 %): the printed fractions follow the
    2-D reading, the printed formula the 3-D one."""
    lams = (1e-3, 1.0, 10.0)
    literal = _equilibration_fractions(lambda lam, nbar: oracle.contact_R2(lam, 0.0, nbar), lams)
    assert all(0.5 < f < 0.65 for f in literal), literal
    planar = _equilibration_fractions(lambda lam, nbar: (1.0 / (2.0 * lam * nbar)) ** 2, lams)
    assert 0.45 < planar[0] < 0.65 and 0.12 < planar[1] < 0.30 and 0.01 < planar[2] < 0.05, planar


def test_maxwellian_stays_maxwellian():
    n = 20000
    pos, vel = inputs.periodic_box(n, seed=12, T=2.0)
    P = params(n_cells=(10, 10, 10), bc=(0, 0, 0), R2=oracle.contact_R2(1e-3, 0, n), dt=0.005)
    p, v = pos, vel
    for s in range(10):
        P.step = s
        p, v = oracle.step(P, p, v)[:2]
    se = math.sqrt(2.0 / n)
    assert np.abs(v.mean(0)).max() < 4 * se
    assert np.abs((v ** 2).mean(0) - 2.0).max() < 4 * 2.0 * math.sqrt(2.0 / n)
    kurt = (v ** 4).mean(0) / (v ** 2).mean(0) ** 2
    assert np.abs(kurt - 3.0).max() < 4 * math.sqrt(96.0 / n)


def test_deterministic_given_seed_and_step():
    pos, vel = inputs.sod_tube(3000, seed=4)
    P = params(n_cells=(20, 1, 1), R2=oracle.contact_R2(1e-3, 0, 3000), dt=1e-3, seed=99, step=3)
    a = oracle.step(P, pos, vel)
    b = oracle.step(P, pos, vel)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])
    P.step = 4
    c = oracle.step(P, pos, vel)
    assert not np.array_equal(a[1], c[1])


def _sod_l1(raw, n, t, nb):
    from analytic import riemann
    k = raw.shape[0] // nb
    R = raw.reshape(nb, k, 8).sum(1)
    N = R[:, 0]
    u = R[:, 1] / N
    c2 = (R[:, 4] + R[:, 5] + R[:, 6]) / N - (R[:, 1:4] ** 2).sum(1) / N ** 2
    dens = N * nb
    n_l = n * 8 / 9 / 0.5
    T = c2 / 3
    ex = riemann.sod_profile(np.linspace(0, 1, nb + 1), t, 0.5, 1.0, 1.0)
    out = {}
    for name, q, qe in (("n", dens / n_l, ex[:, 0]), ("u", u, ex[:, 1]), ("p", dens * T / n_l, ex[:, 2]),
                        ("T", T, ex[:, 3])):
        out[name] = float(np.abs(q - qe).sum() / np.abs(qe).sum())
    return out


def test_sod_tube_against_exact_riemann_small():
    """Sect. "Sod test" at a size the oracle finishes in seconds (20k particles,
    50 c-bins, lambda = 1e-3, t = 0.2).  At this resolution the method's
    collision rate (at most one partner per step) smears the waves, so the
    bound is loose (calibrated: collisional 7-8 % in n, 9-10 % in p and T over
    25 output bins; free streaming 10-11 %, 17-19 %, 16-18 %).  The 2 % bound of
    the shock-tube workload is checked on the device path at 16M particles."""
    n, nc = 20000, 50
    pos, vel = inputs.sod_tube(n, 1)
    P = params(n_cells=(nc, 1, 1), R2=oracle.contact_R2(1e-3, 0, n), dt=0.2 / nc, seed=1)
    steps = 50
    for s in range(steps):
        P.step = s
        pos, vel, best, paired, raw, der, glob, npairs = oracle.step(P, pos, vel)
    err = _sod_l1(raw, n, steps * P.dt, 25)
    assert err["n"] < 0.095 and err["p"] < 0.125 and err["T"] < 0.125, err


def test_sod_tube_in_cubic_c_bins_against_exact_riemann():
    """Sect. "Sod test" in the paper's geometry (cubic c-bins, 20 particles per
    c-bin): 128 x 8 x 8 c-bins over 1 x 1/16 x 1/16 (164k particles), lambda/L =
    1e-3, t = 0.1.  The oracle's profiles, summed over y and z into 32 output
    bins, are within 3.5 % (n) and 4 % (p, T) relative L1 of the exact Riemann
    solution (calibrated: 2.7 %, 3.3 %, 3.1 %; at this resolution the counting
    noise of about 5,000 particles per output bin and the c-bin width 1/128 set
    the floor; the device reaches 1.3 %, 1.1 %, 1.8 % at 1/1024 with 21M)."""
    from analytic import riemann
    ncx, nyz = 128, 8
    L = nyz / ncx
    n = ncx * nyz * nyz * 20
    pos, vel = inputs.sod_tube(n, 1, hi=(1, L, L))
    P = params(n_cells=(ncx, nyz, nyz), hi=(1, L, L), R2=oracle.contact_R2(1e-3, 0, n / (L * L)), dt=0.2 / ncx,
               seed=1)
    steps = int(round(0.1 / P.dt))
    for s in range(steps):
        P.step = s
        pos, vel, best, paired, raw, der, glob, npairs = oracle.step(P, pos, vel)
    rx = raw.reshape(-1, ncx, 8).sum(0)   # rows are c_x fastest: sum over y and z
    nb = 32
    R = rx.reshape(nb, ncx // nb, 8).sum(1)
    N = R[:, 0]
    T = ((R[:, 4] + R[:, 5] + R[:, 6]) / N - (R[:, 1:4] ** 2).sum(1) / N ** 2) / 3
    dens = N * nb / (n * 8 / 9 / 0.5)
    ex = riemann.sod_profile(np.linspace(0, 1, nb + 1), steps * P.dt, 0.5, 1.0, 1.0)
    l1 = [float(np.abs(q - qe).sum() / np.abs(qe).sum()) for q, qe in ((dens, ex[:, 0]), (dens * T, ex[:, 2]),
                                                                     (T, ex[:, 3]))]
    assert l1[0] < 0.035 and l1[1] < 0.04 and l1[2] < 0.04, l1


# ------------------------------------------------------------ adaptive timestep
# Sect. "Simulation setup": dt(t) = dx / v_max(t), v_max the speed of the
# fastest particle; dx the smallest c-bin width (reading for non-square bins).

def test_adaptive_dt_closed_form_345():
    """Fastest particle (3, 4, 0): |v| = 5; c-bins 0.1 x 0.05 -> dt = 0.05 / 5."""
    import oracle
    P = oracle.make_params(2, (10, 20, 1), (0, 0, 0), (1, 1, 1), (0, 0, 0), R2=0.01, dt=1e-3, seed=0)
    vel = np.array([[1.0, 0.0, 0.0], [3.0, 4.0, 0.0], [0.0, 0.0, -2.5], [-4.0, 1.0, 1.0]])
    assert oracle.adaptive_dt(P, vel) == pytest.approx(0.01, rel=2 ** -52)
    P32 = oracle.make_params(2, (10, 20, 1), (0, 0, 0), (1, 1, 1), (0, 0, 0), R2=0.01, dt=1e-3, seed=0, decide32=True)
    assert oracle.adaptive_dt(P32, vel) == pytest.approx(0.01, rel=2 ** -52)


def test_adaptive_dt_at_rest_keeps_given_step():
    import oracle
    P = oracle.make_params(3, (4, 4, 4), (0, 0, 0), (1, 1, 1), (0, 0, 0), R2=0.01, dt=1e-3, seed=0)
    assert oracle.adaptive_dt(P, np.zeros((5, 3)), 0.125) == 0.125


def test_adaptive_dt_no_particle_leaves_its_neighbourhood():
    """Free flight over one adaptive step moves no particle by more than one
    c-bin width in any dimension (the purpose the paper gives for the rule)."""
    import oracle
    from paper_1210_8084_gb300 import inputs
    pos, vel = inputs.periodic_box(5000, seed=4, hi=(1.0, 0.5, 0.25))
    P = oracle.make_params(3, (20, 10, 5), (0, 0, 0), (1.0, 0.5, 0.25), (0, 0, 0), R2=1e-12, dt=1.0, seed=0)
    dt = oracle.adaptive_dt(P, vel)
    P.dt = dt
    p2, v2 = oracle.step(P, pos, vel)[:2]
    assert np.array_equal(v2, vel)                      # R2 ~ 0: no collisions
    w = np.array([0.05, 0.05, 0.05])
    d = np.abs(p2 - pos)
    d = np.minimum(d, np.array([1.0, 0.5, 0.25]) - d)  # periodic
    assert (d <= w * (1 + 1e-12)).all()
    assert np.max(np.linalg.norm(vel, axis=1)) * dt == pytest.approx(0.05, rel=1e-12)


def test_adaptive_dt_follows_the_largest_speed_of_a_maxwellian():
    """N Maxwell speeds (sigma = 1): dx / dt is the largest of N chi(3)
    samples, inside the 1 % - 99 % band of that maximum's exact distribution
    F(x)^N (a mean or rms speed would be far below it)."""
    import oracle
    from scipy import stats
    n = 2_000_000
    vel = np.random.default_rng(12).normal(0.0, 1.0, (n, 3))
    P = oracle.make_params(3, (8, 8, 8), (0, 0, 0), (1, 1, 1), (0, 0, 0), R2=0.01, dt=1.0, seed=0)
    vmax = (1.0 / 8) / oracle.adaptive_dt(P, vel)
    lo = stats.chi(3).ppf(0.01 ** (1.0 / n))
    hi = stats.chi(3).ppf(0.99 ** (1.0 / n))
    assert lo < vmax < hi, (lo, vmax, hi)


# ------------------------------------------------- 2-D velocities (f = 2, gamma = 2)
# The paper's 2-D runs (gamma = 2, Sect. "Sod test"): velocities in the plane,
# outgoing directions isotropic in the plane.

def _box2d(n, seed, **kw):
    from paper_1210_8084_gb300 import inputs
    pos, vel = inputs.periodic_box(n, seed=seed, vel_dim=2, **kw)
    pos[:, 2] = 0.0
    return pos, vel


def test_velocity2d_collisions_conserve_and_stay_in_plane():
    import oracle
    pos, vel = _box2d(20_000, 31)
    P = oracle.make_params(2, (30, 30, 1), (0, 0, 0), (1, 1, 1), (0, 0, 0), R2=2e-4, dt=0.01, seed=5,
                           vel_dim=2)
    p, v = pos, vel
    npairs = 0
    for s in range(5):
        P.step = s
        p, v, best, paired, raw, der, glob, k = oracle.step(P, p, v)
        npairs += k
    assert npairs > 1000
    assert np.all(v[:, 2] == 0.0)
    assert np.allclose(v.sum(0), vel.sum(0), atol=1e-9)
    assert (v ** 2).sum() == pytest.approx((vel ** 2).sum(), rel=1e-12)


def test_velocity2d_gas_relaxes_to_the_2d_maxwell_speed_law():
    """Mono-energetic in the plane, |v| = v_in: the speeds relax to the
    Rayleigh law with T = v_in^2 / 2 (two degrees of freedom); a scatter that
    left the plane or favoured a direction would not."""
    import oracle
    from scipy import stats
    v_in = 2.0
    pos, vel = _box2d(30_000, 32, v_in=v_in)
    P = oracle.make_params(2, (40, 40, 1), (0, 0, 0), (1, 1, 1), (0, 0, 0), R2=3e-4, dt=0.004, seed=6,
                           vel_dim=2)
    p, v = pos, vel
    for s in range(60):
        P.step = s
        p, v = oracle.step(P, p, v)[:2]
    T = v_in ** 2 / 2
    speed = np.linalg.norm(v, axis=1)
    assert stats.kstest(speed / math.sqrt(T), stats.rayleigh.cdf).pvalue > 1e-3
    assert stats.kstest(speed / math.sqrt(T), stats.chi(3).cdf).pvalue < 1e-6


def test_velocity2d_temperature_has_two_degrees_of_freedom():
    import oracle
    pos, vel = _box2d(200_000, 33, T=1.7)
    P = oracle.make_params(2, (1, 1, 1), (0, 0, 0), (1, 1, 1), (0, 0, 0), R2=1e-6, dt=0.01, seed=0, vel_dim=2)
    raw, der, glob = oracle.moments(P, pos, vel)
    assert der[0, 4] == pytest.approx(1.7, rel=0.01)
    P3 = oracle.make_params(2, (1, 1, 1), (0, 0, 0), (1, 1, 1), (0, 0, 0), R2=1e-6, dt=0.01, seed=0)
    assert oracle.moments(P3, pos, vel)[1][0, 4] == pytest.approx(1.7 * 2 / 3, rel=0.01)


# ------------------------------------------------------- absorbing walls (Sedov)
# Sect. "Sedov test": particles that leave the box through an absorbing wall
# are no longer evolved.

def test_absorbing_walls_remove_exactly_the_particles_that_leave():
    """Free flight (no collisions): a particle is removed iff r + v dt lies
    outside the box in an absorbing dimension; removed particles stay removed,
    are nobody's candidate, and leave the moments."""
    import oracle
    from paper_1210_8084_gb300 import inputs
    pos, vel = inputs.periodic_box(4000, seed=51, T=4.0)
    ABS, PER = 2, 0
    P = oracle.make_params(3, (6, 6, 6), (0, 0, 0), (1, 1, 1), (ABS, PER, ABS), R2=1e-14, dt=0.05, seed=1)
    p1, v1, best, paired, raw, der, glob, k = oracle.step(P, pos, vel)
    end = pos + vel * 0.05
    out = (end[:, 0] < 0) | (end[:, 0] > 1) | (end[:, 2] < 0) | (end[:, 2] > 1)
    assert 50 < out.sum() < 3000
    assert np.array_equal(np.isnan(p1[:, 0]), out)
    assert np.all(np.isnan(v1[out])) and np.all(np.isfinite(v1[~out]))
    assert glob[0] == (~out).sum()
    assert glob[1] == pytest.approx(0.5 * (vel[~out] ** 2).sum(), rel=1e-12)
    # a second step: removed particles stay removed and are never candidates
    P.R2 = 1e-3
    P.step = 1
    p2, v2, best2 = oracle.step(P, p1, v1)[:3]
    assert np.all(np.isnan(p2[out, 0]))
    assert np.all(best2[out] == -1)
    assert not np.isin(best2[best2 >= 0], np.nonzero(out)[0]).any()


@pytest.mark.parametrize("dim", [2, 3])
def test_virial_pressure_of_one_hand_placed_pair(dim):
    """The collisional pressure of a single pair, from the stress definition
    (Eq. stress, collisional part r_ij . dp_i at the point of closest approach,
    Eq. 18: p = trace / (d V)), with the pair's impulse counted once for each
    partner and divided by the step (the reading of the garbled virial).  Two
    particles pass each other along x with speeds +-u and impact parameter b
    (along y), so r_ij(t_poca) = (0, b, 0) exactly, whatever the outgoing
    direction: p_vir = 2 b u n_y / (2 d V_c dt) with n = v_i' / u read off the
    oracle's own post-collision velocity.  A virial taken at the start of the
    step (r_ij = (-2a, b, 0)), a dropped partner, a wrong sign or a wrong
    normalisation all change it.  Kinetic part: T = u^2 / f, p_kin = n T."""
    a, b, u = 0.125, 0.0625, 2.0
    dt = 2 * a / u
    lo, hi = (0.0, 0.0, 0.0), (1.0, 1.0, 1.0)
    P = params(dim=dim, n_cells=(1, 1, 1), lo=lo, hi=hi, bc=(0, 0, 0), R2=4 * b * b, dt=dt, seed=77)
    pos = np.array([[0.5 - a, 0.5 + b / 2, 0.5], [0.5 + a, 0.5 - b / 2, 0.5]])
    vel = np.array([[u, 0.0, 0.0], [-u, 0.0, 0.0]])
    seen = 0
    for step in range(6):
        P.step = step
        best = oracle.best_partners(P, pos, vel)
        assert list(best) == [1, 0]
        po, vo, W, paired = oracle.collide_move(P, pos, vel, best)
        assert list(paired) == [1, 0]
        n_hat = vo[0] / u
        assert np.allclose(vo[1], -vo[0], atol=1e-15) and abs(np.linalg.norm(n_hat) - 1) < 1e-14
        raw, der, glob = oracle.moments(P, po, vo, W)
        Vc = 1.0
        expect_w = 2 * b * u * n_hat[1]
        assert raw[0, 7] == pytest.approx(expect_w, abs=1e-14)
        assert der[0, 6] == pytest.approx(expect_w / (2 * dim * Vc * dt), abs=1e-13)
        # kinetic part: bulk velocity 0, v_rms^2 = u^2, f = 3 velocity components
        assert der[0, 4] == pytest.approx(u * u / 3, rel=1e-14)
        assert der[0, 5] == pytest.approx(2 / Vc * u * u / 3, rel=1e-14)
        assert der[0, 7] == pytest.approx(der[0, 5] + der[0, 6], rel=1e-14)
        seen += abs(n_hat[1]) > 0.1
    assert seen >= 2   # the draws give outgoing directions with a real y component


def test_radial_velocity_closed_forms():
    """Eq. vel_r, v_r = (1/N) Sum v . r_hat: a cold radial inflow -v0 r_hat
    gives v_r = -v0 in every occupied c-bin; a rigid rotation about the centre
    gives 0; one hand-placed particle gives v . r / |r| over the position
    dimensions only (z ignored in 2-D)."""
    c = np.array([0.2, 0.3, 0.6])
    P = params(dim=3, n_cells=(4, 4, 4), bc=(1, 1, 1))
    g = np.random.default_rng(5)
    pos = g.random((5000, 3))
    r = pos - c
    rhat = r / np.linalg.norm(r, axis=1, keepdims=True)
    out = oracle.radial(P, pos, -2.5 * rhat, c)
    occ = oracle.moments(P, pos, rhat)[0][:, 0] > 0
    assert np.allclose(out[occ, 1], -2.5, rtol=0, atol=1e-13)
    assert np.allclose(out[occ, 0], -2.5 * oracle.moments(P, pos, rhat)[0][occ, 0], rtol=1e-13)
    omega = np.array([0.3, -1.1, 0.7])
    out = oracle.radial(P, pos, np.cross(omega, r), c)
    assert np.abs(out[:, 1]).max() < 1e-13
    P2 = params(dim=2, n_cells=(2, 2, 1), bc=(1, 1, 0))
    one = oracle.radial(P2, np.array([[0.3, 0.8, 0.9]]), np.array([[1.0, 2.0, 3.0]]), np.array([0.1, 0.4, 0.0]))
    key, _ = oracle.cell_keys(P2, np.array([[0.3, 0.8, 0.9]]))
    assert one[key[0], 1] == pytest.approx((0.2 * 1.0 + 0.4 * 2.0) / math.sqrt(0.2 ** 2 + 0.4 ** 2), rel=1e-15)
    assert np.count_nonzero(one[:, 0]) == 1


# ------------------------------------------------- DSMC comparison variant

def _dsmc_params(n, nc=(8, 8, 8), lam=1e-2, dt=2e-3, T=1.0, seed=4, dim=3):
    P = params(dim=dim, n_cells=nc, bc=(0, 0, 0), R2=oracle.contact_R2(lam, 0, n), dt=dt, seed=seed)
    pos, vel = inputs.periodic_box(n, seed=seed, T=T)
    return P, pos, vel


def test_dsmc_collisions_conserve_momentum_and_energy():
    """Every accepted pair of the random-partner variant scatters in its CM
    frame: total momentum and kinetic energy of the box are unchanged (to
    rounding), and particles that took part have new velocities."""
    P, pos, vel = _dsmc_params(30_000)
    v, collided, acc = oracle.dsmc_collide(P, pos, vel)
    assert acc > 1000
    assert np.abs(v.sum(0) - vel.sum(0)).max() < 1e-10
    assert abs((v * v).sum() / (vel * vel).sum() - 1) < 1e-13
    assert np.all((v != vel).any(1) == (collided == 1))


def test_dsmc_collision_rate_is_the_kinetic_rate():
    """Bird's no-time-counter scheme accepts, per c-bin and step, on average
    1/2 N (N - 1) sigma <g> dt / V_c pairs (<g> the mean relative speed of the
    cell's pairs), i.e. a collision frequency n sigma <g> per particle pair
    density; sigma from Eq. 7.  Summed over the c-bins of a homogeneous box and
    several steps, the accepted count agrees with the brute-force expectation
    within 4 Poisson standard deviations."""
    P, pos, vel = _dsmc_params(6_000, nc=(4, 4, 4), lam=0.02, dt=1.5e-3)
    key, _ = oracle.cell_keys(P, pos)
    sigma = math.pi * P.R2
    Vc = 1.0 / 64
    expect, got = 0.0, 0
    p, v = pos, vel
    for step in range(6):
        P.step = step
        for c in range(64):
            vc = v[key == c]
            N = len(vc)
            g = np.linalg.norm(vc[:, None, :] - vc[None, :, :], axis=2)
            mean_g = g.sum() / (N * (N - 1))
            expect += 0.5 * N * (N - 1) * sigma * mean_g * P.dt / Vc
        v, collided, acc = oracle.dsmc_collide(P, p, v)
        got += acc
    assert expect > 2000
    assert abs(got - expect) < 4 * math.sqrt(expect), (got, expect)


def test_dsmc_mono_energetic_gas_relaxes_to_maxwell():
    """A gas with one speed relaxes under the random-partner collisions to the
    Maxwell speed law at T = v_in^2 / 3 (Kolmogorov-Smirnov)."""
    from scipy import stats
    n = 20_000
    P = params(dim=3, n_cells=(6, 6, 6), bc=(0, 0, 0), R2=oracle.contact_R2(1e-2, 0, n), dt=5e-3, seed=8)
    pos, vel = inputs.periodic_box(n, seed=8, v_in=1.0)
    p, v = pos, vel
    for step in range(40):
        P.step = step
        p, v, collided, acc = oracle.dsmc_step(P, p, v)
    s = np.linalg.norm(v, axis=1)
    T = 1.0 / 3.0
    ks = stats.kstest(s / math.sqrt(T), stats.maxwell.cdf)
    assert ks.pvalue > 1e-3, ks
