"""Pins of the exact Noh solution (oracle/noh.py) against conservation laws
and the jump conditions, not against its own formulas."""
import math

import numpy as np
import pytest

from analytic import noh


def _shell_volume(r0, r1, d):
    c = {1: 2.0, 2: math.pi, 3: 4.0 * math.pi / 3.0}[d]
    return c * (r1 ** d - r0 ** d)


@pytest.mark.parametrize("d,gamma", [(1, 5 / 3), (2, 5 / 3), (2, 2.0), (3, 5 / 3)])
def test_mass_inside_radius_equals_initial_mass_inside_r_plus_v0t(d, gamma):
    """All matter inside R at time t started inside R + v0 t (it moved inward
    at v0 or has stopped inside the shock)."""
    v0, n0, t, R = 1.3, 2.0, 0.7, 2.5
    edges = np.linspace(0.0, R, 400_001)
    mid = 0.5 * (edges[1:] + edges[:-1])
    n = noh.profile(mid, t, v0, n0, gamma, d)[0]
    # integrate exactly the piecewise profile: midpoint rule on a fine grid
    mass = np.sum(n * np.array([_shell_volume(a, b, d) for a, b in zip(edges[:-1], edges[1:])]))
    assert mass == pytest.approx(n0 * _shell_volume(0.0, R + v0 * t, d), rel=2e-4)


@pytest.mark.parametrize("d,gamma", [(1, 5 / 3), (2, 2.0), (3, 5 / 3), (3, 1.4)])
def test_rankine_hugoniot_at_the_shock(d, gamma):
    """Mass, momentum and energy fluxes through the moving shock match
    (upstream: density n1 falling in at v0, cold; downstream: at rest)."""
    v0, n0, t = 1.0, 1.0, 0.5
    rs = noh.shock_radius(t, v0, gamma)
    n1 = noh.profile(rs * (1 + 1e-12), t, v0, n0, gamma, d)[0]
    n2, u2, p2, T2 = noh.profile(rs * (1 - 1e-12), t, v0, n0, gamma, d)
    vs = rs / t
    w1 = v0 + vs                          # upstream speed relative to the shock
    w2 = vs                               # downstream (at rest) relative to the shock
    assert n1 * w1 == pytest.approx(n2 * w2, rel=1e-9)                           # mass
    assert n1 * w1 ** 2 == pytest.approx(n2 * w2 ** 2 + p2, rel=1e-9)           # momentum (p1 = 0)
    h2 = gamma / (gamma - 1.0) * T2       # enthalpy per particle downstream
    assert 0.5 * w1 ** 2 == pytest.approx(0.5 * w2 ** 2 + h2, rel=1e-9)        # energy
    assert u2 == 0.0


def test_strong_shock_compression_is_4_per_dimension_for_monatomic_gas():
    assert noh.shocked_density(1.0, 5 / 3, 3) == pytest.approx(64.0)
    assert noh.shocked_density(1.0, 2.0, 2) == pytest.approx(9.0)    # the paper's 2-D value
