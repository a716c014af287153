"""Pins of the exact Riemann solver used as the Sod reference.

The solver is checked against the jump conditions it must satisfy, not
against itself: Rankine-Hugoniot conservation of mass, momentum and energy
across the shock, isentropy and the Riemann invariant across the rarefaction,
continuity of pressure and velocity across the contact.
"""
import math

import numpy as np
import pytest

from analytic import riemann

SOD = ((1.0, 0.0, 1.0), (0.125, 0.0, 0.1))


def _state_at(xi, left=SOD[0], right=SOD[1], g=5 / 3):
    r, u, p = riemann.sample(np.array([xi]), left, right, g)
    return float(r[0]), float(u[0]), float(p[0])


@pytest.mark.parametrize("gamma", [5 / 3, 1.4, 2.0])
def test_shock_rankine_hugoniot(gamma):
    ws = riemann.wave_speeds(*SOD, gamma)
    S = ws["right_shock"]
    pre = _state_at(S + 1e-6, g=gamma)
    post = _state_at(S - 1e-6, g=gamma)
    e = lambda r, u, p: p / ((gamma - 1) * r) + 0.5 * u * u    # specific total energy
    m_pre, m_post = pre[0] * (pre[1] - S), post[0] * (post[1] - S)
    assert m_post == pytest.approx(m_pre, rel=1e-10)
    assert post[0] * (post[1] - S) ** 2 + post[2] == pytest.approx(pre[0] * (pre[1] - S) ** 2 + pre[2], rel=1e-10)
    flux_e = lambda r, u, p: r * (u - S) * e(r, u, p) + p * u
    assert flux_e(*post) == pytest.approx(flux_e(*pre), rel=1e-9, abs=1e-12)
    assert post[2] > pre[2] and post[0] > pre[0]    # compressive


@pytest.mark.parametrize("gamma", [5 / 3, 1.4])
def test_rarefaction_isentropic_and_invariant(gamma):
    ws = riemann.wave_speeds(*SOD, gamma)
    head, tail = ws["left_head"], ws["left_tail"]
    r0, u0, p0 = SOD[0]
    c0 = math.sqrt(gamma * p0 / r0)
    for xi in np.linspace(head, tail, 7)[1:-1]:
        r, u, p = _state_at(xi, g=gamma)
        assert p / r ** gamma == pytest.approx(p0 / r0 ** gamma, rel=1e-12)
        c = math.sqrt(gamma * p / r)
        assert u + 2 * c / (gamma - 1) == pytest.approx(u0 + 2 * c0 / (gamma - 1), rel=1e-12)
        assert u - c == pytest.approx(xi, rel=1e-10, abs=1e-12)   # characteristic speed = xi in the fan


def test_contact_continuity_and_star_consistency():
    g = 5 / 3
    ws = riemann.wave_speeds(*SOD, g)
    us = ws["contact"]
    lft = _state_at(us - 1e-9, g=g)
    rgt = _state_at(us + 1e-9, g=g)
    assert lft[2] == pytest.approx(rgt[2], rel=1e-12) == ws["p_star"]
    assert lft[1] == pytest.approx(rgt[1], rel=1e-12)
    assert lft[0] > rgt[0]       # density jumps down across the contact
    # far field is untouched
    assert _state_at(-10.0, g=g) == SOD[0] and _state_at(10.0, g=g) == SOD[1]


def test_cell_average_profile_mass_conservation():
    """Total mass in a closed tube is the initial mass while waves stay inside."""
    edges = np.linspace(0.0, 1.0, 401)
    prof = riemann.sod_profile(edges, 0.15, x0=0.5, n_left=1.0, p_left=1.0)
    mass = prof[:, 0].sum() * (edges[1] - edges[0])
    assert mass == pytest.approx(0.5 * (1.0 + 0.125), rel=2e-4)
    mom = (prof[:, 0] * prof[:, 1]).sum() * (edges[1] - edges[0])
    # momentum = impulse of the pressure difference at the ends: (p_l - p_r) t
    assert mom == pytest.approx((1.0 - 0.1) * 0.15, rel=2e-3)
