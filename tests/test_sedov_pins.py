"""Pins of the Sedov-Taylor similarity solution (oracle/sedov.py) against
conservation laws the integration does not use."""
import numpy as np
import pytest

from analytic import sedov

CASES = [(3, 5.0 / 3.0), (2, 5.0 / 3.0), (2, 2.0), (1, 1.4), (3, 1.4)]


@pytest.mark.parametrize("j,gamma", CASES)
def test_energy_first_integral_holds_along_the_profile(j, gamma):
    """Energy conservation through every sphere that moves with the profile
    gives P / G = (gamma - 1) V^2 (1 - V) / (2 (gamma V - 1)); the ODEs use only
    mass, momentum and entropy.  Checked where gamma V - 1 > 0.05 (the relation
    is singular at the centre, where V -> 1 / gamma)."""
    xi, V, G, P = sedov.profile(j, gamma)
    ok = gamma * V - 1.0 > 0.05
    assert ok.sum() > 50
    lhs = P[ok] / G[ok]
    rhs = (gamma - 1.0) * V[ok] ** 2 * (1.0 - V[ok]) / (2.0 * (gamma * V[ok] - 1.0))
    assert np.max(np.abs(lhs / rhs - 1.0)) < 1e-7


@pytest.mark.parametrize("j,gamma", CASES)
def test_all_swept_mass_is_inside_the_shock(j, gamma):
    """j int_0^1 G xi^(j-1) dxi = 1: the shell holds the mass of the uniform
    sphere (cylinder, slab) it swept up."""
    xi, V, G, P = sedov.profile(j, gamma)
    mass = np.trapezoid((G * xi ** (j - 1))[::-1], xi[::-1])
    assert j * mass == pytest.approx(1.0, abs=2e-4)


@pytest.mark.parametrize("j,gamma", CASES)
def test_centre_is_homologous(j, gamma):
    """Near the centre the hot, rarefied gas expands homologously with
    v = a r / (gamma t), i.e. V -> 1 / gamma, and the density vanishes."""
    xi, V, G, P = sedov.profile(j, gamma)
    assert V[-1] == pytest.approx(1.0 / gamma, rel=1e-4)
    assert G[-1] < 1e-2 * G[0]


def test_classical_constant_of_the_monatomic_spherical_blast():
    """r_s = beta (E t^2 / rho0)^(1/5) with beta close to 1.15 for gamma = 5/3
    (the textbook value of the spherical point blast)."""
    beta = sedov.alpha(3, 5.0 / 3.0) ** (-1.0 / 5.0)
    assert 1.14 < beta < 1.16
