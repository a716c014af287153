"""Exact solution of the Noh implosion (test infrastructure only).

Sect. "Noh test": a cold gas of density n0 streams towards the origin with
radial speed v0 (zero pressure).  A shock leaves the origin at
r_s = (gamma - 1) v0 t / 2; outside it the gas keeps falling in with density
n0 (1 + v0 t / r)^(d - 1); inside it the gas is at rest with density
n0 ((gamma + 1) / (gamma - 1))^d and all the inflow's kinetic energy turned
into heat.  d = 1, 2, 3 for planar, cylindrical and spherical geometry.
Units m = 1, k_B = 1: p = n T, internal energy per particle T / (gamma - 1).
"""
import numpy as np


def shock_radius(t, v0, gamma):
    return 0.5 * (gamma - 1.0) * v0 * t


def shocked_density(n0, gamma, d):
    return n0 * ((gamma + 1.0) / (gamma - 1.0)) ** d


def profile(r, t, v0, n0, gamma, d):
    """(n, u_r, p, T) at radii r and time t > 0."""
    r = np.asarray(r, dtype=np.float64)
    rs = shock_radius(t, v0, gamma)
    inside = r < rs
    n = np.where(inside, shocked_density(n0, gamma, d), n0 * (1.0 + v0 * t / np.maximum(r, 1e-300)) ** (d - 1))
    u = np.where(inside, 0.0, -v0)
    # the shocked gas holds the inflow's kinetic energy v0^2 / 2 per particle as heat
    T = np.where(inside, (gamma - 1.0) * 0.5 * v0 ** 2, 0.0)
    return n, u, n * T, T
