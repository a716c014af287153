"""Self-similar Sedov-Taylor point blast in a uniform cold medium (test
infrastructure only).

Sect. "Sedov test": the shock radius is r_s = (E t^2 / (alpha n0))^(1/(2+j)) with
alpha a constant of order one fixed by gamma (j = 1, 2, 3: planar, cylindrical,
spherical).  The paper does not give alpha; it follows from the similarity
solution computed here.

Scaled variables (m = 1, rho0 = n0): with a = 2 / (2 + j) (r_s ~ t^a) and
xi = r / r_s,
    v = a (r / t) V(xi),   rho = rho0 G(xi),   p = rho0 a^2 (r / t)^2 P(xi).
Mass, momentum and entropy conservation of the Euler equations give, at each xi,
a linear system for (G', V', P') (derivatives in xi):
    xi (V - 1) G' + xi G V'                    = -j G V
    a xi (V - 1) V' + (a xi / G) P'            = V - a V^2 - 2 a P / G
    -gamma xi (V - 1) G' / G + xi (V - 1) P'/P = -2 (a V - 1) / a
integrated inwards from the strong-shock jump at xi = 1:
    V = 2 / (gamma + 1),  G = (gamma + 1) / (gamma - 1),  P = 2 / (gamma + 1).
The blast energy fixes alpha:
    E = Omega_j rho0 a^2 r_s^(j+2) / t^2 * I,  I = int_0^1 (G V^2 / 2 + P / (gamma - 1)) xi^(j+1) dxi,
so alpha = Omega_j a^2 I with Omega_j = 2, 2 pi, 4 pi.
"""
import math

import numpy as np
from scipy.integrate import solve_ivp

_OMEGA = {1: 2.0, 2: 2.0 * math.pi, 3: 4.0 * math.pi}


def _rhs(s, y, j, gamma):
    """Derivatives in s = ln xi (xi d/dxi) of (V, G, P): the system above with
    xi G', xi V', xi P' as unknowns."""
    V, G, P = y
    a = 2.0 / (2.0 + j)
    # unknowns (dG/ds, dV/ds, dP/ds)
    A = np.array([
        [V - 1.0, G, 0.0],
        [0.0, a * (V - 1.0), a / G],
        [-gamma * (V - 1.0) / G, 0.0, (V - 1.0) / P],
    ])
    rhs = np.array([-j * G * V, V - a * V * V - 2.0 * a * P / G, -2.0 * (a * V - 1.0) / a])
    dG, dV, dP = np.linalg.solve(A, rhs)
    return [dV, dG, dP]


def profile(j=3, gamma=5.0 / 3.0, xi_min=0.05, n=2000):
    """(xi, V, G, P) from the shock (xi = 1) inwards to xi_min, xi decreasing.
    Towards the centre V -> 1/gamma, G -> 0 and P grows as xi^-2 (a finite
    central pressure); the approach to that singular point is integrated no
    further than xi_min."""
    y0 = [2.0 / (gamma + 1.0), (gamma + 1.0) / (gamma - 1.0), 2.0 / (gamma + 1.0)]
    s_eval = np.linspace(0.0, math.log(xi_min), n)
    sol = solve_ivp(_rhs, (0.0, math.log(xi_min)), y0, t_eval=s_eval, args=(j, gamma), method="RK45",
                    rtol=1e-9, atol=1e-13)
    if not sol.success:
        raise RuntimeError(sol.message)
    xi = np.exp(sol.t)
    V, G, P = sol.y
    return xi, V, G, P


def alpha(j=3, gamma=5.0 / 3.0, xi_min=0.05):
    """The constant of r_s = (E t^2 / (alpha rho0))^(1/(2+j)).  Inside xi_min the
    energy is that of the constant central pressure (P ~ xi^-2, G -> 0):
    int_0^xi_min P xi^(j+1) / (gamma - 1) dxi = P(xi_min) xi_min^(j+2) / (j (gamma - 1))."""
    xi, V, G, P = profile(j, gamma, xi_min)
    a = 2.0 / (2.0 + j)
    f = (0.5 * G * V * V + P / (gamma - 1.0)) * xi ** (j + 1)
    I = np.trapezoid(f[::-1], xi[::-1]) + P[-1] * xi[-1] ** (j + 2) / (j * (gamma - 1.0))
    return _OMEGA[j] * a * a * I


def shock_radius(E, n0, t, j=3, gamma=5.0 / 3.0, alpha_value=None):
    al = alpha(j, gamma) if alpha_value is None else alpha_value
    return (E * t * t / (al * n0)) ** (1.0 / (2.0 + j))
