"""Pins of the oracle's macroscopic quantities (Eqs. densita..sforzi, written
in V0 = sqrt(2RT0) units)."""
import numpy as np

import oracle


def _o(eps=1e-6, nv=32, vmax=5.0):
    return oracle.Oracle(nx=1, ny=1, kn=1.0, nv=nv, vmax=vmax, nt=1, seed=1, eps=eps)


def test_linear_perturbations():
    """Linearised Maxwellian perturbations return their parameters:
    h = rho0 -> rho; h = 2 u0 v_x -> u_x; h = theta0 (v^2 - 3/2) -> theta;
    h = 2 a v_x v_y -> P_xy = a (with eps -> 0)."""
    o = _o()
    V = o.velocities()
    v2 = (V ** 2).sum(1)
    cases = [
        (0.3 * np.ones(o.nvt), 0, 0.3),
        (2 * 0.2 * V[:, 0], 1, 0.2),
        (2 * -0.4 * V[:, 2], 3, -0.4),
        (0.5 * (v2 - 1.5), 4, 0.5),
        (2 * 0.7 * V[:, 0] * V[:, 1], 8, 0.7),
        (2 * 0.7 * V[:, 1] * V[:, 2], 10, 0.7),
    ]
    for h, k, val in cases:
        m = o.moments(h[None, :])[0]
        assert abs(m[k] - val) < 1e-7, (k, m)
        # O(eps) nonlinear terms (eps = 1e-6) stay below 1e-6
        others = np.delete(np.arange(11), [k] + ([5, 6, 7] if k == 4 else []))
        if k != 0:
            assert np.max(np.abs(m[others])) < 1e-6, (k, m)


def test_nonlinear_shifted_maxwellian():
    """f = n (pi T)^{-3/2} exp(-|v - V|^2 / T) with n = 1 + eps rho0,
    V = eps u0, T = 1 + eps theta0 returns rho0, u0, theta0 (up to the grid
    quadrature) at finite eps, and the isotropic stress of a Maxwellian,
    Pi_ij = (n T - 1) / eps delta_ij."""
    eps = 0.3
    o = _o(eps=eps, nv=40, vmax=6.0)
    V = o.velocities()
    rho0, u0, th0 = 0.4, np.array([0.5, -0.2, 0.1]), 0.25
    n, T = 1 + eps * rho0, 1 + eps * th0
    f = n * (np.pi * T) ** -1.5 * np.exp(-((V - eps * u0) ** 2).sum(1) / T)
    phi0 = np.pi ** -1.5 * np.exp(-(V ** 2).sum(1))
    h = (f / phi0 - 1) / eps
    m = o.moments(h[None, :])[0]
    assert abs(m[0] - rho0) < 1e-8
    assert np.allclose(m[1:4], u0, atol=1e-8)
    assert abs(m[4] - th0) < 1e-8
    # pressure tensor of a Maxwellian: p_ij / p0 = n T delta_ij
    p = (n * T - 1) / eps
    assert np.allclose(m[5:8], p, atol=1e-7) and np.allclose(m[8:], 0, atol=1e-8)
