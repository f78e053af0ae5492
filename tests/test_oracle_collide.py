"""Pins of the oracle's collision step (Eqs. monteCarloInt, collision_step,
rinorm_a, correzione)."""
from math import erf

import numpy as np

import oracle
from paper_1005_5405_gb300 import workloads


def _cell(nv=12, vmax=4.0, nt=4000, seed=3, eps=0.1, nx=1, ny=1, **kw):
    return oracle.Oracle(nx=nx, ny=ny, kn=1.0, nv=nv, vmax=vmax, nt=nt, seed=seed, eps=eps, **kw)


def _psi(o):
    V = o.velocities()
    return np.stack([np.ones(len(V)), V[:, 0], V[:, 1], V[:, 2], (V ** 2).sum(1)])


def test_zero_state_is_exact_fixed_point():
    """h = 0 gives g = 0 for every sample, so nothing changes (bit-exact)."""
    o = _cell(nx=3, ny=2)
    h = np.zeros((o.nr, o.nvt))
    out, mom = o.collide(h, step=0)
    assert np.array_equal(out, h) and np.array_equal(mom, np.zeros_like(mom))


def test_single_collision_conserves_mass_in_N_space():
    """P3: one in-box sample moves as much N = w h out of v, v1 as it puts
    into v*, v1* (the bracket of Eq. coll8Dim sums to zero)."""
    o = _cell(nt=1, seed=9)
    w = o.weights()
    rng = np.random.default_rng(0)
    for step in range(20):
        s = o.samples(step)
        if (s["idx"] < 0).any():
            continue
        h = rng.normal(size=(1, o.nvt))
        _, _, stage = o.collide(h, step=step, samples=s, with_stage=True)
        dN = (stage - h) * w
        assert abs(dN.sum()) < 1e-16 + 1e-14 * np.abs(dN).sum()
        assert np.count_nonzero(np.abs(dN) > 1e-300) <= 4


def test_correction_restores_conserved_moments():
    """P4: after the correction, sum w psi h^{n+1} = sum w psi h~ for
    psi = 1, v, |v|^2, although the uncorrected h_c misses them."""
    p = workloads.small(nx=3, ny=2, nv=12, vmax=4.0)
    h = workloads.warm_state(p, seed=11, noise=0.05)
    o = _cell(nx=3, ny=2, nt=5000)
    out, _, stage = o.collide(h, step=4, with_stage=True)
    w = o.weights()
    P = _psi(o) * w
    pre, post, raw = h @ P.T, out @ P.T, stage @ P.T
    scale = np.abs(h) @ np.abs(P).T
    assert np.max(np.abs(post - pre) / scale) < 1e-12
    assert np.max(np.abs(raw[:, 1:] - pre[:, 1:]) / scale[:, 1:]) > 1e-8


def test_homogeneous_relaxation_keeps_rho_u_theta():
    p = workloads.small(nx=2, ny=1, nv=12, vmax=4.0)
    h = workloads.warm_state(p, seed=2)
    o = _cell(nx=2, ny=1, nt=3000, eps=0.2)
    m0 = o.moments(h)
    for n in range(5):
        h, m = o.collide(h, step=n)
    assert np.allclose(m[:, :5], m0[:, :5], rtol=1e-11, atol=1e-12)
    assert np.max(np.abs(m[:, 5:] - m0[:, 5:])) > 1e-4     # stresses relax


def test_eps_scaling_identity():
    """P7: the scheme is written in f = Phi0 (1 + eps h), so running with
    (eps, h) and (2 eps, h / 2) gives the same eps h (streaming, walls,
    collision and correction)."""
    p = workloads.small(nx=4, ny=4, nv=10, vmax=4.0)
    h = workloads.warm_state(p, seed=5)
    a = oracle.Oracle(nx=4, ny=4, kn=1.0, nv=10, vmax=4.0, nt=2000, seed=8, eps=0.1, lid_u0=0.08)
    b = oracle.Oracle(nx=4, ny=4, kn=1.0, nv=10, vmax=4.0, nt=2000, seed=8, eps=0.2, lid_u0=0.08)
    ha, hb = h.copy(), h / 2
    for n in range(3):
        ha, _ = a.step(ha, n)
        hb, _ = b.step(hb, n)
    assert np.max(np.abs(0.1 * ha - 0.2 * hb)) < 1e-12 * np.max(np.abs(0.1 * ha))


def test_hard_sphere_stress_relaxation_rate():
    """P6: an anisotropic Maxwellian h = v_x^2 - v_y^2 relaxes its normal
    stress difference at p0/mu_1 = 1.016034 per lambda0/V0 (first Sonine
    approximation; lambda0 uses the exact hard-sphere viscosity).  The discrete
    rate converges as dv^2; extrapolate from two grids."""
    rates = {}
    for nv, vmax in ((24, 4.5), (32, 5.0)):
        o = _cell(nv=nv, vmax=vmax, nt=300_000, seed=11, eps=1e-3)
        V = o.velocities()
        w = o.weights()
        q = V[:, 0] ** 2 - V[:, 1] ** 2
        h = q[None, :].copy()
        P0 = 2 * np.sum(w * h[0] * q)
        r = []
        for step in range(6):
            h1, _ = o.collide(h, step=step)
            r.append(-(2 * np.sum(w * h1[0] * q) - P0) / (P0 * o.dt))
        rates[o.dv] = np.mean(r)
    (d1, r1), (d2, r2) = sorted(rates.items())
    r0 = (r2 * d1 ** 2 - r1 * d2 ** 2) / (d1 ** 2 - d2 ** 2)
    assert abs(r0 - 1.016034) < 0.04, (rates, r0)
    assert 1.0 < r1 < 1.12


def _collision_frequency(r):
    """nu(v) = int Phi0(v1) |v - v1| dv1 for Phi0 = pi^{-3/2} e^{-v^2}."""
    return np.exp(-r * r) / np.sqrt(np.pi) + (r + 0.5 / r) * np.vectorize(erf)(r)


def test_collision_frequency_closed_form():
    rng = np.random.default_rng(3)
    x = rng.normal(scale=np.sqrt(0.5), size=(400_000, 3))
    for r in (0.3, 1.0, 2.2):
        v = np.array([r, 0.0, 0.0])
        mc = np.linalg.norm(x - v, axis=1).mean()
        assert abs(mc - _collision_frequency(r)) < 4e-3


def test_loss_term_against_closed_form():
    """For h = 1 on a single node j0 the loss part of Eq. coll8Dim is
    pi K [ int_C Phi0 nu dv + (1 + eps) int_C int_C Phi0 Phi01 |v - v1| ],
    using E_k |k.v_r| = |v_r| / 2."""
    o = _cell(nv=4, vmax=2.0, nt=2_000_000, seed=3, eps=0.5)
    j0 = (1 * 4 + 2) * 4 + 1
    h = np.zeros(64)
    h[j0] = 1.0
    gain, loss = o.mc_dNdt(h)
    a, dv = o.node_v(), o.dv
    c = np.array([a[1], a[2], a[1]])

    def cell_rule(n):
        x, w = np.polynomial.legendre.leggauss(n)
        x, w = x * dv / 2, w * dv / 2
        X = np.stack(np.meshgrid(c[0] + x, c[1] + x, c[2] + x, indexing="ij"), -1).reshape(-1, 3)
        Wt = np.einsum("i,j,k->ijk", w, w, w).ravel()
        return X, Wt * np.pi ** -1.5 * np.exp(-(X ** 2).sum(1))

    X, wp = cell_rule(10)
    I1 = np.sum(wp * _collision_frequency(np.linalg.norm(X, axis=1)))
    X, wp = cell_rule(8)
    I2 = np.einsum("i,j,ij->", wp, wp, np.linalg.norm(X[:, None] - X[None], axis=2))
    expect = np.pi * oracle.K_HARD_SPHERE * (I1 + (1 + o.eps) * I2)
    assert abs(loss[j0] - expect) < 5e-3 * expect
    # mass: gains and losses balance over the box for in-box samples
    s = o.samples(0)
    inbox = (s["idx"] >= 0).all(1)
    assert inbox.mean() > 0.5


def test_drifting_maxwellian_is_statistical_fixed_point():
    """P5: for h = (exp(2 eps u.v - eps^2 u^2) - 1)/eps, g (1+...) is a
    collision invariant, so dN/dt vanishes up to grid bias and noise, while a
    random h of the same size does not."""
    eps = 0.5
    o = _cell(nv=16, vmax=4.0, nt=1_000_000, seed=7, eps=eps)
    V = o.velocities()
    u = np.array([0.6, -0.3, 0.2])
    hM = (np.exp(2 * eps * V @ u - eps ** 2 * u @ u) - 1) / eps
    g, l = o.mc_dNdt(hM)
    resid = np.linalg.norm(g - l) / np.linalg.norm(l)
    hr = np.random.default_rng(1).normal(size=hM.size) * np.std(hM)
    g3, l3 = o.mc_dNdt(hr)
    assert resid < 0.12
    assert np.linalg.norm(g3 - l3) / np.linalg.norm(l3) > 0.5


def test_h_theorem_windowed():
    """P8: the H-function sum dV f ln f of a bimodal positive f decreases
    over windows of steps in homogeneous relaxation."""
    eps = 1.0
    o = oracle.Oracle(nx=1, ny=1, kn=10.0, nv=16, vmax=4.5, nt=20_000, seed=21, eps=eps)
    V = o.velocities()
    w = o.weights()
    dV = o.dv ** 3
    phi0 = w / dV
    f = 0.5 * np.pi ** -1.5 * (np.exp(-((V[:, 0] - 0.8) ** 2) - V[:, 1] ** 2 - V[:, 2] ** 2)
                               + np.exp(-((V[:, 0] + 0.8) ** 2) - V[:, 1] ** 2 - V[:, 2] ** 2))
    h = ((f / phi0 - 1) / eps)[None, :]

    def H(hh):
        ff = phi0 * (1 + eps * hh[0])
        ff = np.where(ff > 0, ff, 1e-300)
        return np.sum(dV * ff * np.log(ff))

    Hs = [H(h)]
    for n in range(30):
        h, _ = o.collide(h, step=n)
        Hs.append(H(h))
    Hs = np.array(Hs)
    win = Hs[::10]
    assert np.all(np.diff(win) < 0), Hs
    assert Hs[-1] < Hs[0] - 1e-3
