"""Pins of the oracle's free streaming (Eq. streaming2D) and diffuse walls
(Eq. bcMax with the zero-mass-flux condition)."""
import numpy as np

import oracle
from paper_1005_5405_gb300 import workloads


def _o(**kw):
    args = dict(nx=6, ny=5, kn=1.0, nv=8, vmax=3.5, nt=10, seed=1)
    args.update(kw)
    return oracle.Oracle(**args)


def test_rest_state_is_fixed():
    o = _o(lid_u0=0.0, eps=0.1)
    h = np.zeros((o.nr, o.nvt))
    # exact up to the rounding of n_w = 1 (one ulp of the flux sums)
    assert np.max(np.abs(o.stream(h))) < 1e-13


def test_quadratic_profile_closed_form():
    """Interior cells: for h = x^2 + y^2 the upwind scheme gives exactly
    x^2 + y^2 - 2 (x v_x + y v_y) dt + (|v_x| dx + |v_y| dy) dt."""
    o = _o(nx=7, ny=7, lid_u0=0.05)
    L = 1.0
    dx = L / o.nx
    xc = -L / 2 + (np.arange(o.nx) + 0.5) * dx
    yc = (np.arange(o.ny) + 0.5) * dx
    X = np.tile(xc, o.ny)
    Y = np.repeat(yc, o.nx)
    V = o.velocities()
    h = (X ** 2 + Y ** 2)[:, None] * np.ones((1, o.nvt))
    ht = o.stream(h)
    dt = o.dt
    ref = (X ** 2 + Y ** 2)[:, None] - 2 * dt * (X[:, None] * V[None, :, 0] + Y[:, None] * V[None, :, 1]) \
        + dt * (np.abs(V[None, :, 0]) * dx + np.abs(V[None, :, 1]) * dx)
    ix, iy = np.arange(o.nr) % o.nx, np.arange(o.nr) // o.nx
    inner = (ix > 0) & (ix < o.nx - 1) & (iy > 0) & (iy < o.ny - 1)
    assert np.max(np.abs(ht[inner] - ref[inner])) < 1e-14


def test_cfl_one_is_exact_shift():
    """At Courant number 1 along x and 0 along y the update is a shift by one
    cell (odd nv so a node with v_y = 0 exists)."""
    o = _o(nx=6, ny=3, nv=5, vmax=2.5, cfl=1.0, lid_u0=0.0, eps=1.0)
    rng = np.random.default_rng(0)
    h = rng.normal(size=(o.nr, o.nvt))
    ht = o.stream(h)
    n = o.nv
    jp = ((n - 1) * n + n // 2) * n + 1       # v_x max, v_y = 0
    jm = (0 * n + n // 2) * n + 3             # v_x min, v_y = 0
    for c in range(o.nr):
        ix = c % o.nx
        if ix > 0:
            assert abs(ht[c, jp] - h[c - 1, jp]) < 1e-14 * (1 + abs(h[c - 1, jp]))
        if ix < o.nx - 1:
            assert abs(ht[c, jm] - h[c + 1, jm]) < 1e-14 * (1 + abs(h[c + 1, jm]))


def test_wall_density_closed_forms():
    """h = 0: walls at rest emit n_w = 1 (grid symmetry); the tangentially
    moving lid emits n_w = 1 up to the midpoint rule's Gaussian error."""
    o = _o(lid_u0=0.07)
    nw = o.wall_density(np.zeros((o.nr, o.nvt)))
    assert np.max(np.abs(nw[: 2 * o.ny + o.nx] - 1)) < 1e-14
    assert np.max(np.abs(nw[2 * o.ny + o.nx:] - 1)) < 1e-6


def test_zero_net_mass_flux_per_face():
    o = _o(lid_u0=0.1, nv=10, vmax=4.0)
    p = workloads.small(nx=o.nx, ny=o.ny, nv=o.nv, vmax=4.0)
    h = workloads.warm_state(p, seed=3)
    nw = o.wall_density(h)
    V = o.velocities()
    w = o.weights()
    faces = ([(f, f * o.nx, (1, 0)) for f in range(o.ny)]
             + [(o.ny + f, f * o.nx + o.nx - 1, (-1, 0)) for f in range(o.ny)]
             + [(2 * o.ny + f, f, (0, 1)) for f in range(o.nx)]
             + [(2 * o.ny + o.nx + f, (o.ny - 1) * o.nx + f, (0, -1)) for f in range(o.nx)])
    for f, c, (nxh, nyh) in faces:
        vn = V[:, 0] * nxh + V[:, 1] * nyh
        out = np.sum(-vn[vn < 0] * w[vn < 0] * (1 + o.eps * h[c, vn < 0]))
        gin = np.array([o.ghost(0, f, nw[f], j) for j in np.nonzero(vn > 0)[0]])
        inn = np.sum(vn[vn > 0] * w[vn > 0] * (1 + o.eps * gin))
        assert abs(inn - out) < 1e-13 * out


def test_streaming_conserves_mass():
    o = _o(lid_u0=0.1, nv=10, vmax=4.0)
    p = workloads.small(nx=o.nx, ny=o.ny, nv=o.nv, vmax=4.0)
    h = workloads.warm_state(p, seed=4)
    w = o.weights()
    m0 = np.sum(h * w)
    m1 = np.sum(o.stream(h) * w)
    assert abs(m1 - m0) < 1e-12 * np.sum(np.abs(h * w))


def test_lid_shear_closed_form():
    """Gas at rest under a lid moving at U: the x-momentum flux through the
    lid is 2/eps * U * (-1/(2 sqrt(pi))) = -U / (eps sqrt(pi)) in the
    continuum.  The half-range velocity sum has a kink at v_y = 0, so the
    discrete value converges to it as dv^2."""
    errs = []
    for nv in (16, 32, 64):
        U = 0.05
        o = _o(nx=2, ny=2, nv=nv, vmax=4.5, lid_u0=U, eps=0.1)
        d = o.lid_shear(np.zeros((o.nr, o.nvt)))
        exact = -U / (0.1 * np.sqrt(np.pi))
        assert np.allclose(d, d[0], rtol=1e-14)
        errs.append(abs(d[-1] - exact) / abs(exact))
    assert errs[0] < 0.04 and errs[2] < 0.003
    assert 3.5 < errs[0] / errs[1] < 4.5 and 3.5 < errs[1] / errs[2] < 4.5


def test_single_cell_step_matches_full_step():
    """The per-cell oracle entry (used to check sampled cells of large runs)
    reproduces the whole-cavity step bit for bit."""
    o = oracle.Oracle(nx=5, ny=4, kn=1.0, nv=8, vmax=4.0, nt=300, seed=3, lid_u0=0.1)
    p = workloads.small(nx=5, ny=4, nv=8)
    h = workloads.warm_state(p, seed=2)
    full, mom = o.step(h, 2)
    for c in range(o.nr):
        ix, iy = c % 5, c // 5
        out, m = o.step_cell(c, h[c], h[c - 1] if ix > 0 else None, h[c + 1] if ix < 4 else None,
                             h[c - 5] if iy > 0 else None, h[c + 5] if iy < 3 else None, step=2)
        assert np.array_equal(out, full[c])
        assert np.allclose(m, mom[c], rtol=1e-13, atol=1e-15)
