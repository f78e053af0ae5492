"""Stretched grids (Sec. 5.1): velocity cells growing outward from the origin
with progression ratio rv, spatial cells shrinking toward the side walls
(rx) and the lid (ry).  Pins from geometry, exact conservation, closed forms
and central differences."""
import numpy as np
import pytest

import oracle
from paper_1005_5405_gb300 import workloads


def _o(**kw):
    base = dict(nx=5, ny=4, kn=1.0, nv=10, vmax=3.0, nt=800, seed=3, eps=0.1,
                rv=0.9, rx=0.8, ry=0.85)
    base.update(kw)
    return oracle.Oracle(**base)


def test_velocity_edges_geometry():
    o = _o(nv=20, vmax=3.0, rv=0.945)
    e = o.axis_edges()
    w = np.diff(e)
    assert abs(e[0] + 3.0) < 1e-14 and abs(e[-1] - 3.0) < 1e-14
    assert np.allclose(e, -e[::-1], rtol=0, atol=1e-15)          # symmetric about 0
    assert e[10] == 0.0
    # outward from the origin each cell is 1/rv times the previous one
    right = w[10:]
    assert np.allclose(right[1:] / right[:-1], 1.0 / 0.945, rtol=1e-12)
    assert np.allclose(w[:10], w[10:][::-1], rtol=1e-13)
    assert w.argmin() in (9, 10) and np.allclose(o.axis_widths(), w, rtol=1e-14)
    v = o.node_v()
    assert np.allclose(v, 0.5 * (e[1:] + e[:-1]), rtol=0, atol=1e-15)


def test_near_uniform_ratio_approaches_uniform_grid():
    a = _o(nv=12, vmax=4.0, rv=1.0 - 1e-9).axis_edges()
    b = _o(nv=12, vmax=4.0, rv=0.0).axis_edges()
    assert np.max(np.abs(a - b)) < 1e-6


def test_spatial_widths_geometry():
    o = _o(nx=9, ny=7, kn=0.5, rx=0.8, ry=0.7)
    dx, dy = o.cell_widths()
    L = 2.0
    assert abs(dx.sum() - L) < 1e-13 and abs(dy.sum() - L) < 1e-13
    assert np.allclose(dx, dx[::-1], rtol=1e-14)                  # symmetric in x
    assert np.allclose(dx[:4] / dx[1:5], 0.8, rtol=1e-13)         # shrinking toward x = -L/2
    assert np.allclose(dy[1:] / dy[:-1], 0.7, rtol=1e-13)         # shrinking toward the lid
    assert dy.argmin() == 6 and dx.argmin() in (0, 8)


def test_node_lookup_matches_brute_force_on_stretched_edges():
    o = _o(nv=10, vmax=3.0, rv=0.8)
    e = o.axis_edges()
    rng = np.random.default_rng(0)
    pts = rng.uniform(-3.4, 3.4, size=(400, 3))
    pts[:20, 0] = e[rng.integers(0, 11, 20)]                       # exactly on edges
    for v in pts:
        j, _ = o.node_of(v)
        ids = []
        for c in range(3):
            k = np.searchsorted(e, v[c], side="right") - 1
            ids.append(k if 0 <= k < 10 and v[c] < e[-1] else -1)
        expect = -1 if min(ids) < 0 else (ids[0] * 10 + ids[1]) * 10 + ids[2]
        assert j == expect, (v, j, expect)


def _mass(o, h):
    dx, dy = o.cell_widths()
    area = np.outer(dy, dx).ravel()            # cell = iy * nx + ix
    return float(area @ (h @ o.weights()))


@pytest.mark.parametrize("rv,rx,ry", [(0.9, 0.8, 0.85), (0.0, 0.7, 0.0), (0.85, 0.0, 0.0)])
def test_full_step_conserves_total_mass(rv, rx, ry):
    """Diffuse walls have zero net mass flux and the upwind update of a cell
    of width dx_i is a flux difference, so sum_c dx dy sum_j w h is exact to
    rounding; using a neighbour's width instead of the cell's own breaks it."""
    o = _o(rv=rv, rx=rx, ry=ry)
    p = workloads.small(nx=5, ny=4, nv=10, vmax=3.0)
    h = workloads.warm_state(p, seed=5)
    m0 = _mass(o, h)
    h1, _ = o.step(h, 0)
    m1 = _mass(o, h1)
    scale = float(np.abs(np.outer(*o.cell_widths()[::-1]).ravel() @ (np.abs(h) @ o.weights())))
    assert abs(m1 - m0) <= 1e-13 * scale, (m0, m1)


def test_upwind_on_nonuniform_cells_linear_profile():
    """h = a x_c (cell centres) in the interior: the update of a cell of width
    dx_i with v_x > 0 is a x_i - (v dt / dx_i) a (x_i - x_{i-1}), where the
    centre distance is (dx_i + dx_{i-1}) / 2."""
    o = _o(nx=9, ny=3, rv=0.0, rx=0.8, ry=0.0)
    dx, _ = o.cell_widths()
    x = np.cumsum(dx) - dx / 2
    a = 0.3
    h = np.repeat(np.tile(a * x, 3)[:, None], o.nvt, axis=1)
    ht = o.stream(h, 0)
    v = o.velocities()
    dt = o.dt
    for ix in range(2, 7):
        c = 1 * 9 + ix                          # middle row: no y gradient
        for j in np.nonzero((v[:, 0] > 0) & (np.abs(v[:, 1]) > 0))[0][:50]:
            expect = a * x[ix] - v[j, 0] * dt / dx[ix] * a * (x[ix] - x[ix - 1])
            assert abs(ht[c, j] - expect) < 1e-13, (ix, j)


def test_collision_conserves_invariants_with_stretched_weights():
    o = _o(rv=0.85, nx=2, ny=2)
    p = workloads.small(nx=2, ny=2, nv=10, vmax=3.0)
    h = workloads.warm_state(p, seed=8)
    hn, _ = o.collide(h, step=1)
    w, v = o.weights(), o.velocities()
    psi = np.column_stack([np.ones(len(w)), v, (v ** 2).sum(axis=1)])
    for c in range(4):
        before = (w * h[c]) @ psi
        after = (w * hn[c]) @ psi
        assert np.allclose(after, before, rtol=0, atol=1e-12 * (1 + np.abs(before).max()))


def test_rest_state_is_a_fixed_point_on_stretched_grids():
    o = _o(lid_u0=0.0, rv=0.9, rx=0.8, ry=0.85)
    h1, _ = o.step(np.zeros((o.nr, o.nvt)), 0)
    assert np.abs(h1).max() < 1e-11      # rounding, amplified where w_j is tiny


def test_adjoint_on_stretched_grids_matches_central_differences():
    prof = np.array([0.1, 0.12, 0.08])

    def make(pr):
        return oracle.Oracle(nx=3, ny=3, kn=2.0, nv=6, vmax=3.5, nt=300, seed=9, eps=0.1,
                             lid_profile=np.asarray(pr, dtype=np.float64), rv=0.8, rx=0.8, ry=0.7)

    p = workloads.small(nx=3, ny=3, nv=6, vmax=3.5)
    h0 = workloads.warm_state(p, seed=3)
    M = 2

    def J(pr, h):
        o = make(pr)
        tot = 0.0
        for n in range(M):
            tot += o.lid_shear(h, n)[-1] / M
            h, _ = o.step(h, n)
        return tot

    o = make(prof)
    hs = [h0]
    for n in range(M):
        hs.append(o.step(hs[-1], n)[0])
    lam = np.zeros_like(h0)
    g = np.zeros(3)
    for n in range(M - 1, -1, -1):
        lam, g = o.adjoint_step(hs[n], lam, step=n, wD=1.0 / M, grad_lid=g)
    e = 1e-6
    d = np.random.default_rng(1).standard_normal(h0.shape)
    fd = (J(prof, h0 + e * d) - J(prof, h0 - e * d)) / (2 * e)
    assert abs(fd - float(np.sum(lam * d))) <= 1e-7 * abs(fd) + 1e-12
    for i in range(3):
        dp = np.zeros(3)
        dp[i] = e
        fd = (J(prof + dp, h0) - J(prof - dp, h0)) / (2 * e)
        assert abs(fd - g[i]) <= 1e-7 * abs(fd) + 1e-12, (i, fd, g[i])
