"""Conservation on the GPU (Sec. 3: the correction of Eqs. rinorm_a and
correzione makes every collision step conserve the moments 1, v, |v|^2 of
h~ exactly; free streaming with diffuse walls conserves the total mass).

The sums are taken here, in FP64, over the states the GPU stored.  Each is
compared with its L1 scale sum_j w_j |psi_j| |h_j| (h is a deviation, so its
moments themselves may be near zero); the physical reading (relative to the
moments of f = Phi0 (1 + eps h)) is printed beside it.  The bar is 1e-6
relative for FP32 states.
"""
import numpy as np
import pytest

from paper_1005_5405_gb300 import binding, workloads
from tests.gpu_helpers import conserved, invariants, make

pytestmark = pytest.mark.gpu

NAMES = ["mass", "x-momentum", "y-momentum", "z-momentum", "energy"]


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    torch.cuda.set_device(0)
    yield


def _v32(nxy=6, **kw):
    """32^3 velocities on [-5, 5]^3 with 2x10^4 samples and the cell size of
    the 256x256 cavity: the benchmark's velocity grid and sample set."""
    return workloads.small(nx=nxy, ny=nxy, nv=32, vmax=5.0, nt=20000, seed=3,
                           kn=0.05 * 256 / nxy, **kw)


@pytest.fixture(params=["auto", "ordered", "early_tail", "tma", "cell4", "generic"])
def kernel(request, monkeypatch):
    """The active-node kernel (the benchmark's), with the joint term order
    forced on, with the increment sums started early by the collision warps
    (below 32^3 velocities: the 32^3 kernel always sums after a barrier);
    with the streaming sources brought in by bulk copies (TMA); the
    4-node-vector kernel; the generic kernel."""
    for k in ("BZ_KERNEL", "BZ_LAZY_ORDER", "BZ_LAZY_NOORDER", "BZ_LAZY_ORDER_CHUNK",
              "BZ_SOLVE_FALLBACK", "BZ_LAZY_EARLY_TAIL", "BZ_LAZY_TMA"):
        monkeypatch.delenv(k, raising=False)
    if request.param == "ordered":
        monkeypatch.setenv("BZ_LAZY_ORDER", "1")
    elif request.param == "early_tail":
        monkeypatch.setenv("BZ_LAZY_EARLY_TAIL", "1")
    elif request.param == "tma":
        monkeypatch.setenv("BZ_LAZY_TMA", "1")
    elif request.param in ("cell4", "generic"):
        monkeypatch.setenv("BZ_KERNEL", request.param)
    return request.param


def _check(before, after, scale, tol, what):
    d = (after - before).abs()
    rel = (d / scale.clamp_min(1e-300)).max(dim=0).values.cpu().numpy()
    for k, name in enumerate(NAMES):
        print(f"{what}: {name} changed by {rel[k]:.2e} of its L1 scale (worst cell)")
    assert (rel <= tol).all(), (what, rel)


@pytest.mark.parametrize("nv", [32, 24, 16])
def test_collision_step_conserves(kernel, nv):
    """One relaxation (sampling, collision, correction; no streaming) per
    cell: sum_j w_j psi_j h^{n+1}_j = sum_j w_j psi_j h_j for psi = 1, v,
    |v|^2, to 1e-6 of the L1 scale, in every cell, for three steps."""
    import torch
    if nv == 32:
        p = _v32(eps=0.05)
    else:
        p = workloads.small(nx=6, ny=5, nv=nv, vmax=4.5, nt=10000, seed=4, kn=0.8, eps=0.1)
    cav, o, h0 = make(p, seed=9)
    if kernel in ("auto", "ordered", "early_tail", "tma"):
        assert cav.get_info().kernel_variant == 2
    wpsi = invariants(o)
    h = cav.get_state()[0].clone()
    for n in range(3):
        m0, s0 = conserved(h, wpsi)
        cav.step_ex(1, binding.BZ_DO_COLLIDE)
        h = cav.get_state()[0].clone()
        m1, _ = conserved(h, wpsi)
        _check(m0, m1, s0, 1e-6, f"{kernel} {nv}^3 step {n}")
    assert cav.stats()[3] == 0          # no solve needed its fallback


def test_fused_step_conserves_the_moments_of_h_tilde(kernel):
    """A full step: the moments of h^{n+1} equal those of the post-streaming
    h~ (Eq. rinorm_a), h~ taken from a BZ_DO_STREAM step of the same state on
    a second handle (a separate streaming kernel: its rounding differs by an
    ulp per node)."""
    p = _v32(nxy=8, eps=0.05, lid_u0=0.05)
    a, o, h0 = make(p, seed=10)
    b, _, _ = make(p, seed=10)
    wpsi = invariants(o)
    for n in range(2):
        b.set_state(a.get_state()[0].clone(), step=n)
        b.step_ex(1, binding.BZ_DO_STREAM)
        mt, st = conserved(b.get_state()[0], wpsi)
        a.step(1)
        m1, _ = conserved(a.get_state()[0], wpsi)
        _check(mt, m1, st, 1e-6, f"{kernel} full step {n}")


def test_homogeneous_relaxation_keeps_rho_u_theta():
    """Spatially homogeneous relaxation on the active-node kernel (50
    relaxation steps with no streaming) of an anisotropic, drifting state
    with T_x != T_y: density, mean velocity and temperature of f stay
    constant to 1e-6 relative, while the anisotropy relaxes."""
    import torch
    import oracle
    p = _v32(nxy=4, eps=0.1)
    v = oracle.Oracle(**p.kwargs()).velocities()
    # a + b v_x + c (v_x^2 - v_y^2) + d (|v|^2 - 3/2), one set per cell, with
    # |c| in [0.2, 0.4] so that every cell has an anisotropy to relax
    rng = np.random.default_rng(12)
    coef = rng.uniform(-0.3, 0.3, size=(p.nr, 4))
    coef[:, 2] = rng.choice([-1.0, 1.0], p.nr) * rng.uniform(0.2, 0.4, p.nr)
    basis = np.stack([np.ones(len(v)), v[:, 0], v[:, 0] ** 2 - v[:, 1] ** 2,
                      np.sum(v * v, axis=1) - 1.5])
    h0 = coef @ basis
    cav, o, h0 = make(p, h0=h0)
    assert cav.get_info().kernel_variant == 2
    wpsi = invariants(o)
    w = torch.from_numpy(o.weights()).cuda()
    vt = torch.from_numpy(v).cuda()

    def fields(h):
        """rho_f, u_f, T_f of f = Phi0 (1 + eps h) per cell (V0 units:
        T_f = (2/3) <|v - u|^2>)."""
        f = w * (1.0 + o.eps * h.double())
        n = f.sum(1)
        u = (f @ vt) / n[:, None]
        e = (f * (vt * vt).sum(1)).sum(1) / n
        T = (2.0 / 3.0) * (e - (u * u).sum(1))
        return n, u, T

    def aniso(h):
        return (w * h.double() * (vt[:, 0] ** 2 - vt[:, 1] ** 2)).sum(1)

    h = cav.get_state()[0].clone()
    n0, u0, T0 = fields(h)
    a0 = aniso(h)
    for _ in range(5):
        cav.step_ex(10, binding.BZ_DO_COLLIDE)
    h = cav.get_state()[0].clone()
    n1, u1, T1 = fields(h)
    dn = ((n1 - n0).abs() / n0).max().item()
    du = (u1 - u0).abs().max().item()
    dT = ((T1 - T0).abs() / T0).max().item()
    print(f"50 relaxation steps: |d rho|/rho {dn:.2e}, |d u| {du:.2e}, |d T|/T {dT:.2e}")
    assert dn <= 1e-6 and du <= 1e-6 and dT <= 1e-6
    # the anisotropy decays (the collisions act)
    assert (aniso(h).abs() < 0.9 * a0.abs()).all()


def test_closed_cavity_total_mass_1000_steps(monkeypatch):
    """The driven cavity is closed (diffuse walls have zero net mass flux,
    Eq. bcMax): over 1000 full steps on the benchmark's path (32^3
    velocities, 2x10^4 samples, the term order forced on) the total mass
    sum_cells sum_j w_j h_j drifts by at most 1e-6 of its L1 scale (and far
    less than that of the mass of f)."""
    monkeypatch.setenv("BZ_LAZY_ORDER", "1")
    p = _v32(nxy=16, lid_u0=0.0, lid_amp=0.05, lid_period=50.0)
    cav, o, h0 = make(p, seed=13)
    assert cav.get_info().kernel_variant == 2
    wpsi = invariants(o)[:, :1]
    m0, s0 = conserved(cav.get_state()[0], wpsi)
    M0, S0 = m0.sum().item(), s0.sum().item()
    fmass = p.nr * float(o.weights().sum()) / o.eps      # sum w (1/eps + h) at rest
    worst = 0.0
    for k in range(10):
        cav.step(100)
        m, _ = conserved(cav.get_state()[0], wpsi)
        d = abs(m.sum().item() - M0)
        worst = max(worst, d / S0)
        print(f"after {100 * (k + 1)} steps: total mass drift {d / S0:.2e} of the L1 scale, "
              f"{d / (fmass + M0):.2e} of the mass of f")
    assert worst <= 1e-6
    assert cav.stats()[5] == 0


@pytest.mark.parametrize("kernel_env", [None, "cell4", "generic"])
def test_solve_fallback_is_counted(monkeypatch, kernel_env):
    """BZ_SOLVE_FALLBACK=1 sends every correction solve to its pivoted
    fallback: bz_stats()[3] counts one per cell and step on every kernel, and
    the result still matches the oracle."""
    from tests.gpu_helpers import f_metric, state
    monkeypatch.setenv("BZ_SOLVE_FALLBACK", "1")
    if kernel_env:
        monkeypatch.setenv("BZ_KERNEL", kernel_env)
    p = workloads.small(nx=5, ny=4, nv=16, vmax=4.0, nt=3000, seed=8, eps=0.1)
    cav, o, h0 = make(p)
    cav.step(2)
    assert cav.stats()[3] == 2 * p.nr
    h1, _ = o.step(h0, 0)
    h2, _ = o.step(h1, 1)
    assert f_metric(o, state(cav), h2) < 2e-5
