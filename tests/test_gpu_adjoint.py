"""GPU adjoint (bz_adjoint_step) against the oracle's FP64 adjoint, and the
autograd rollout against central finite differences and against an oracle
rollout, with the random stream fixed (same seeds on both sides)."""
import numpy as np
import pytest

import oracle
from paper_1005_5405_gb300 import binding, workloads

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    t = pytest.importorskip("torch")
    if not t.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    t.cuda.set_device(0)
    return t


def _problem(dtype, nx=6, ny=5, nv=12, nt=3000, kn=1.0):
    prof = 0.1 + 0.02 * np.sin(np.arange(nx) + 0.3)
    return workloads.small(nx=nx, ny=ny, nv=nv, vmax=4.0, nt=nt, seed=13, dtype=dtype,
                           kn=kn, eps=0.1, lid_profile=prof)


def _tensor(torch, x, dtype):
    return torch.from_numpy(np.ascontiguousarray(x)).to(dtype).cuda()


@pytest.mark.parametrize("dtype,tol,kernel", [("f64", 1e-10, "auto"), ("f32", 2e-4, "auto"),
                                              ("f32", 2e-4, "generic")])
@pytest.mark.parametrize("step,wD", [(0, 0.0), (7, 0.8)])
def test_adjoint_step_matches_oracle(torch, monkeypatch, dtype, tol, kernel, step, wD):
    """FP32 with a multiple-of-4 velocity axis runs the quad kernel unless
    BZ_KERNEL=generic selects the scalar one; FP64 always runs the latter."""
    if kernel == "generic":
        monkeypatch.setenv("BZ_KERNEL", "generic")
    p = _problem(dtype)
    tdt = torch.float64 if dtype == "f64" else torch.float32
    npdt = np.float64 if dtype == "f64" else np.float32
    h = workloads.warm_state(p, seed=21).astype(npdt)
    lam = np.random.default_rng(5).standard_normal((p.nr, p.nvt)).astype(npdt)
    o = oracle.Oracle(**p.kwargs())
    ref, gref = o.adjoint_step(h.astype(np.float64), lam.astype(np.float64), step=step, wD=wD)

    cav = binding.Cavity(p)
    g = torch.zeros(p.nx, dtype=torch.float64, device="cuda")
    out = cav.adjoint_step(step, _tensor(torch, h, tdt), _tensor(torch, lam, tdt), grad_lid=g,
                           wD=wD)
    torch.cuda.synchronize()
    got = out.double().cpu().numpy()
    scale = np.abs(ref).max()
    assert np.abs(got - ref).max() <= tol * scale, np.abs(got - ref).max() / scale
    gg = g.cpu().numpy()
    assert np.abs(gg - gref).max() <= tol * np.abs(gref).max(), (gg, gref)


def test_adjoint_step_in_place_and_accumulates(torch):
    """lam_out may be lam_in; grad_lid is added to, not overwritten."""
    p = _problem("f64")
    h = _tensor(torch, workloads.warm_state(p, seed=3), torch.float64)
    lam = _tensor(torch, np.random.default_rng(1).standard_normal((p.nr, p.nvt)), torch.float64)
    cav = binding.Cavity(p)
    g1 = torch.zeros(p.nx, dtype=torch.float64, device="cuda")
    ref = cav.adjoint_step(3, h, lam.clone(), grad_lid=g1, wD=0.5)
    g2 = torch.full((p.nx,), 2.0, dtype=torch.float64, device="cuda")
    buf = lam.clone()
    cav.adjoint_step(3, h, buf, buf, grad_lid=g2, wD=0.5)
    torch.cuda.synchronize()
    # Shared-memory atomics make the summation order vary from run to run.
    assert torch.allclose(buf, ref, rtol=1e-12, atol=1e-12 * float(ref.abs().max()))
    assert torch.allclose(g2 - 2.0, g1, rtol=1e-14, atol=1e-14)


def test_adjoint_step_rejects_overlap(torch):
    p = _problem("f32")
    cav = binding.Cavity(p)
    h = torch.zeros((p.nr, p.nvt), dtype=torch.float32, device="cuda")
    with pytest.raises(binding.BzError) as e:
        cav.adjoint_step(0, h, h.clone(), h)
    assert e.value.status == binding.BZ_EINVAL


def _J(torch, cav, prof, h0, M, c):
    from paper_1005_5405_gb300 import autodiff
    hM, d = autodiff.rollout(cav, prof, h0, M, every=2)
    return float(d) + float((hM.double() * c).sum())


def test_rollout_gradient_matches_central_differences_f64(torch):
    """J = D_bar + <c, h^M> over 5 steps (checkpoints every 2 steps, so the
    backward pass replays three segments): autograd gradient in the lid face
    speeds and in a random direction of h^0 against central differences."""
    from paper_1005_5405_gb300 import autodiff
    p = _problem("f64", kn=2.0)
    M = 5
    cav = binding.Cavity(p)
    prof = torch.tensor(p.lid_profile, dtype=torch.float64, requires_grad=True)
    h0 = _tensor(torch, workloads.warm_state(p, seed=4), torch.float64).requires_grad_(True)
    c = _tensor(torch, 1e-3 * np.random.default_rng(2).standard_normal((p.nr, p.nvt)),
                torch.float64)
    hM, d = autodiff.rollout(cav, prof, h0, M, every=2)
    J = d + (hM * c).sum()
    J.backward()
    gU, gh = prof.grad.numpy().copy(), h0.grad.detach().clone()

    e = 1e-6
    base = p.lid_profile.copy()
    for i in range(p.nx):
        dp = np.zeros(p.nx)
        dp[i] = e
        jp = _J(torch, cav, torch.tensor(base + dp), h0.detach(), M, c)
        jm = _J(torch, cav, torch.tensor(base - dp), h0.detach(), M, c)
        fd = (jp - jm) / (2 * e)
        assert abs(fd - gU[i]) <= 1e-6 * abs(fd) + 1e-10, (i, fd, gU[i])
    d0 = _tensor(torch, np.random.default_rng(8).standard_normal((p.nr, p.nvt)), torch.float64)
    jp = _J(torch, cav, torch.tensor(base), h0.detach() + e * d0, M, c)
    jm = _J(torch, cav, torch.tensor(base), h0.detach() - e * d0, M, c)
    fd = (jp - jm) / (2 * e)
    ad = float((gh * d0).sum())
    assert abs(fd - ad) <= 1e-6 * abs(fd) + 1e-10, (fd, ad)


def test_rollout_gradient_f32_matches_oracle_rollout(torch):
    """The FP32 path's lid gradient of D_bar over 6 steps against the
    oracle's FP64 adjoint through the same steps (states of the oracle's own
    forward run): agreement to 1e-3 relative."""
    from paper_1005_5405_gb300 import autodiff
    p = _problem("f32", nv=16, kn=2.0)
    M = 6
    h0 = workloads.warm_state(p, seed=6).astype(np.float32)
    o = oracle.Oracle(**p.kwargs())
    hs = [h0.astype(np.float64)]
    for n in range(M):
        hs.append(o.step(hs[-1], n)[0])
    lam = np.zeros_like(hs[0])
    gref = np.zeros(p.nx)
    for n in range(M - 1, -1, -1):
        lam, gref = o.adjoint_step(hs[n], lam, step=n, wD=1.0 / M, grad_lid=gref)

    cav = binding.Cavity(p)
    prof = torch.tensor(p.lid_profile, dtype=torch.float64, requires_grad=True)
    h0t = _tensor(torch, h0, torch.float32).requires_grad_(True)
    _, d = autodiff.rollout(cav, prof, h0t, M, every=4)
    d.backward()
    g = prof.grad.numpy()
    assert np.abs(g - gref).max() <= 1e-3 * np.abs(gref).max(), (g, gref)
    gh = h0t.grad.double().cpu().numpy()
    assert np.abs(gh - lam).max() <= 1e-3 * np.abs(lam).max()
