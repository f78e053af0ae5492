"""Host logic of the autograd rollout (checkpointing, segment replay, the
step numbers and states handed to each adjoint step, the scaling of the lid
shear weight), run on the CPU against a toy linear "cavity" whose adjoint is
written out by hand and checked against torch's own autograd of the same
toy."""
import types

import numpy as np
import pytest
import torch

from paper_1005_5405_gb300 import autodiff

NX, NY, NVT = 3, 2, 5
ALPHA, BETA, KAPPA = 0.9, 0.07, 0.3
W = torch.linspace(0.5, 1.5, NVT, dtype=torch.float64)


def _gamma(n):
    return 0.01 * (n + 1)


def _toy_step(h, U, n):
    """h^{n+1} = alpha h + beta roll(h) + gamma_n U[ix(c)]."""
    col = torch.arange(NX * NY) % NX
    return ALPHA * h + BETA * torch.roll(h, 1, dims=1) + _gamma(n) * U[col][:, None]


def _toy_shear(h, U):
    lid = h[(NY - 1) * NX:]
    s = (lid * W).sum(dim=1) + KAPPA * U
    return torch.cat([s, s.mean()[None]])


class FakeCavity:
    """Implements the Cavity methods the rollout uses, on the toy model."""

    def __init__(self):
        self.p = types.SimpleNamespace(nx=NX, ny=NY, nr=NX * NY, nvt=NVT, lid_amp=0.0,
                                       lid_period=0.0)
        self.torch_dtype = torch.float64
        self.U = torch.zeros(NX, dtype=torch.float64)
        self.h = torch.zeros(NX * NY, NVT, dtype=torch.float64)
        self.n = 0
        self.seen = {}          # step -> state seen in the forward pass
        self.adj_calls = []

    def set_lid(self, u0, amp, period, profile=None):
        self.U = torch.as_tensor(profile, dtype=torch.float64).clone()

    def set_state(self, h, step):
        self.h, self.n = h.clone(), step

    def get_state(self):
        return self.h.clone(), self.n

    def lid_shear(self, out):
        out.copy_(_toy_shear(self.h, self.U))

    def step(self, k):
        for _ in range(k):
            self.seen.setdefault(self.n, self.h.clone())
            self.h = _toy_step(self.h, self.U, self.n)
            self.n += 1

    def adjoint_step(self, step, h_n, lam_in, lam_out, grad_lid, wD):
        assert torch.equal(h_n, self.seen[step]), step
        self.adj_calls.append(step)
        col = torch.arange(NX * NY) % NX
        gl = _gamma(step) * torch.zeros(NX, dtype=torch.float64).index_add(
            0, col, lam_in.sum(dim=1))
        grad_lid += gl + wD * KAPPA / NX
        out = ALPHA * lam_in + BETA * torch.roll(lam_in, -1, dims=1)
        out[(NY - 1) * NX:] += wD * W / NX
        lam_out.copy_(out)
        return lam_out


def _reference(U, h0, M, step0):
    h, ds = h0, []
    for n in range(M):
        ds.append(_toy_shear(h, U)[-1])
        h = _toy_step(h, U, step0 + n)
    return h, torch.stack(ds).mean()


@pytest.mark.parametrize("M,every,step0", [(1, 50, 0), (7, 3, 4), (6, 2, 0), (5, 5, 1)])
def test_rollout_matches_autograd_of_the_same_steps(M, every, step0):
    rng = np.random.default_rng(M * 10 + every)
    U0 = torch.tensor(rng.uniform(0.05, 0.15, NX))
    h00 = torch.tensor(rng.standard_normal((NX * NY, NVT)))
    c = torch.tensor(rng.standard_normal((NX * NY, NVT)))

    U, h0 = U0.clone().requires_grad_(True), h00.clone().requires_grad_(True)
    hM, d = _reference(U, h0, M, step0)
    (3.0 * d + (hM * c).sum()).backward()

    cav = FakeCavity()
    U2, h02 = U0.clone().requires_grad_(True), h00.clone().requires_grad_(True)
    hM2, d2 = autodiff.rollout(cav, U2, h02, M, step0=step0, every=every)
    assert torch.allclose(hM2, hM.detach()) and abs(float(d2) - float(d)) < 1e-12
    (3.0 * d2 + (hM2 * c).sum()).backward()
    assert torch.allclose(U2.grad, U.grad, rtol=1e-12, atol=1e-14)
    assert torch.allclose(h02.grad, h0.grad, rtol=1e-12, atol=1e-14)
    # Every step's adjoint ran exactly once, last step first within a segment.
    assert sorted(cav.adj_calls) == list(range(step0, step0 + M))
    assert cav.adj_calls[0] == step0 + M - 1


def test_rollout_only_shear_objective():
    U = torch.tensor([0.1, 0.2, 0.3], dtype=torch.float64, requires_grad=True)
    h0 = torch.zeros(NX * NY, NVT, dtype=torch.float64, requires_grad=True)
    _, d = autodiff.rollout(FakeCavity(), U, h0, 4, every=2)
    d.backward()
    U2 = U.detach().clone().requires_grad_(True)
    h02 = h0.detach().clone().requires_grad_(True)
    _reference(U2, h02, 4, 0)[1].backward()
    assert torch.allclose(U.grad, U2.grad) and torch.allclose(h0.grad, h02.grad)


def test_rollout_rejects_bad_arguments():
    with pytest.raises(ValueError):
        autodiff.rollout(FakeCavity(), torch.zeros(NX + 1, dtype=torch.float64),
                         torch.zeros(NX * NY, NVT, dtype=torch.float64), 3)
    with pytest.raises(ValueError):
        autodiff.rollout(FakeCavity(), torch.zeros(NX, dtype=torch.float64),
                         torch.zeros(NX * NY, NVT, dtype=torch.float64), 0)
