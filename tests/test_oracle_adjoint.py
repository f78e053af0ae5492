"""Pin of the oracle's FP64 adjoint: central finite differences of
J = (1/M) sum_{n<M} D_n (time-averaged lid shear, Sec. 5.2) with the random
stream fixed, in random directions of the initial state and in every lid-face
speed."""
import numpy as np

import oracle
from paper_1005_5405_gb300 import workloads


def _oracle(profile, eps=0.1):
    return oracle.Oracle(nx=3, ny=3, kn=2.0, nv=6, vmax=3.5, nt=300, seed=9, eps=eps,
                         lid_profile=np.asarray(profile, dtype=np.float64))


def _J(profile, h0, M):
    o = _oracle(profile)
    h, J = h0.copy(), 0.0
    for n in range(M):
        J += o.lid_shear(h, n)[-1] / M
        h, _ = o.step(h, n)
    return J


def _adjoint(profile, h0, M):
    o = _oracle(profile)
    hs = [h0.copy()]
    for n in range(M):
        hs.append(o.step(hs[-1], n)[0])
    lam = np.zeros_like(h0)
    g = np.zeros(o.nx)
    for n in range(M - 1, -1, -1):
        lam, g = o.adjoint_step(hs[n], lam, step=n, wD=1.0 / M, grad_lid=g)
    return lam, g


def test_adjoint_matches_central_differences():
    M = 3
    prof = np.array([0.10, 0.12, 0.08])
    p = workloads.small(nx=3, ny=3, nv=6, vmax=3.5)
    h0 = workloads.warm_state(p, seed=3)
    lam0, gU = _adjoint(prof, h0, M)
    rng = np.random.default_rng(0)
    e = 1e-6
    for _ in range(3):
        d = rng.standard_normal(h0.shape)
        fd = (_J(prof, h0 + e * d, M) - _J(prof, h0 - e * d, M)) / (2 * e)
        ad = float(np.sum(lam0 * d))
        assert abs(fd - ad) <= 1e-7 * abs(fd) + 1e-12, (fd, ad)
    for i in range(3):
        dp = np.zeros(3)
        dp[i] = e
        fd = (_J(prof + dp, h0, M) - _J(prof - dp, h0, M)) / (2 * e)
        assert abs(fd - gU[i]) <= 1e-8 * abs(fd) + 1e-12, (i, fd, gU[i])


def test_adjoint_of_collision_alone_is_linear_in_lambda():
    """The adjoint step is linear in lam (the transposed Jacobian)."""
    prof = np.array([0.1, 0.1, 0.1])
    o = _oracle(prof)
    p = workloads.small(nx=3, ny=3, nv=6, vmax=3.5)
    h0 = workloads.warm_state(p, seed=5)
    rng = np.random.default_rng(1)
    a, b = rng.standard_normal(h0.shape), rng.standard_normal(h0.shape)
    la, ga = o.adjoint_step(h0, a, step=1)
    lb, gb = o.adjoint_step(h0, b, step=1)
    lab, gab = o.adjoint_step(h0, 2 * a - 3 * b, step=1)
    assert np.allclose(lab, 2 * la - 3 * lb, rtol=1e-10, atol=1e-12)
    assert np.allclose(gab, 2 * ga - 3 * gb, rtol=1e-10, atol=1e-14)
