"""Shared helpers of the GPU parity tests (no method arithmetic)."""
import numpy as np

import oracle
from paper_1005_5405_gb300 import binding, workloads


def phi0(o):
    """The global Maxwellian Phi0(v_j) = pi^{-3/2} exp(-|v_j|^2) at every node
    (its definition, on uniform and stretched grids alike)."""
    v = o.velocities()
    return np.pi ** -1.5 * np.exp(-np.sum(v * v, axis=1))


def f_metric(o, h_g, h_o):
    """max |f_gpu - f_oracle| / max f with f = Phi0 (1 + eps h) per node."""
    p0 = phi0(o)
    f_o = p0 * (1.0 + o.eps * np.asarray(h_o, dtype=np.float64))
    f_g = p0 * (1.0 + o.eps * np.asarray(h_g, dtype=np.float64))
    return float(np.max(np.abs(f_g - f_o)) / np.max(np.abs(f_o)))


def make(p, h0=None, seed=5):
    """A Cavity and the oracle for problem p, both starting from h0 (the
    warm state rounded to the state dtype, so both sides read identical
    inputs)."""
    cav = binding.Cavity(p)
    o = oracle.Oracle(**p.kwargs())
    if h0 is None:
        h0 = workloads.warm_state(p, seed=seed)
    h0 = np.asarray(h0, dtype=np.float32 if p.dtype == "f32" else np.float64)
    cav.set_state(h0, step=0)
    return cav, o, h0.astype(np.float64)


def state(cav):
    return cav.get_state()[0].cpu().numpy().astype(np.float64)


def invariants(o):
    """(nvt, 5) weighted collision invariants w_j psi_j, psi = 1, v_x, v_y,
    v_z, |v|^2, in FP64 (the oracle's node weights and velocities)."""
    w = o.weights()
    v = o.velocities()
    psi = np.stack([np.ones(len(w)), v[:, 0], v[:, 1], v[:, 2], np.sum(v * v, axis=1)], axis=1)
    return w[:, None] * psi


def conserved(h, wpsi):
    """Per-cell sums sum_j w_j psi_j h_j (nr, 5) and the L1 scale
    sum_j w_j |psi_j| |h_j| (nr, 5), in FP64 on h's device (h: torch tensor
    (nr, nvt), any float dtype; wpsi: numpy (nvt, 5))."""
    import torch
    W = torch.from_numpy(wpsi).to(h.device)
    hd = h.double()
    return hd @ W, hd.abs() @ W.abs()
