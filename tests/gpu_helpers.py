"""Shared helpers of the GPU parity tests (no method arithmetic)."""
import numpy as np

import oracle
from paper_1005_5405_gb300 import binding, workloads


def f_metric(o, h_g, h_o):
    """max |f_gpu - f_oracle| / max f with f = Phi0 (1 + eps h) per node."""
    phi0 = o.weights() / o.dv ** 3
    f_o = phi0 * (1.0 + o.eps * np.asarray(h_o, dtype=np.float64))
    f_g = phi0 * (1.0 + o.eps * np.asarray(h_g, dtype=np.float64))
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
