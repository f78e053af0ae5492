"""Seeded synthetic workloads: problem statements and initial states.

This module holds no arithmetic of the method.  It names the cavity problems
the library is exercised on (sizes, Knudsen numbers, lid motion, sample counts,
seeds) and builds seeded initial deviational states on the velocity grid.
Both the CUDA path and the CPU oracle consume what it produces; neither
imports the other.

Problems (driven cavity of Sec. 5.1: square box, lid moving along +x at
y = L, diffuse walls at T0, initial uniform Maxwellian n0 = 1, h0 = 0):

  cavity16_v12   16x16 cells, 12^3 velocities on [-4,4]^3, Kn 1, lid 0.1,
                 1000 samples/step, seed 1, FP64 state
  cavity64_v24   64x64 cells, 24^3 on [-4.5,4.5]^3, Kn 0.1, lid 0.1,
                 10^4 samples/step, seed 2, FP32 state
  cavity256_v32  256x256 cells, 32^3 on [-5,5]^3, Kn 0.05, lid
                 0.05 sin(2 pi t / 50), 2x10^4 samples/step, seed 3, FP32
  adjoint128_v20 128x128 cells, 20^3 on [-4.5,4.5]^3, Kn 0.2, per-face lid
                 0.1 + N(0, 0.01^2), 5000 samples/step, seed 4, FP32
  percell64_v24  cavity64_v24 with its own 10^4 samples in every cell
  paper_cavity   the paper's own setups (stretched grids, lid 0.01), delta
                 0.1, 1, 10
"""
from __future__ import annotations

from dataclasses import dataclass, field, asdict
from typing import Optional

import numpy as np


@dataclass
class Problem:
    name: str
    nx: int
    ny: int
    kn: float
    nv: int
    vmax: float
    nt: int
    seed: int
    dtype: str = "f32"          # "f32" or "f64" state
    lid_u0: float = 0.1
    lid_amp: float = 0.0
    lid_period: float = 0.0
    lid_profile: Optional[np.ndarray] = field(default=None, repr=False)
    eps: float = 0.0            # 0 => max |U|
    cfl: float = 0.5
    instance: int = 0
    per_cell: bool = False
    steps: int = 1
    rv: float = 0.0             # stretched velocity cells (0 or 1: uniform)
    rx: float = 0.0             # stretched spatial cells toward the side walls
    ry: float = 0.0             # ... and toward the lid

    @property
    def nr(self) -> int:
        return self.nx * self.ny

    @property
    def nvt(self) -> int:
        return self.nv ** 3

    @property
    def nodes(self) -> int:
        return self.nr * self.nvt

    def kwargs(self) -> dict:
        """Keyword arguments shared by the oracle and the library binding."""
        d = asdict(self)
        for k in ("name", "dtype", "steps"):
            d.pop(k)
        return d


def cavity16_v12() -> Problem:
    return Problem("cavity16_v12", 16, 16, 1.0, 12, 4.0, 1000, 1, dtype="f64", steps=100)


def cavity64_v24() -> Problem:
    return Problem("cavity64_v24", 64, 64, 0.1, 24, 4.5, 10_000, 2, steps=2000)


def cavity256_v32() -> Problem:
    return Problem("cavity256_v32", 256, 256, 0.05, 32, 5.0, 20_000, 3, lid_u0=0.0,
                   lid_amp=0.05, lid_period=50.0, steps=1000)


def cavity64_v32() -> Problem:
    """64x64 cells with the cell size, velocity grid and samples of
    cavity256_v32 (state 0.54 GB, above L2): the profiling case."""
    return Problem("cavity64_v32", 64, 64, 0.2, 32, 5.0, 20_000, 3, lid_u0=0.0,
                   lid_amp=0.05, lid_period=50.0, steps=1000)


def adjoint128_v20(seed: int = 4) -> Problem:
    rng = np.random.default_rng(seed)
    prof = 0.1 + 0.01 * rng.standard_normal(128)
    return Problem("adjoint128_v20", 128, 128, 0.2, 20, 4.5, 5000, seed, lid_profile=prof,
                   steps=500)


def percell64_v24() -> Problem:
    """cavity64_v24 with an independent sample set in every cell."""
    return Problem("percell64_v24", 64, 64, 0.1, 24, 4.5, 10_000, 2, per_cell=True, steps=2000)


def paper_cavity(delta: float) -> Problem:
    """The paper's driven-cavity setups (Sec. 5.1): lid speed 0.01, velocity
    box [-3, 3]^3 with stretched cells, stretched spatial cells refined toward
    the lid corners.  delta = 0.1 and 1: 160x160 cells, 20^3 nodes (rv
    0.945), rx 0.996, ry 0.998, 1024 (delta 0.1) or 6144 (delta 1) samples
    per step; delta = 10: 192x192 cells, 18^3 nodes (rv 0.970), rx 0.990,
    ry 0.995, 8192 samples.  FP32."""
    if delta >= 10:
        return Problem("paper_delta10", 192, 192, 1.0 / delta, 18, 3.0, 8192, 6, lid_u0=0.01,
                       rv=0.970, rx=0.990, ry=0.995, steps=1000)
    nt = 1024 if delta <= 0.1 else 6144
    return Problem(f"paper_delta{delta:g}", 160, 160, 1.0 / delta, 20, 3.0, nt, 5, lid_u0=0.01,
                   rv=0.945, rx=0.996, ry=0.998, steps=1000)


def batch64(n: int = 64, seed0: int = 100, nt: int = 5000) -> list:
    """Batched workload: n independent cavities, instance k drawn with
    numpy.random.default_rng(seed0 + k): square grid side from
    {32, 48, 64, 96, 128}, velocity grid from {16^3, 20^3, 24^3} (box 4.0 for
    16^3, 4.5 otherwise), Kn log-uniform in [0.05, 5], lid speed uniform in
    [0.01, 0.2]; FP32, nt samples per step, Philox seed seed0 + k, instance k."""
    out = []
    for k in range(n):
        rng = np.random.default_rng(seed0 + k)
        side = int(rng.choice([32, 48, 64, 96, 128]))
        nv = int(rng.choice([16, 20, 24]))
        kn = float(np.exp(rng.uniform(np.log(0.05), np.log(5.0))))
        u = float(rng.uniform(0.01, 0.2))
        out.append(Problem(f"batch{seed0 + k}", side, side, kn, nv, 4.0 if nv == 16 else 4.5, nt,
                           seed0 + k, lid_u0=u, instance=k, steps=500))
    return out


def small(name="small", nx=8, ny=8, nv=12, vmax=4.0, nt=1000, seed=1, **kw) -> Problem:
    """A problem small enough for the oracle to finish in well under a second."""
    return Problem(name, nx, ny, kw.pop("kn", 1.0), nv, vmax, nt, seed, **kw)


def axis_nodes(nv: int, vmax: float) -> np.ndarray:
    """Cell-centred node coordinates of one velocity axis."""
    dv = 2.0 * vmax / nv
    return -vmax + (np.arange(nv) + 0.5) * dv


def warm_state_device(p: Problem, seed: int = 7, noise: float = 0.01, torch=None):
    """The same kind of state as `warm_state`, built on the current CUDA
    device with PyTorch (for grids too large to build on the host).  The
    per-cell coefficients come from numpy's seeded generator; the per-node
    noise from a seeded torch generator.  Returns a (nr, nv^3) tensor in the
    problem's state dtype."""
    if torch is None:
        import torch
    dt = torch.float64 if p.dtype == "f64" else torch.float32
    rng = np.random.default_rng(seed)
    coef = torch.from_numpy(0.3 * rng.standard_normal((p.nr, 6))).to(dt).cuda()
    a = torch.from_numpy(axis_nodes(p.nv, p.vmax)).to(dt).cuda()
    vx, vy, vz = torch.meshgrid(a, a, a, indexing="ij")
    vx, vy, vz = vx.reshape(-1), vy.reshape(-1), vz.reshape(-1)
    basis = torch.stack([torch.ones_like(vx), vx, vy, vz, vx * vx + vy * vy + vz * vz - 1.5,
                         vx * vy])
    h = coef @ basis
    gen = torch.Generator(device="cuda").manual_seed(seed)
    h += noise * torch.randn(h.shape, generator=gen, device="cuda", dtype=dt)
    return h


def warm_state(p: Problem, seed: int = 7, noise: float = 0.01) -> np.ndarray:
    """Seeded smooth-plus-noise deviational state h0[cell, node] (float64).

    Per cell: a + b.v + c (|v|^2 - 3/2) + d v_x v_y with coefficients drawn
    from N(0, 0.3^2), plus `noise` N(0,1) per node; used to make the collision
    integral non-zero from the first step."""
    rng = np.random.default_rng(seed)
    a = axis_nodes(p.nv, p.vmax)
    vx, vy, vz = np.meshgrid(a, a, a, indexing="ij")
    vx, vy, vz = vx.ravel(), vy.ravel(), vz.ravel()
    v2 = vx * vx + vy * vy + vz * vz
    coef = 0.3 * rng.standard_normal((p.nr, 6))
    basis = np.stack([np.ones_like(vx), vx, vy, vz, v2 - 1.5, vx * vy], axis=0)
    h = coef @ basis
    h += noise * rng.standard_normal(h.shape)
    return h
