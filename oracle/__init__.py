"""FP64 CPU oracle for the semi-regular Boltzmann step (test infrastructure).

This package is test infrastructure: only the test-suite, the smoke check and
the benchmark's CPU-baseline leg may import it.  The product library neither
imports nor links it, and it shares no code with the CUDA path.  The C source
(`bz_oracle.c`) follows the paper (Frezzotti, Ghiroldi & Gibelli, "Solving the
Boltzmann equation on GPUs") equation by equation in double precision; this
module only builds it and marshals numpy arrays through ctypes.

Pins and their status (every function is checked against something other than
itself by the `-m "not gpu"` tests):
  philox      statistical checks on CPU; word-for-word cross-check against
              cuRAND's Philox4x32-10 on the GPU (the Random123 known-answer
              vectors are not available offline)
  sample      exact collision invariants of the kinematics (P2), the
              distribution moments of v, v1, k
  stream      exact one-cell shift at Courant number 1, zero-flux walls,
              mass conservation, h = 0 fixed point
  collide     per-collision mass, exact conservation after the correction,
              h = 0 fixed point, eps-scaling identity, H-theorem, the hard-
              sphere stress relaxation rate, the loss term of Eq. coll8Dim
              against the closed-form hard-sphere collision frequency, the
              drifting Maxwellian as a statistical fixed point
  moments     analytic Maxwellian perturbations
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None

# Hard-sphere collision constant K = n0 sigma^2 lambda0 with lambda0 built on
# the hard-sphere viscosity mu0 = 1.016034 (5/16) sigma^-2 sqrt(m k T0 / pi)
# (Chapman & Cowling; Sec. 5.1 of the paper): K = (5 * 1.016034 / 16) sqrt(2/pi).
K_HARD_SPHERE = 5.0 * 1.016034 / 16.0 * np.sqrt(2.0 / np.pi)


def build(force: bool = False) -> str:
    """Compile the oracle into oracle/_build/liboracle.so (gcc, OpenMP)."""
    src = os.path.join(_HERE, "bz_oracle.c")
    hdr = os.path.join(_HERE, "bz_oracle.h")
    if (not force and os.path.exists(_SO)
            and os.path.getmtime(_SO) >= max(os.path.getmtime(src), os.path.getmtime(hdr))):
        return _SO
    os.makedirs(_BUILD, exist_ok=True)
    tmp = _SO + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-ffp-contract=off", "-fopenmp", "-fPIC", "-shared",
           "-std=c11", "-o", tmp, src, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _SO)
    return _SO


class Problem(C.Structure):
    _fields_ = [
        ("nx", C.c_int32), ("ny", C.c_int32), ("kn", C.c_double),
        ("nv", C.c_int32), ("vmax", C.c_double), ("eps", C.c_double),
        ("cfl", C.c_double), ("kcoll", C.c_double), ("nt", C.c_int64),
        ("seed", C.c_uint32), ("instance", C.c_uint32), ("per_cell", C.c_int32),
        ("lid_u0", C.c_double), ("lid_amp", C.c_double), ("lid_period", C.c_double),
        ("lid_profile", C.POINTER(C.c_double)),
        ("rv", C.c_double), ("rx", C.c_double), ("ry", C.c_double),
    ]


class Sample(C.Structure):
    _fields_ = [
        ("v", C.c_double * 3), ("v1", C.c_double * 3), ("k", C.c_double * 3),
        ("vs", C.c_double * 3), ("v1s", C.c_double * 3),
        ("s", C.c_double), ("W", C.c_double),
        ("idx", C.c_int32 * 4), ("near_face", C.c_int32),
    ]


SAMPLE_DTYPE = np.dtype([
    ("v", "<f8", 3), ("v1", "<f8", 3), ("k", "<f8", 3), ("vs", "<f8", 3),
    ("v1s", "<f8", 3), ("s", "<f8"), ("W", "<f8"), ("idx", "<i4", 4),
    ("near_face", "<i4"),
], align=True)
assert SAMPLE_DTYPE.itemsize == C.sizeof(Sample)

_P = C.POINTER(Problem)
_D = C.POINTER(C.c_double)
_U32 = C.POINTER(C.c_uint32)


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = C.CDLL(_SO)
            sig = {
                "bzo_dv": (C.c_double, [_P]), "bzo_dx": (C.c_double, [_P]),
                "bzo_dy": (C.c_double, [_P]), "bzo_dt": (C.c_double, [_P]),
                "bzo_node_v": (C.c_double, [_P, C.c_int32]),
                "bzo_weight": (C.c_double, [_P, C.c_int32]),
                "bzo_lid_speed": (C.c_double, [_P, C.c_int32, C.c_int64]),
                "bzo_philox4x32_10": (None, [_U32, _U32, _U32]),
                "bzo_node_of": (C.c_int32, [_P, _D, C.POINTER(C.c_int32)]),
                "bzo_sample_all": (None, [_P, C.c_int64, C.c_uint32, C.c_void_p]),
                "bzo_num_faces": (C.c_int32, [_P]),
                "bzo_wall_density": (None, [_P, C.c_int64, _D, _D]),
                "bzo_ghost": (C.c_double, [_P, C.c_int64, C.c_int32, C.c_double, C.c_int32]),
                "bzo_stream": (None, [_P, C.c_int64, _D, _D]),
                "bzo_collide": (None, [_P, C.c_int64, C.c_void_p, _D, _D, _D, _D]),
                "bzo_step": (None, [_P, C.c_int64, _D, _D, _D]),
                "bzo_moments": (None, [_P, _D, _D]),
                "bzo_step_cell": (None, [_P, C.c_int64, C.c_int32, _D, _D, _D, _D, _D, _D, _D]),
                "bzo_lid_shear": (None, [_P, C.c_int64, _D, _D]),
                "bzo_mc_dNdt": (None, [_P, C.c_int64, _D, _D, _D]),
                "bzo_num_threads": (C.c_int32, []),
                "bzo_adjoint_step": (None, [_P, C.c_int64, _D, _D, _D, _D, C.c_double]),
                "bzo_axis_edge": (C.c_double, [_P, C.c_int32]),
                "bzo_axis_width": (C.c_double, [_P, C.c_int32]),
                "bzo_cell_dx": (C.c_double, [_P, C.c_int32]),
                "bzo_cell_dy": (C.c_double, [_P, C.c_int32]),
            }
            for name, (res, args) in sig.items():
                f = getattr(L, name)
                f.restype = res
                f.argtypes = args
            _lib = L
    return _lib


def _dptr(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(_D)


class Oracle:
    """A problem statement bound to the FP64 oracle.

    Parameters mirror the paper's statement of the problem: spatial grid
    (nx, ny) on a square cavity of side L = 1/kn, a cubic velocity grid of
    nv^3 nodes on [-vmax, vmax]^3, the deviation parameter eps, the maximum
    Courant number, the number of Monte Carlo samples per step and the
    Philox key (seed, instance)."""

    def __init__(self, nx, ny, kn, nv, vmax, nt, seed, eps=None, cfl=0.5,
                 kcoll=K_HARD_SPHERE, instance=0, per_cell=False, lid_u0=0.1,
                 lid_amp=0.0, lid_period=0.0, lid_profile=None, rv=0.0, rx=0.0, ry=0.0):
        if eps is None or eps == 0.0:
            if lid_profile is not None:
                eps = float(np.max(np.abs(lid_profile))) + abs(lid_amp)
            else:
                eps = abs(lid_u0) + abs(lid_amp)
            if eps == 0.0:
                eps = 1.0
        self._profile = None
        if lid_profile is not None:
            self._profile = np.ascontiguousarray(lid_profile, dtype=np.float64)
            assert self._profile.shape == (nx,)
        self.p = Problem(nx, ny, kn, nv, vmax, eps, cfl, kcoll, nt, seed, instance,
                         1 if per_cell else 0, lid_u0, lid_amp, lid_period,
                         _dptr(self._profile) if self._profile is not None else None,
                         rv, rx, ry)
        self.L = lib()
        self.nx, self.ny, self.nv = nx, ny, nv
        self.nr = nx * ny
        self.nvt = nv ** 3
        self.eps = eps

    # derived quantities ------------------------------------------------
    @property
    def dt(self):
        return self.L.bzo_dt(C.byref(self.p))

    @property
    def dv(self):
        return self.L.bzo_dv(C.byref(self.p))

    @property
    def dx(self):
        return self.L.bzo_dx(C.byref(self.p))

    def axis_edges(self):
        """Per-axis velocity cell edges (nv + 1,)."""
        return np.array([self.L.bzo_axis_edge(C.byref(self.p), k) for k in range(self.nv + 1)])

    def axis_widths(self):
        return np.array([self.L.bzo_axis_width(C.byref(self.p), j) for j in range(self.nv)])

    def cell_widths(self):
        """(dx per column (nx,), dy per row (ny,))."""
        return (np.array([self.L.bzo_cell_dx(C.byref(self.p), i) for i in range(self.nx)]),
                np.array([self.L.bzo_cell_dy(C.byref(self.p), i) for i in range(self.ny)]))

    def node_v(self):
        """Per-axis node velocities (nv,)."""
        return np.array([self.L.bzo_node_v(C.byref(self.p), j) for j in range(self.nv)])

    def weights(self):
        """dV Phi0(v_j) for all nodes (nv^3,)."""
        return np.array([self.L.bzo_weight(C.byref(self.p), j) for j in range(self.nvt)])

    def velocities(self):
        """(nv^3, 3) node velocities in the library's node order."""
        a = self.node_v()
        jx, jy, jz = np.meshgrid(np.arange(self.nv), np.arange(self.nv),
                                 np.arange(self.nv), indexing="ij")
        return np.stack([a[jx.ravel()], a[jy.ravel()], a[jz.ravel()]], axis=1)

    def lid_speed(self, ix, step):
        return self.L.bzo_lid_speed(C.byref(self.p), ix, step)

    # method --------------------------------------------------------------
    def samples(self, step, cellword=0xFFFFFFFF):
        out = np.zeros(self.p.nt, dtype=SAMPLE_DTYPE)
        self.L.bzo_sample_all(C.byref(self.p), step, cellword, out.ctypes.data)
        return out

    def node_of(self, v):
        v = np.ascontiguousarray(v, dtype=np.float64)
        nf = C.c_int32(0)
        j = self.L.bzo_node_of(C.byref(self.p), _dptr(v), C.byref(nf))
        return j, nf.value

    def wall_density(self, h, step=0):
        h = self._state(h)
        nw = np.zeros(self.L.bzo_num_faces(C.byref(self.p)))
        self.L.bzo_wall_density(C.byref(self.p), step, _dptr(h), _dptr(nw))
        return nw

    def ghost(self, step, face, nw, j):
        return self.L.bzo_ghost(C.byref(self.p), step, face, nw, j)

    def stream(self, h, step=0):
        h = self._state(h)
        out = np.empty_like(h)
        self.L.bzo_stream(C.byref(self.p), step, _dptr(h), _dptr(out))
        return out

    def collide(self, ht, step=0, samples=None, with_stage=False):
        ht = self._state(ht)
        out = np.empty_like(ht)
        mom = np.empty((self.nr, 11))
        stage = np.empty_like(ht) if with_stage else None
        sp = None
        if samples is not None:
            samples = np.ascontiguousarray(samples, dtype=SAMPLE_DTYPE)
            assert samples.shape == (self.p.nt,)
            sp = samples.ctypes.data
        self.L.bzo_collide(C.byref(self.p), step, sp, _dptr(ht), _dptr(out), _dptr(mom),
                           _dptr(stage) if stage is not None else None)
        if with_stage:
            return out, mom, stage
        return out, mom

    def step(self, h, step=0):
        h = self._state(h)
        out = np.empty_like(h)
        mom = np.empty((self.nr, 11))
        self.L.bzo_step(C.byref(self.p), step, _dptr(h), _dptr(out), _dptr(mom))
        return out, mom

    def step_cell(self, c, own, left=None, right=None, below=None, above=None, step=0):
        """One step of cell c from its own and neighbouring slabs (None at walls)."""
        def arr(a):
            if a is None:
                return None
            a = np.ascontiguousarray(a, dtype=np.float64)
            assert a.shape == (self.nvt,)
            return a
        sl = [arr(x) for x in (own, left, right, below, above)]
        out = np.empty(self.nvt)
        mom = np.empty(11)
        self.L.bzo_step_cell(C.byref(self.p), step, c, *[(_dptr(a) if a is not None else None)
                                                         for a in sl], _dptr(out), _dptr(mom))
        return out, mom

    def run(self, h, nsteps, step0=0):
        mom = None
        for n in range(step0, step0 + nsteps):
            h, mom = self.step(h, n)
        return h, mom

    def adjoint_step(self, h, lam, step=0, wD=0.0, grad_lid=None):
        """dJ/dh^n from lam = dJ/dh^{n+1}; dJ/dU (nx) is added to grad_lid."""
        h = self._state(h)
        lam = self._state(lam)
        out = np.empty_like(h)
        if grad_lid is None:
            grad_lid = np.zeros(self.nx)
        assert grad_lid.dtype == np.float64 and grad_lid.shape == (self.nx,)
        self.L.bzo_adjoint_step(C.byref(self.p), step, _dptr(h), _dptr(lam), _dptr(out),
                                _dptr(grad_lid), wD)
        return out, grad_lid

    def moments(self, h):
        h = self._state(h)
        mom = np.empty((self.nr, 11))
        self.L.bzo_moments(C.byref(self.p), _dptr(h), _dptr(mom))
        return mom

    def lid_shear(self, h, step=0):
        h = self._state(h)
        out = np.empty(self.nx + 1)
        self.L.bzo_lid_shear(C.byref(self.p), step, _dptr(h), _dptr(out))
        return out

    def mc_dNdt(self, h_cell, step=0):
        """Monte Carlo estimate of dN_j/dt for one cell: (gain, loss)."""
        h_cell = np.ascontiguousarray(h_cell, dtype=np.float64)
        assert h_cell.shape == (self.nvt,)
        gain = np.empty(self.nvt)
        loss = np.empty(self.nvt)
        self.L.bzo_mc_dNdt(C.byref(self.p), step, _dptr(h_cell), _dptr(gain), _dptr(loss))
        return gain, loss

    def _state(self, h):
        h = np.ascontiguousarray(h, dtype=np.float64)
        assert h.size == self.nr * self.nvt, (h.shape, self.nr, self.nvt)
        return h.reshape(self.nr, self.nvt)


def philox(ctr, key):
    """Philox4x32-10 words for one counter (4 uint32) and key (2 uint32)."""
    c = (C.c_uint32 * 4)(*[int(x) & 0xFFFFFFFF for x in ctr])
    k = (C.c_uint32 * 2)(*[int(x) & 0xFFFFFFFF for x in key])
    o = (C.c_uint32 * 4)()
    lib().bzo_philox4x32_10(c, k, o)
    return [int(x) for x in o]


def num_threads() -> int:
    return int(lib().bzo_num_threads())
