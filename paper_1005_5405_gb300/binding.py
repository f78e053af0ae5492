"""ctypes binding of the C ABI in include/bz.h (argument marshalling only).

Every function of the ABI is exposed under its C name; `Cavity` wraps a
handle for convenience.  PyTorch is used only for device memory and streams
(tensors' data pointers and `torch.cuda.current_stream().cuda_stream`).  The
library must be the in-tree build; there is no fallback of any kind: if the
shared object is missing or fails to load, the import raises.
"""
from __future__ import annotations

import ctypes as C
import os
from typing import Optional

import numpy as np

from .workloads import Problem

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "_lib", "libbz.so")

BZ_OK, BZ_EINVAL, BZ_ENOMEM, BZ_ECUDA, BZ_EDEVICE, BZ_ETIMEOUT, BZ_ENONFINITE, BZ_ESTATE, \
    BZ_EUNSUPPORTED = range(9)
BZ_F32, BZ_F64 = 0, 1
BZ_SHARED, BZ_PER_CELL = 0, 1
BZ_DO_STREAM, BZ_DO_COLLIDE, BZ_SPLIT = 1, 2, 4

STATUS_NAMES = {0: "BZ_OK", 1: "BZ_EINVAL", 2: "BZ_ENOMEM", 3: "BZ_ECUDA", 4: "BZ_EDEVICE",
                5: "BZ_ETIMEOUT", 6: "BZ_ENONFINITE", 7: "BZ_ESTATE", 8: "BZ_EUNSUPPORTED"}


class BzError(RuntimeError):
    def __init__(self, status: int, where: str, msg: str):
        super().__init__(f"{where}: {STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


class bz_space(C.Structure):
    _fields_ = [("nx", C.c_int32), ("ny", C.c_int32), ("kn", C.c_double),
                ("rx", C.c_double), ("ry", C.c_double)]


class bz_vel(C.Structure):
    _fields_ = [("nv", C.c_int32), ("vmax", C.c_double), ("rv", C.c_double)]


class bz_walls(C.Structure):
    _fields_ = [("lid_u0", C.c_double), ("lid_amp", C.c_double), ("lid_period", C.c_double),
                ("lid_profile", C.POINTER(C.c_double))]


class bz_params(C.Structure):
    _fields_ = [("n_pairs", C.c_int64), ("seed", C.c_uint32), ("instance", C.c_uint32),
                ("eps", C.c_double), ("cfl", C.c_double), ("kcoll", C.c_double),
                ("dtype", C.c_int32), ("sample_mode", C.c_int32)]


class bz_info(C.Structure):
    _fields_ = [("dt", C.c_double), ("dx", C.c_double), ("dy", C.c_double),
                ("dv", C.c_double), ("eps", C.c_double), ("kcoll", C.c_double),
                ("nodes", C.c_int64), ("state_bytes", C.c_int64), ("step", C.c_int64),
                ("nr", C.c_int32), ("nvt", C.c_int32), ("dtype", C.c_int32),
                ("threads_per_cell", C.c_int32), ("smem_bytes", C.c_int32),
                ("kernel_variant", C.c_int32), ("plan_batch", C.c_int32),
                ("plan_end", C.c_int64)]


_H = C.c_void_p
_V = C.c_void_p
_SIGNATURES = {
    "bz_create": [C.POINTER(bz_space), C.POINTER(bz_vel), C.POINTER(bz_walls),
                  C.POINTER(bz_params), C.POINTER(_H)],
    "bz_destroy": [_H],
    "bz_step": [_H, C.c_int32, _V],
    "bz_step_ex": [_H, C.c_int32, C.c_uint32, _V],
    "bz_moments": [_H, _V, _V],
    "bz_lid_shear": [_H, _V, _V],
    "bz_get_state": [_H, _V, C.POINTER(C.c_int64), _V],
    "bz_set_state": [_H, _V, C.c_int64, _V],
    "bz_set_lid": [_H, C.c_double, C.c_double, C.c_double, C.POINTER(C.c_double)],
    "bz_get_info": [_H, C.POINTER(bz_info)],
    "bz_stats": [_H, C.POINTER(C.c_int64)],
    "bz_sample_plan": [_H, C.c_int64, _V, _V, _V],
    "bz_sample_plan_cell": [_H, C.c_int64, C.c_int32, _V, _V, _V],
    "bz_philox": [C.c_uint32, C.c_uint32, _V, C.c_int64, _V],
    "bz_adjoint_step": [_H, C.c_int64, _V, _V, _V, _V, C.c_double, _V],
    "bz_profile": [_H, C.c_int32],
    "bz_profile_read": [_H, C.POINTER(C.c_double), C.POINTER(C.c_int64)],
    "bz_phase_clocks": [_H, C.POINTER(C.c_int64), C.c_int32],
    "bz_collide_noalloc": [C.POINTER(bz_space), C.POINTER(bz_vel), C.POINTER(bz_params),
                           C.c_int64, _V, _V, _V, _V],
    "bz_batch_create": [C.c_int32, C.POINTER(bz_space), C.POINTER(bz_vel), C.POINTER(bz_walls),
                        C.POINTER(bz_params), C.POINTER(_H)],
    "bz_batch_destroy": [_H],
    "bz_batch_step": [_H, C.c_int32, _V],
    "bz_batch_set_state": [_H, C.c_int32, _V, C.c_int64, _V],
    "bz_batch_get_state": [_H, C.c_int32, _V, C.POINTER(C.c_int64), _V],
    "bz_batch_moments": [_H, C.c_int32, _V, _V],
    "bz_batch_tune": [_H, C.c_int32, _V, C.POINTER(C.c_int32), C.POINTER(C.c_double),
                      C.POINTER(C.c_int32)],
    "bz_batch_schedule": [_H, C.POINTER(C.c_int32)],
}

_lib = None


def load(path: str = LIB_PATH):
    """Load libbz.so (raises if it is missing: there is no fallback path)."""
    global _lib
    if _lib is None:
        if not os.path.exists(path):
            raise ImportError(f"libbz.so not built at {path}; run "
                              f"`python -m paper_1005_5405_gb300.build`")
        L = C.CDLL(path)
        for name, args in _SIGNATURES.items():
            f = getattr(L, name)
            f.argtypes = args
            f.restype = C.c_int
        L.bz_last_error.argtypes = []
        L.bz_last_error.restype = C.c_char_p
        L.bz_version.argtypes = []
        L.bz_version.restype = C.c_char_p
        _lib = L
    return _lib


def exported_symbols():
    return sorted(list(_SIGNATURES) + ["bz_last_error", "bz_version"])


def check(status: int, where: str):
    if status != BZ_OK:
        raise BzError(status, where, load().bz_last_error().decode())


def _stream_ptr(stream) -> Optional[int]:
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def _ptr(x) -> int:
    """Data pointer of a torch tensor or numpy array (contiguous)."""
    if isinstance(x, np.ndarray):
        assert x.flags.c_contiguous
        return x.ctypes.data
    assert x.is_contiguous()
    return x.data_ptr()


class Cavity:
    """One driven-cavity solver instance on the current CUDA device."""

    def __init__(self, p: Problem, kcoll: float = 0.0):
        L = load()
        self.p = p
        self._prof = None
        prof_ptr = None
        if p.lid_profile is not None:
            self._prof = np.ascontiguousarray(p.lid_profile, dtype=np.float64)
            prof_ptr = self._prof.ctypes.data_as(C.POINTER(C.c_double))
        sp = bz_space(p.nx, p.ny, p.kn, p.rx, p.ry)
        ve = bz_vel(p.nv, p.vmax, p.rv)
        wa = bz_walls(p.lid_u0, p.lid_amp, p.lid_period, prof_ptr)
        pa = bz_params(p.nt, p.seed, p.instance, p.eps, p.cfl, kcoll,
                       BZ_F64 if p.dtype == "f64" else BZ_F32,
                       BZ_PER_CELL if p.per_cell else BZ_SHARED)
        h = _H()
        check(L.bz_create(C.byref(sp), C.byref(ve), C.byref(wa), C.byref(pa), C.byref(h)),
              "bz_create")
        self.h = h
        self.info = self.get_info()

    def close(self):
        if getattr(self, "h", None):
            load().bz_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ---------------------------------------------------------------------
    def get_info(self) -> bz_info:
        o = bz_info()
        check(load().bz_get_info(self.h, C.byref(o)), "bz_get_info")
        return o

    @property
    def torch_dtype(self):
        import torch
        return torch.float64 if self.p.dtype == "f64" else torch.float32

    def step(self, n: int = 1, stream=None):
        check(load().bz_step(self.h, n, _stream_ptr(stream)), "bz_step")

    def step_ex(self, n: int, flags: int, stream=None):
        check(load().bz_step_ex(self.h, n, flags, _stream_ptr(stream)), "bz_step_ex")

    def moments(self, out=None, stream=None):
        import torch
        if out is None:
            out = torch.empty((self.p.nr, 11), dtype=torch.float64, device="cuda")
        check(load().bz_moments(self.h, _ptr(out), _stream_ptr(stream)), "bz_moments")
        return out

    def lid_shear(self, out=None, stream=None):
        import torch
        if out is None:
            out = torch.empty(self.p.nx + 1, dtype=torch.float64, device="cuda")
        check(load().bz_lid_shear(self.h, _ptr(out), _stream_ptr(stream)), "bz_lid_shear")
        return out

    def get_state(self, out=None, stream=None):
        import torch
        if out is None:
            out = torch.empty((self.p.nr, self.p.nvt), dtype=self.torch_dtype, device="cuda")
        st = C.c_int64()
        check(load().bz_get_state(self.h, _ptr(out), C.byref(st), _stream_ptr(stream)),
              "bz_get_state")
        return out, st.value

    def set_state(self, src, step: int = 0, stream=None):
        import torch
        if isinstance(src, np.ndarray):
            src = torch.from_numpy(np.ascontiguousarray(src)).to(self.torch_dtype).cuda()
        assert src.dtype == self.torch_dtype and src.numel() == self.p.nr * self.p.nvt
        check(load().bz_set_state(self.h, _ptr(src.contiguous()), step, _stream_ptr(stream)),
              "bz_set_state")
        torch.cuda.current_stream().synchronize()

    def set_lid(self, u0=0.0, amp=0.0, period=0.0, profile=None):
        ptr = None
        if profile is not None:
            self._prof = np.ascontiguousarray(profile, dtype=np.float64)
            ptr = self._prof.ctypes.data_as(C.POINTER(C.c_double))
        check(load().bz_set_lid(self.h, u0, amp, period, ptr), "bz_set_lid")

    def stats(self):
        out = (C.c_int64 * 8)()
        check(load().bz_stats(self.h, out), "bz_stats")
        return list(out)

    def profile(self, enable):
        """0 off; 1 (or True) per-kernel event timing; 2 also the phase trace."""
        check(load().bz_profile(self.h, int(enable)), "bz_profile")

    def phase_clocks(self):
        out = (C.c_int64 * 72)()
        check(load().bz_phase_clocks(self.h, out, 72), "bz_phase_clocks")
        return np.array(list(out), dtype=np.int64).reshape(8, 9)

    def profile_read(self):
        """(ms, launches) per kernel class: walls, sampling, per-cell, streaming."""
        ms = (C.c_double * 4)()
        n = (C.c_int64 * 4)()
        check(load().bz_profile_read(self.h, ms, n), "bz_profile_read")
        return list(ms), list(n)

    def sample_plan(self, step: int):
        idx = np.zeros((self.p.nt, 4), dtype=np.int32)
        W = np.zeros(self.p.nt, dtype=np.float64)
        check(load().bz_sample_plan(self.h, step, idx.ctypes.data, W.ctypes.data,
                                    _stream_ptr(None)), "bz_sample_plan")
        return idx, W

    def sample_plan_cell(self, step: int, cell: int):
        """bz_sample_plan_cell: the sample set of one cell as the per-cell
        step draws it ((nt, 4) node indices, (nt,) weights W)."""
        idx = np.zeros((self.p.nt, 4), dtype=np.int32)
        W = np.zeros(self.p.nt, dtype=np.float64)
        check(load().bz_sample_plan_cell(self.h, step, cell, idx.ctypes.data, W.ctypes.data,
                                         _stream_ptr(None)), "bz_sample_plan_cell")
        return idx, W


    def adjoint_step(self, step: int, h_n, lam_in, lam_out=None, grad_lid=None, wD: float = 0.0,
                     stream=None):
        """bz_adjoint_step: dJ/dh^n from lam_in = dJ/dh^{n+1} (CUDA tensors of
        shape (nr, nv^3) in the handle's dtype; lam_out may be lam_in).  dJ/dU
        of the lid faces is added to grad_lid ((nx,) float64 CUDA tensor) when
        given; wD weights the lid shear D_n of h_n in J.  Returns lam_out."""
        import torch
        if lam_out is None:
            lam_out = torch.empty_like(lam_in)
        for t in (h_n, lam_in, lam_out):
            assert t.dtype == self.torch_dtype and t.numel() == self.p.nr * self.p.nvt
        if grad_lid is not None:
            assert grad_lid.dtype == torch.float64 and grad_lid.numel() == self.p.nx
        check(load().bz_adjoint_step(self.h, step, _ptr(h_n), _ptr(lam_in), _ptr(lam_out),
                                     _ptr(grad_lid) if grad_lid is not None else None,
                                     float(wD), _stream_ptr(stream)), "bz_adjoint_step")
        return lam_out


NOALLOC_MAX_PAIRS = 65536


def collide_noalloc(p: Problem, step: int, h_in, h_out, mom=None, stream=None):
    """bz_collide_noalloc: one relaxation step of the caller's state without
    any device allocation by the library (see include/bz.h).  h_in/h_out are
    CUDA tensors of shape (nr, nv^3) in the problem's dtype; mom is an
    optional (nr, 11) float64 CUDA tensor; p.eps must be > 0."""
    sp = bz_space(p.nx, p.ny, p.kn, p.rx, p.ry)
    ve = bz_vel(p.nv, p.vmax, p.rv)
    pa = bz_params(p.nt, p.seed, p.instance, p.eps, p.cfl, 0.0,
                   BZ_F64 if p.dtype == "f64" else BZ_F32,
                   BZ_PER_CELL if p.per_cell else BZ_SHARED)
    check(load().bz_collide_noalloc(C.byref(sp), C.byref(ve), C.byref(pa), step, _ptr(h_in),
                                    _ptr(h_out), _ptr(mom) if mom is not None else None,
                                    _stream_ptr(stream)), "bz_collide_noalloc")


def _structs(p: Problem, kcoll: float = 0.0):
    prof = None
    if p.lid_profile is not None:
        prof = np.ascontiguousarray(p.lid_profile, dtype=np.float64)
    wa = bz_walls(p.lid_u0, p.lid_amp, p.lid_period,
                  prof.ctypes.data_as(C.POINTER(C.c_double)) if prof is not None else None)
    pa = bz_params(p.nt, p.seed, p.instance, p.eps, p.cfl, kcoll,
                   BZ_F64 if p.dtype == "f64" else BZ_F32,
                   BZ_PER_CELL if p.per_cell else BZ_SHARED)
    return bz_space(p.nx, p.ny, p.kn, p.rx, p.ry), bz_vel(p.nv, p.vmax, p.rv), wa, pa, prof


class Batch:
    """Independent cavity instances advanced together (bz_batch_*)."""

    def __init__(self, problems):
        L = load()
        self.problems = list(problems)
        n = len(self.problems)
        st = [_structs(p) for p in self.problems]
        self._keep = [s[4] for s in st]
        sp = (bz_space * n)(*[s[0] for s in st])
        ve = (bz_vel * n)(*[s[1] for s in st])
        wa = (bz_walls * n)(*[s[2] for s in st])
        pa = (bz_params * n)(*[s[3] for s in st])
        h = _H()
        check(L.bz_batch_create(n, sp, ve, wa, pa, C.byref(h)), "bz_batch_create")
        self.h = h

    def close(self):
        if getattr(self, "h", None):
            load().bz_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def step(self, n=1, stream=None):
        check(load().bz_batch_step(self.h, n, _stream_ptr(stream)), "bz_batch_step")

    def set_state(self, i, src, step=0, stream=None):
        import torch
        p = self.problems[i]
        if isinstance(src, np.ndarray):
            src = torch.from_numpy(np.ascontiguousarray(src, dtype=np.float32)).cuda()
        assert src.dtype == torch.float32 and src.numel() == p.nr * p.nvt
        check(load().bz_batch_set_state(self.h, i, _ptr(src.contiguous()), step,
                                        _stream_ptr(stream)), "bz_batch_set_state")

    def get_state(self, i, stream=None):
        import torch
        p = self.problems[i]
        out = torch.empty((p.nr, p.nvt), dtype=torch.float32, device="cuda")
        st = C.c_int64()
        check(load().bz_batch_get_state(self.h, i, _ptr(out), C.byref(st), _stream_ptr(stream)),
              "bz_batch_get_state")
        return out, st.value

    def moments(self, i, stream=None):
        import torch
        out = torch.empty((self.problems[i].nr, 11), dtype=torch.float64, device="cuda")
        check(load().bz_batch_moments(self.h, i, _ptr(out), _stream_ptr(stream)), "bz_batch_moments")
        return out

    def tune(self, trial_steps=2, stream=None):
        choice = C.c_int32()
        ms = (C.c_double * 16)()
        nc = C.c_int32()
        check(load().bz_batch_tune(self.h, trial_steps, _stream_ptr(stream), C.byref(choice), ms,
                                   C.byref(nc)), "bz_batch_tune")
        return choice.value, list(ms)[: nc.value]

    def schedule(self):
        out = (C.c_int32 * 4)()
        check(load().bz_batch_schedule(self.h, out), "bz_batch_schedule")
        return {"threads": out[0], "ctas": out[1], "strip": out[2], "fanout_branches": out[3]}


def philox(key, ctr):
    """Device Philox4x32-10 words for counters ctr (n,4) under key (k0, k1)."""
    ctr = np.ascontiguousarray(ctr, dtype=np.uint32).reshape(-1, 4)
    out = np.zeros_like(ctr)
    check(load().bz_philox(int(key[0]) & 0xFFFFFFFF, int(key[1]) & 0xFFFFFFFF, ctr.ctypes.data,
                           ctr.shape[0], out.ctypes.data), "bz_philox")
    return out
