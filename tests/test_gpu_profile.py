"""Timing support of the active-node path on the GPU: the per-kernel event
timing (bz_profile) inside the two-step CUDA graphs, and the plan batch the
handle reports (bz_info.plan_batch, plan_end)."""
import numpy as np
import pytest

import oracle
from paper_1005_5405_gb300 import binding, workloads
from tests.gpu_helpers import f_metric, state

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    torch.cuda.set_device(0)
    yield


@pytest.fixture(autouse=True)
def _env(monkeypatch):
    for k in ("BZ_KERNEL", "BZ_LAZY_MCAP", "BZ_LAZY_ORDER", "BZ_LAZY_NOORDER", "BZ_LAZY_ORDER_CHUNK",
              "BZ_LAZY_G", "BZ_LAZY_TMA", "BZ_LAZY_AHEAD", "BZ_GRAPH"):
        monkeypatch.delenv(k, raising=False)


def _v32(nxy):
    return workloads.small(nx=nxy, ny=nxy, nv=32, vmax=5.0, nt=20000, seed=3, kn=0.05 * 256 / nxy,
                           lid_u0=0.0, lid_amp=0.05, lid_period=50.0)


@pytest.mark.parametrize("graphs", ["1", "0"])
def test_profiled_steps_match_unprofiled(monkeypatch, graphs):
    """With profiling on, the steps run as before (in two-step graphs whose
    timed launches are event nodes armed with fresh events per replay, or
    launch by launch): the states match an unprofiled handle's to FP32
    rounding, and bz_profile_read counts one per-cell launch per step with a
    positive time (inside the graphs only the per-cell kernel is timed: the
    walls count the steps run launch by launch)."""
    import torch
    monkeypatch.setenv("BZ_GRAPH", graphs)
    monkeypatch.setenv("BZ_LAZY_ORDER", "1")
    p = _v32(12)
    h0 = workloads.warm_state(p, seed=21).astype(np.float32)
    a, b = binding.Cavity(p), binding.Cavity(p)
    assert a.get_info().kernel_variant == 2
    a.set_state(h0, step=0)
    b.set_state(h0, step=0)
    a.profile(True)
    a.step(6)
    a.step(3)
    torch.cuda.synchronize()
    a.profile(False)
    ms, n = a.profile_read()
    b.step(6)
    b.step(3)
    o = oracle.Oracle(**p.kwargs())
    assert f_metric(o, state(a), state(b)) < 1e-6
    assert n[2] == 9 and n[0] == (1 if graphs == "1" else 9), n
    assert ms[0] > 0 and ms[2] > 0, ms
    # Profiling off again: the graphs are captured without events.
    a.step(4)
    b.step(4)
    assert f_metric(o, state(a), state(b)) < 1e-6
    assert a.profile_read()[1] == [0, 0, 0, 0]


def test_plan_batch_fills_the_order_kernels_waves():
    """Small runs keep 32 steps per plan batch; where the term order runs
    (from 12 CTA iterations on) and 32 plans need more than one wave of its
    CTAs, the batch grows to fill the last wave, even and at most 64.  The
    first step builds the batch: plan_end is then plan_batch."""
    small = binding.Cavity(_v32(12))
    assert small.get_info().plan_batch == 32
    cav = binding.Cavity(_v32(96))           # 2304 groups of 4 cells: 15 per CTA
    info = cav.get_info()
    assert info.kernel_variant == 2
    K = info.plan_batch
    assert 32 <= K <= 64 and K % 2 == 0, K
    h0 = workloads.warm_state(_v32(96), seed=5).astype(np.float32)
    cav.set_state(h0, step=0)
    cav.step(3)
    info = cav.get_info()
    assert info.step == 3 and info.plan_end == K
    cav.step(K - 3)
    cav.step(2)
    assert cav.get_info().plan_end == 2 * K
