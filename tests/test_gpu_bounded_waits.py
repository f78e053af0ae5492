"""Bounded waits on the GPU.  The active-node kernel's bulk-copy ring
(BZ_LAZY_TMA=1) waits on mbarriers; each wait gives up after one second of
the global timer, sets the handle's error word and lets the kernel finish.
A test switch makes CTA 0 expect 16 bytes more than its first copies bring,
so that its first wait runs out without any fault: bz_stats then returns
BZ_ETIMEOUT once, and the handle and the context stay usable."""
import time

import pytest

from paper_1005_5405_gb300 import binding, workloads
from tests.gpu_helpers import f_metric, make, state

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    torch.cuda.set_device(0)


def test_ring_wait_that_runs_out_is_reported(monkeypatch):
    for k in ("BZ_KERNEL", "BZ_LAZY_MCAP", "BZ_LAZY_ORDER", "BZ_LAZY_NOORDER", "BZ_LAZY_G"):
        monkeypatch.delenv(k, raising=False)
    monkeypatch.setenv("BZ_LAZY_TMA", "1")
    p = workloads.small(nx=8, ny=8, nv=32, vmax=5.0, nt=20000, seed=3, kn=0.05 * 256 / 8)
    cav, o, h0 = make(p, seed=11)
    assert cav.get_info().kernel_variant == 2
    cav.step(1)
    cav.stats()                                   # no timeout in a normal step

    monkeypatch.setenv("BZ_LAZY_TMA_TIMEOUT_TEST", "1")
    t0 = time.time()
    try:
        cav.step(1)
    except binding.BzError as e:                  # the step's result is invalid
        assert e.status == binding.BZ_ENONFINITE
    with pytest.raises(binding.BzError) as e:
        cav.stats()
    elapsed = time.time() - t0
    assert e.value.status == binding.BZ_ETIMEOUT
    print(f"the wait ran out and the step ended after {elapsed:.1f} s")
    assert elapsed < 30.0
    cav.stats()                                   # reported once

    # The handle still steps correctly.
    monkeypatch.delenv("BZ_LAZY_TMA_TIMEOUT_TEST")
    cav.set_state(h0.astype("float32"), step=0)
    cav.step(1)
    h_o, _ = o.step(h0, 0)
    err = f_metric(o, state(cav), h_o)
    print(f"after the timeout: one step from the initial state matches the oracle to {err:.2e}")
    assert err < 1e-5
    cav.stats()
