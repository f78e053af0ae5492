"""Batched instances (bz_batch_*): every instance of a batch advances exactly
as a single-instance handle of the same problem would (and as the oracle)."""
import numpy as np
import pytest

import oracle
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


def _problems():
    return [
        workloads.small(nx=6, ny=5, nv=12, vmax=4.0, nt=1500, seed=31, lid_u0=0.08),
        workloads.small(nx=4, ny=7, nv=16, vmax=4.0, nt=2500, seed=32, kn=0.5, lid_u0=0.15,
                        instance=1),
        workloads.small(nx=5, ny=5, nv=20, vmax=4.5, nt=3000, seed=33, kn=2.0, lid_u0=0.03,
                        instance=2),
    ]


def _warm(p, seed):
    return workloads.warm_state(p, seed=seed).astype(np.float32)


@pytest.mark.parametrize("mode", ["persistent", "fanout", "fanout_ordered", "lz", "lz_ordered",
                                  "lz_per_step", "lz_overflow"])
def test_batch_matches_single_instances_and_oracle(monkeypatch, mode):
    """Every schedule: the persistent 4-node-vector kernels over all
    instances; the fan-out graph of the instances' own active-node steps
    (each with its sample plan on its own second stream), also with the joint
    term order forced on in every instance and in the single-instance
    handles; the persistent active-node kernels over all instances, copying
    each instance's plans built ahead (also with the term order forced on),
    or building every instance's plan in the step, and with every instance's
    compact arrays capped below its active nodes (every step then takes the
    gated 4-node-vector fallback).  Three steps without a read, then one step
    at a time against the oracle restarted from the batch's state."""
    for k in ("BZ_LAZY_ORDER", "BZ_LAZY_MCAP", "BZ_BATCH_MODE", "BZ_BATCH_LZ_AHEAD"):
        monkeypatch.delenv(k, raising=False)
    if mode.startswith("fanout"):
        monkeypatch.setenv("BZ_BATCH_MODE", "fanout")
    if mode.startswith("lz"):
        monkeypatch.setenv("BZ_BATCH_MODE", "lz")
    if mode in ("fanout_ordered", "lz_ordered"):
        monkeypatch.setenv("BZ_LAZY_ORDER", "1")
    if mode == "lz_per_step":
        monkeypatch.setenv("BZ_BATCH_LZ_AHEAD", "0")
    if mode == "lz_overflow":
        monkeypatch.setenv("BZ_LAZY_MCAP", "8")
    ps = _problems()
    b = binding.Batch(ps)
    expect = {"persistent": 0, "lz": -1, "lz_ordered": -1, "lz_per_step": -1, "lz_overflow": -1}.get(mode)
    branches = b.schedule()["fanout_branches"]
    assert branches == expect if expect is not None else branches > 0
    singles = []
    for i, p in enumerate(ps):
        h0 = _warm(p, 40 + i)
        b.set_state(i, h0, step=2)
        cav, o, _ = make(p, h0=h0)
        cav.set_state(h0, step=2)
        singles.append((cav, o, h0.astype(np.float64)))
    b.step(3)
    for i, (cav, o, h0) in enumerate(singles):
        cav.step(3)
        hb, st = b.get_state(i)
        assert st == 5
        assert f_metric(o, hb.double().cpu().numpy(), state(cav)) < 1e-6, i
    for n in range(5, 7):
        prev = [b.get_state(i)[0].double().cpu().numpy() for i in range(len(ps))]
        b.step(1)
        for i, (cav, o, _) in enumerate(singles):
            ref, mom = o.step(prev[i], n)
            hb, st = b.get_state(i)
            assert st == n + 1
            assert f_metric(o, hb.double().cpu().numpy(), ref) < 1e-5, (i, n)
            assert np.allclose(b.moments(i).cpu().numpy(), mom, rtol=1e-4,
                               atol=1e-5 * (1 + np.abs(mom).max())), (i, n)


def test_tuner_keeps_state_and_graph_replay_is_exact(monkeypatch):
    ps = _problems()
    b = binding.Batch(ps)
    for i, p in enumerate(ps):
        b.set_state(i, _warm(p, 50 + i), step=0)
    before = [b.get_state(i)[0].clone() for i in range(len(ps))]
    choice, ms = b.tune(trial_steps=1)
    assert 0 <= choice < len(ms) and min(t for t in ms if t > 0) == ms[choice]
    for i in range(len(ps)):
        h, st = b.get_state(i)
        assert st == 0 and bool((h == before[i]).all())
    sched = b.schedule()
    assert sched["threads"] in (512, 1024) and sched["strip"] in (4, 8, 16)
    assert sched["fanout_branches"] in (-1, 0, 1, 2, 4, 8)
    # 9 persistent 4-node schedules + 4 fan-out widths + the persistent
    # active-node schedule
    assert len(ms) == 14
    b.step(4)
    monkeypatch.setenv("BZ_GRAPH", "0")
    c = binding.Batch(ps)
    for i, p in enumerate(ps):
        c.set_state(i, _warm(p, 50 + i), step=0)
    c.step(4)
    o = oracle.Oracle(**ps[0].kwargs())
    assert f_metric(o, b.get_state(0)[0].double().cpu().numpy(),
                    c.get_state(0)[0].double().cpu().numpy()) < 1e-6


def test_batch_rejects_unsupported_instances():
    with pytest.raises(binding.BzError) as e:
        binding.Batch([workloads.small(nv=10)])
    assert e.value.status == binding.BZ_EUNSUPPORTED
    with pytest.raises(binding.BzError) as e:
        binding.Batch([workloads.small(nv=12, dtype="f64")])
    assert e.value.status == binding.BZ_EUNSUPPORTED
