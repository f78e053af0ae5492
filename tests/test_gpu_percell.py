"""Per-cell sample sets (BZ_PER_CELL): every cell draws its own Monte Carlo
samples, the Philox counter carrying the cell index.  The generic per-cell
kernel draws them in its gather phase; results must match the oracle run in
the same mode."""
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


CASES = [
    workloads.small(nx=5, ny=4, nv=12, vmax=4.0, nt=800, seed=21, dtype="f64", per_cell=True),
    workloads.small(nx=4, ny=6, nv=16, vmax=4.0, nt=2500, seed=22, dtype="f32", per_cell=True,
                    eps=0.1),
    workloads.small(nx=3, ny=3, nv=8, vmax=2.0, nt=1500, seed=23, dtype="f32", per_cell=True),
]
IDS = ["f64_12", "f32_16", "outbox_8"]


@pytest.mark.parametrize("p", CASES, ids=IDS)
def test_per_cell_fused_step_matches_oracle(p):
    cav, o, h0 = make(p)
    assert cav.get_info().kernel_variant == 0
    h_g = h0
    for n in range(3):
        cav.step(1)
        h_o, mom_o = o.step(h_g, n)           # the oracle restarts from the GPU state
        h_g = state(cav)
        assert f_metric(o, h_g, h_o) < (1e-10 if p.dtype == "f64" else 1e-5), n
    mom_g = cav.moments().cpu().numpy()
    assert np.allclose(mom_g, mom_o, rtol=1e-4, atol=1e-5 * (1 + np.abs(mom_o).max()))


@pytest.mark.parametrize("p", CASES[:2], ids=IDS[:2])
def test_per_cell_collide_matches_oracle(p):
    cav, o, h0 = make(p)
    cav.step_ex(1, binding.BZ_DO_COLLIDE)
    h_o, _ = o.collide(h0, step=0)
    assert f_metric(o, state(cav), h_o) < (1e-10 if p.dtype == "f64" else 1e-5)


def test_per_cell_redraw_queue_capacity_changes_nothing(monkeypatch):
    """The FP32 per-cell sampler queues the samples near a face for an FP64
    redraw after its loop; with the queue cut to 0 or 5 entries they are
    redrawn in place instead.  The samples are the same either way: each
    run matches the oracle step by step, the runs agree to the rounding of
    the shared-memory atomics, and the out-of-box and face-proximity counters
    are equal."""
    p = workloads.small(nx=4, ny=4, nv=24, vmax=4.5, nt=8000, seed=26, dtype="f32",
                        per_cell=True, eps=0.1)
    out = {}
    for cap in (None, "0", "5"):
        if cap is None:
            monkeypatch.delenv("BZ_REDRAW_CAP", raising=False)
        else:
            monkeypatch.setenv("BZ_REDRAW_CAP", cap)
        cav, o, h0 = make(p, seed=27)
        h_g = h0
        for n in range(3):
            cav.step(1)
            h_o, _ = o.step(h_g, n)
            h_g = state(cav)
            assert f_metric(o, h_g, h_o) < 1e-5, (cap, n)
        out[cap] = (h_g, list(cav.stats()[1:3]))
    for cap in ("0", "5"):
        assert f_metric(o, out[cap][0], out[None][0]) < 1e-6, cap
        assert out[cap][1] == out[None][1], cap


def test_per_cell_sets_differ_from_the_shared_set():
    """The same problem with the shared set gives a different result (the
    samples differ), while both conserve mass exactly."""
    p = CASES[1]
    a, o, h0 = make(p)
    q = workloads.small(nx=4, ny=6, nv=16, vmax=4.0, nt=2500, seed=22, dtype="f32", eps=0.1)
    b, _, _ = make(q, h0=h0)
    a.step_ex(1, binding.BZ_DO_COLLIDE)
    b.step_ex(1, binding.BZ_DO_COLLIDE)
    ha, hb = state(a), state(b)
    assert f_metric(o, ha, hb) > 1e-6
    w = o.weights()
    assert np.allclose((ha * w).sum(axis=1), (h0 * w).sum(axis=1), atol=1e-5)


@pytest.mark.parametrize("cap", [None, "3"])
def test_per_cell_out_of_box_counter(monkeypatch, cap):
    """Samples with a node outside the box are counted cell by cell: the
    count equals the oracle's over every cell's own set (also when the FP64
    redraw queue holds 3 samples and the rest are redrawn in place)."""
    if cap is not None:
        monkeypatch.setenv("BZ_REDRAW_CAP", cap)
    p = CASES[2]
    cav, o, h0 = make(p)
    cav.step(1)
    st = cav.stats()
    expect = sum(int((o.samples(0, cellword=c)["idx"] < 0).any(axis=1).sum()) for c in range(p.nr))
    assert st[1] == expect


def test_per_cell_adjoint_is_unsupported():
    torch = pytest.importorskip("torch")
    p = CASES[1]
    cav = binding.Cavity(p)
    h = torch.zeros((p.nr, p.nvt), dtype=torch.float32, device="cuda")
    with pytest.raises(binding.BzError) as e:
        cav.adjoint_step(0, h, h.clone())
    assert e.value.status == binding.BZ_EUNSUPPORTED


@pytest.mark.parametrize("nv,vmax,nt,dtype", [(24, 4.5, 40000, "f32"), (32, 5.0, 40000, "f32"),
                                              (8, 2.0, 20000, "f32"), (8, 0.01, 4000, "f32"),
                                              (12, 4.0, 2000, "f64")])
def test_per_cell_sample_plan_matches_oracle(nv, vmax, nt, dtype):
    """Every cell's own sample set as the per-cell step draws it: the node
    indices equal the oracle's FP64 selection for every sample (FP32 handles
    draw in FP32 and redraw in FP64 near a face), and W = cw |s| is within
    the FP32 error of s (2e-5 cw absolute; 1e-12 relative for FP64).  The
    handles use the shared set: the per-cell sampler does not depend on the
    mode, and 4x10^4 per-cell samples would not fit the per-cell kernel's
    shared memory."""
    p = workloads.small(nx=3, ny=2, nv=nv, vmax=vmax, nt=nt, seed=31, dtype=dtype)
    cav = binding.Cavity(p)
    o = oracle.Oracle(**p.kwargs())
    prev = None
    for step, cell in [(0, 0), (1, 5), (57, 3), (57, 4)]:
        idx, W = cav.sample_plan_cell(step, cell)
        s = o.samples(step, cellword=cell)
        same = (idx == s["idx"]).all(1)
        assert same.all(), (np.nonzero(~same), s["near_face"][~same])
        cw = float(np.max(s["W"]) / np.max(np.abs(s["s"])))
        err = np.abs(W - s["W"])
        if dtype == "f32":
            assert np.max(err) <= 2e-5 * cw + 1e-7 * np.max(s["W"])
        else:
            assert np.max(err) <= 1e-12 * np.max(s["W"])
        if prev is not None:
            assert not np.array_equal(W, prev)        # the cells draw different sets
        prev = W
    print(f"per-cell sampler: 0 node mismatches in {4 * nt} samples")


def test_per_cell_sample_plan_rejects_bad_arguments():
    p = CASES[1]
    cav = binding.Cavity(p)
    for step, cell in [(-1, 0), (0, -1), (0, p.nr)]:
        with pytest.raises(binding.BzError) as e:
            cav.sample_plan_cell(step, cell)
        assert e.value.status == binding.BZ_EINVAL
