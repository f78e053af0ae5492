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


def test_per_cell_out_of_box_counter():
    """Samples with a node outside the box are counted cell by cell: the
    count equals the oracle's over every cell's own set."""
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
