"""Stretched velocity and spatial grids (Sec. 5.1) on the GPU against the
oracle: node selection on stretched velocity cells, streaming with per-cell
widths, full steps, the width-weighted lid shear, total-mass conservation.
FP32 grids with a multiple-of-4 velocity axis run the active-node kernel
(and, forced, the 4-node-vector kernel); the others the generic kernel."""
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


@pytest.fixture(params=["auto", "ordered", "cell4", "generic"])
def kernel(request, monkeypatch):
    for k in ("BZ_KERNEL", "BZ_LAZY_ORDER", "BZ_LAZY_NOORDER", "BZ_LAZY_ORDER_CHUNK"):
        monkeypatch.delenv(k, raising=False)
    if request.param == "ordered":
        monkeypatch.setenv("BZ_LAZY_ORDER", "1")
        monkeypatch.setenv("BZ_LAZY_ORDER_CHUNK", "16")
    elif request.param in ("cell4", "generic"):
        monkeypatch.setenv("BZ_KERNEL", request.param)
    return request.param


def expected_variant(p, kernel):
    """The per-cell kernel the library picks for p under the fixture."""
    fast = p.dtype == "f32" and p.nv % 4 == 0 and p.nv >= 12
    if kernel == "generic" or not fast:
        return 0
    return 1 if kernel == "cell4" else 2


CASES = [
    workloads.small(nx=5, ny=4, nv=10, vmax=3.0, nt=900, seed=31, dtype="f64", eps=0.1,
                    rv=0.9, rx=0.8, ry=0.85),
    workloads.small(nx=6, ny=5, nv=12, vmax=3.0, nt=2000, seed=32, dtype="f32", eps=0.1,
                    rv=0.945, rx=0.9, ry=0.95),
    workloads.small(nx=4, ny=4, nv=12, vmax=4.0, nt=1500, seed=33, dtype="f32", rx=0.8),
    workloads.small(nx=4, ny=3, nv=16, vmax=3.0, nt=1500, seed=34, dtype="f32", rv=0.9),
]
IDS = ["f64_all", "f32_all", "f32_space_only", "f32_velocity_only"]


@pytest.mark.parametrize("p", CASES, ids=IDS)
def test_sample_plan_on_stretched_velocity_cells(p):
    cav = binding.Cavity(p)
    o = oracle.Oracle(**p.kwargs())
    idx, W = cav.sample_plan(3)
    ref = o.samples(3)
    assert np.array_equal(idx, ref["idx"])
    assert np.allclose(W, ref["W"], rtol=0, atol=1e-12 * np.abs(ref["W"]).max())


@pytest.mark.parametrize("p", CASES, ids=IDS)
def test_streaming_with_per_cell_widths(p, kernel):
    cav, o, h0 = make(p)
    assert cav.get_info().kernel_variant == expected_variant(p, kernel)
    cav.step_ex(1, binding.BZ_DO_STREAM)
    assert f_metric(o, state(cav), o.stream(h0, 0)) < (1e-12 if p.dtype == "f64" else 1e-6)


@pytest.mark.parametrize("p", CASES, ids=IDS)
def test_fused_steps_on_stretched_grids(p, kernel):
    cav, o, h0 = make(p)
    assert cav.get_info().kernel_variant == expected_variant(p, kernel)
    h_g = h0
    for n in range(3):
        cav.step(1)
        h_o, mom_o = o.step(h_g, n)           # the oracle restarts from the GPU state
        h_g = state(cav)
        assert f_metric(o, h_g, h_o) < (1e-10 if p.dtype == "f64" else 1e-5), n
    mom_g = cav.moments().cpu().numpy()
    assert np.allclose(mom_g, mom_o, rtol=1e-4, atol=1e-5 * (1 + np.abs(mom_o).max()))


def test_lid_shear_is_the_width_weighted_mean(kernel):
    p = CASES[1]
    cav, o, h0 = make(p)
    cav.step(2)
    h = state(cav)
    d = cav.lid_shear().cpu().numpy()
    ref = o.lid_shear(h, 2)
    assert np.allclose(d, ref, rtol=1e-4, atol=1e-6 * np.abs(ref).max())


@pytest.mark.parametrize("p", [CASES[0], CASES[1], CASES[3]], ids=["f64_all", "f32_all", "f32_velocity_only"])
def test_total_mass_is_conserved_on_the_gpu(p, kernel):
    cav, o, h0 = make(p)
    dx, dy = o.cell_widths()
    area = np.outer(dy, dx).ravel()
    w = o.weights()
    m0 = area @ (h0 @ w)
    cav.step(3)
    m3 = area @ (state(cav) @ w)
    tol = 1e-12 if p.dtype == "f64" else 1e-6
    assert abs(m3 - m0) < tol * (area @ (np.abs(h0) @ w))


def test_stretched_grids_reject_the_adjoint():
    torch = pytest.importorskip("torch")
    p = CASES[1]
    cav = binding.Cavity(p)
    h = torch.zeros((p.nr, p.nvt), dtype=torch.float32, device="cuda")
    with pytest.raises(binding.BzError) as e:
        cav.adjoint_step(0, h, h.clone())
    assert e.value.status == binding.BZ_EUNSUPPORTED
