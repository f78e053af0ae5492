"""bz_collide_noalloc: the collision step for callers that cannot allocate
device memory (pool-allocator applications that forbid cudaMalloc, and
latency-critical loops where cudaMalloc/cudaFree would synchronise the
device).  It must give the same result as the ordinary entry point
(bz_step_ex with BZ_DO_COLLIDE on a handle), call after call, although its
only scratch is a static device array reused by every call.

This file is collected last on purpose, so that a run that stops at the first
failure has already run every other test; it passes alone in a fresh process
as well as after the rest of the suite."""
import numpy as np
import pytest

from paper_1005_5405_gb300 import binding, workloads


def _problem(dtype, nt=3000):
    return workloads.small(nx=6, ny=5, nv=12, vmax=4.0, nt=nt, seed=13, dtype=dtype, eps=0.1)


def test_noalloc_rejects_overlapping_buffers():
    """h_in and h_out must not share a byte (checked on the host before any
    device work, so this runs without a GPU too): an output that starts one
    element into the input is refused, the same buffer twice as well."""
    p = _problem("f32")
    buf = np.zeros(p.nr * p.nvt + 1, dtype=np.float32)
    for a, b in ((buf[:-1], buf[1:]), (buf[1:], buf[:-1]), (buf[:-1], buf[:-1])):
        with pytest.raises(binding.BzError) as e:
            binding.collide_noalloc(p, 0, a, b, stream=0)
        assert e.value.status == binding.BZ_EINVAL and "overlap" in str(e.value)


def test_noalloc_rejects_too_many_samples():
    """The sample set must fit the static scratch (checked before any device
    work, so this runs without a GPU too)."""
    p = _problem("f32", nt=binding.NOALLOC_MAX_PAIRS + 1)
    h = np.zeros((p.nr, p.nvt), dtype=np.float32)
    with pytest.raises(binding.BzError) as e:
        binding.collide_noalloc(p, 0, h, np.zeros_like(h), stream=0)
    assert e.value.status == binding.BZ_EINVAL and "static scratch" in str(e.value)


@pytest.mark.gpu
@pytest.mark.parametrize("dtype", ["f32", "f64"])
def test_noalloc_matches_collide_entry_point(dtype):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    import oracle
    from tests.gpu_helpers import f_metric

    torch.cuda.set_device(0)
    p = _problem(dtype)
    tdt = torch.float64 if dtype == "f64" else torch.float32
    h0 = torch.from_numpy(workloads.warm_state(p, seed=21)).to(tdt).cuda()

    # The ordinary entry point: two collision steps on a handle.
    cav = binding.Cavity(p)
    cav.set_state(h0.clone(), step=4)
    ref, mref = [], []
    for _ in range(2):
        cav.step_ex(1, binding.BZ_DO_COLLIDE)
        ref.append(cav.get_state()[0].clone())
        mref.append(cav.moments().clone())
    torch.cuda.synchronize()

    # The allocation-free entry point, two calls in a row (steps 4 and 5).
    o = oracle.Oracle(**p.kwargs())
    src = h0.clone()
    for k, step in enumerate((4, 5)):
        dst = torch.empty_like(src)
        mom = torch.empty((p.nr, 11), dtype=torch.float64, device="cuda")
        binding.collide_noalloc(p, step, src, dst, mom)
        torch.cuda.synchronize()
        err = f_metric(o, dst.double().cpu().numpy(), ref[k].double().cpu().numpy())
        assert err < 1e-5, (step, err)
        m, r = mom.cpu().numpy(), mref[k].cpu().numpy()
        assert np.allclose(m, r, rtol=1e-4, atol=1e-6 * (1 + np.abs(r).max())), step
        # and against the oracle's relaxation of the same input
        h_o, m_o = o.collide(src.double().cpu().numpy(), step=step)
        assert f_metric(o, dst.double().cpu().numpy(), h_o) < 1e-5, step
        assert np.allclose(m, m_o, rtol=1e-4, atol=1e-6 * (1 + np.abs(m_o).max())), step
        src = dst


@pytest.mark.gpu
def test_noalloc_size_limits():
    """A large sample set that still fits shared memory next to a 24^3 slab
    (40000 samples, FP32) runs and matches the oracle; 65536 samples (the
    scratch's maximum) next to a 32^3 slab do not fit and are refused with
    BZ_EUNSUPPORTED."""
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    import oracle
    from tests.gpu_helpers import f_metric

    torch.cuda.set_device(0)
    p = workloads.small(nx=3, ny=2, nv=24, vmax=4.5, nt=40000, seed=17, eps=0.1)
    o = oracle.Oracle(**p.kwargs())
    h0 = workloads.warm_state(p, seed=5).astype(np.float32)
    src = torch.from_numpy(h0).cuda()
    dst = torch.empty_like(src)
    mom = torch.empty((p.nr, 11), dtype=torch.float64, device="cuda")
    binding.collide_noalloc(p, 2, src, dst, mom)
    torch.cuda.synchronize()
    h_o, m_o = o.collide(h0.astype(np.float64), step=2)
    assert f_metric(o, dst.double().cpu().numpy(), h_o) < 1e-5
    assert np.allclose(mom.cpu().numpy(), m_o, rtol=1e-4, atol=1e-6 * (1 + np.abs(m_o).max()))

    q = workloads.small(nx=2, ny=2, nv=32, vmax=5.0, nt=binding.NOALLOC_MAX_PAIRS, seed=3, eps=0.1)
    a = torch.zeros((q.nr, q.nvt), dtype=torch.float32, device="cuda")
    b = torch.empty_like(a)
    with pytest.raises(binding.BzError) as e:
        binding.collide_noalloc(q, 0, a, b)
    assert e.value.status == binding.BZ_EUNSUPPORTED
