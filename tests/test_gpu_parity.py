"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

Tolerances: node selection is integer work and must agree exactly, with no
exception (both sides flag samples whose velocity lies within 1e-9 dv of a
cell face, where an ulp of difference between libm and CUDA's log/cos/sin
could move a node; none may differ either).  Floating point: max |f_gpu -
f_oracle| / max f <= 1e-5 per step with f = Phi0 (1 + eps h), the oracle
restarted from the GPU's state before every step (so the bound does not grow
with the step count); macroscopic fields within 1e-4 of their range after
200 steps of both sides running on their own.
"""
import os
import subprocess
import tempfile
import ctypes as C

import numpy as np
import pytest

import oracle
from paper_1005_5405_gb300 import binding, workloads
from tests.gpu_helpers import f_metric, make, state

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    torch.cuda.set_device(0)
    yield


# ---------------------------------------------------------------- Philox
def test_device_philox_matches_oracle():
    rng = np.random.default_rng(1)
    ctr = rng.integers(0, 2 ** 32, size=(20000, 4), dtype=np.uint64).astype(np.uint32)
    ctr[:16] = np.arange(64).reshape(16, 4)
    for key in [(0, 0), (1, 2), (0xDEADBEEF, 0x12345678)]:
        dev = binding.philox(key, ctr)
        ref = np.array([oracle.philox(c, key) for c in ctr[:4000]], dtype=np.uint32)
        assert np.array_equal(dev[:4000], ref)


def test_device_philox_matches_curand():
    """Cross-check against cuRAND's Philox4x32-10 device function."""
    nvcc = "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not available")
    d = tempfile.mkdtemp()
    so = os.path.join(d, "curand_ref.so")
    subprocess.run([nvcc, "-gencode=arch=compute_103a,code=sm_103a", "-shared", "-Xcompiler",
                    "-fPIC", "-cudart", "shared", "-o", so, os.path.join(HERE, "_curand_ref.cu")],
                   check=True)
    L = C.CDLL(so)
    rng = np.random.default_rng(2)
    ctr = rng.integers(0, 2 ** 32, size=(50000, 4), dtype=np.uint64).astype(np.uint32)
    for key in [(7, 9), (0xFFFFFFFF, 0), (3, 0xCAFEF00D)]:
        out = np.zeros_like(ctr)
        assert L.curand_philox_ref(C.c_uint32(key[0]), C.c_uint32(key[1]),
                                   C.c_void_p(ctr.ctypes.data), C.c_int(len(ctr)),
                                   C.c_void_p(out.ctypes.data)) == 0
        assert np.array_equal(out, binding.philox(key, ctr))
        ref = np.array([oracle.philox(c, key) for c in ctr[:2000]], dtype=np.uint32)
        assert np.array_equal(out[:2000], ref)


# ---------------------------------------------------------------- sampling
@pytest.mark.parametrize("nv,vmax,nt,dtype", [(12, 4.0, 1000, "f64"), (24, 4.5, 10000, "f32"),
                                              (32, 5.0, 20000, "f32"), (8, 2.0, 5000, "f32")])
def test_sample_plan_matches_oracle(nv, vmax, nt, dtype):
    p = workloads.small(nx=2, ny=2, nv=nv, vmax=vmax, nt=nt, seed=3, dtype=dtype)
    cav = binding.Cavity(p)
    o = oracle.Oracle(**p.kwargs())
    flagged = 0
    for step in (0, 1, 57):
        idx, W = cav.sample_plan(step)
        s = o.samples(step)
        same = (idx == s["idx"]).all(1)
        flagged += int((s["near_face"] != 0).sum())
        assert same.all(), (np.nonzero(~same), s["near_face"][~same])
        # s = v_r.k suffers cancellation, so ulp-level differences of libm and
        # CUDA cos/sin/log show up relative to the largest weight only
        assert np.max(np.abs(W - s["W"])) <= 1e-12 * np.max(s["W"])
    print(f"node selection: 0 mismatches in {3 * nt} samples, {flagged} near a face")


# ---------------------------------------------------------------- sub-steps
CASES = [
    workloads.small(nx=6, ny=5, nv=12, vmax=4.0, nt=1000, seed=1, dtype="f64"),
    workloads.small(nx=6, ny=5, nv=12, vmax=4.0, nt=3000, seed=2, dtype="f32"),
    workloads.small(nx=7, ny=3, nv=16, vmax=4.0, nt=4000, seed=3, dtype="f32", lid_u0=0.2),
    workloads.small(nx=1, ny=1, nv=10, vmax=4.0, nt=2000, seed=4, dtype="f32"),
    workloads.small(nx=4, ny=4, nv=5, vmax=3.0, nt=700, seed=5, dtype="f32"),
    workloads.small(nx=3, ny=4, nv=24, vmax=4.5, nt=10000, seed=6, dtype="f32", kn=0.1),
    workloads.small(nx=3, ny=3, nv=8, vmax=2.0, nt=3000, seed=7, dtype="f32"),  # many out-of-box
]
IDS = ["f64_12", "f32_12", "f32_16_rect", "single_cell", "odd_nv5", "f32_24", "outbox"]


@pytest.mark.parametrize("p", CASES, ids=IDS)
def test_stream_matches_oracle(p):
    cav, o, h0 = make(p)
    cav.step_ex(1, binding.BZ_DO_STREAM)
    assert f_metric(o, state(cav), o.stream(h0, 0)) < 1e-6


@pytest.mark.parametrize("p", CASES, ids=IDS)
def test_collide_matches_oracle(p, kernel):
    cav, o, h0 = make(p)
    cav.step_ex(1, binding.BZ_DO_COLLIDE)
    h_o, mom_o = o.collide(h0, step=0)
    assert f_metric(o, state(cav), h_o) < 1e-5
    mom_g = cav.moments().cpu().numpy()
    assert np.allclose(mom_g, mom_o, rtol=1e-4, atol=1e-6 * (1 + np.abs(mom_o).max()))


@pytest.fixture(params=["auto", "ordered", "ordered_g2", "unordered", "joint_tail", "overflow", "tma",
                        "tma_ordered", "cell4", "t512", "generic"])
def kernel(request, monkeypatch):
    """Run a test with the library's own choice of per-cell kernel (the FP32
    active-node kernel with deferred correction where it applies); with that
    kernel's term runs in the joint bank-aware order (forced on, in chunks of
    16 or 24 positions, for groups of four cells and of two), and with no
    order; with the increment sums after a CTA barrier instead of started
    early by the collision warps (the default below 32^3 velocities); with
    that kernel's compact arrays capped below the step's
    active-node count (every step then takes the k_cell4 fallback on the
    device); with the streaming sources brought in by bulk copies (TMA) on
    mbarriers, with and without the term order; with the FP32 4-node-vector kernel (BZ_KERNEL=cell4) in its
    1024- and 512-thread shapes; and with the generic kernel."""
    for k in ("BZ_KERNEL", "BZ_CELL_THREADS", "BZ_LAZY_MCAP", "BZ_LAZY_ORDER", "BZ_LAZY_NOORDER",
              "BZ_LAZY_ORDER_CHUNK", "BZ_LAZY_G", "BZ_LAZY_EARLY_TAIL", "BZ_LAZY_TMA"):
        monkeypatch.delenv(k, raising=False)
    if request.param in ("tma", "tma_ordered"):
        monkeypatch.setenv("BZ_LAZY_TMA", "1")
    if request.param == "tma_ordered":
        monkeypatch.setenv("BZ_LAZY_ORDER", "1")
        monkeypatch.setenv("BZ_LAZY_ORDER_CHUNK", "16")
    if request.param == "joint_tail":
        monkeypatch.setenv("BZ_LAZY_EARLY_TAIL", "0")
    if request.param == "ordered":
        monkeypatch.setenv("BZ_LAZY_ORDER", "1")
        monkeypatch.setenv("BZ_LAZY_ORDER_CHUNK", "16")
    elif request.param == "ordered_g2":
        monkeypatch.setenv("BZ_LAZY_ORDER", "1")
        monkeypatch.setenv("BZ_LAZY_ORDER_CHUNK", "24")
        monkeypatch.setenv("BZ_LAZY_G", "2")
    elif request.param == "unordered":
        monkeypatch.setenv("BZ_LAZY_NOORDER", "1")
    if request.param == "generic":
        monkeypatch.setenv("BZ_KERNEL", "generic")
    elif request.param == "cell4":
        monkeypatch.setenv("BZ_KERNEL", "cell4")
    elif request.param == "t512":
        monkeypatch.setenv("BZ_KERNEL", "cell4")
        monkeypatch.setenv("BZ_CELL_THREADS", "512")
    elif request.param == "overflow":
        monkeypatch.setenv("BZ_LAZY_MCAP", "8")
    return request.param


@pytest.mark.parametrize("p", CASES, ids=IDS)
def test_fused_step_matches_oracle(p, kernel):
    cav, o, h0 = make(p)
    if kernel == "generic":
        assert cav.get_info().kernel_variant == 0
    if kernel in ("cell4", "t512"):
        assert cav.get_info().kernel_variant in (0, 1)
    h_g = h0
    for n in range(3):
        cav.step(1)
        h_o, mom_o = o.step(h_g, n)           # the oracle restarts from the GPU state
        h_g = state(cav)
        assert f_metric(o, h_g, h_o) < 1e-5, n
    mom_g = cav.moments().cpu().numpy()
    assert np.allclose(mom_g, mom_o, rtol=1e-4, atol=1e-5 * (1 + np.abs(mom_o).max()))


def test_split_path_matches_fused_path():
    p = CASES[2]
    a, o, h0 = make(p)
    b, _, _ = make(p)
    a.step(2)
    b.step_ex(2, binding.BZ_SPLIT)
    assert f_metric(o, state(a), state(b)) < 1e-6


def test_graph_replay_matches_plain_launches(monkeypatch):
    """bz_step replays a captured two-step CUDA graph (the kernels read the
    step number from device memory); the result must equal plain launches,
    also across an odd step count, a lid change and a state reset."""
    p = CASES[2]
    monkeypatch.setenv("BZ_GRAPH", "0")
    a, o, h0 = make(p)
    a.step(5)
    a.set_lid(0.05)
    a.step(3)
    monkeypatch.delenv("BZ_GRAPH")
    b, _, _ = make(p)
    b.step(5)
    b.set_lid(0.05)
    b.step(3)
    assert a.get_state()[1] == b.get_state()[1] == 8
    assert f_metric(o, state(a), state(b)) < 1e-6
    st = b.stats()
    assert st[0] == 8
    b.set_state(h0.astype(np.float32), step=0)
    b.step(4)
    c, _, _ = make(p)
    c.set_lid(0.05)
    monkeypatch.setenv("BZ_GRAPH", "0")
    c.step(4)
    assert f_metric(o, state(b), state(c)) < 1e-6


def test_gw_in_global_scratch_path():
    """Enough samples that the per-sample products do not fit in shared
    memory next to a 32^3 slab: the kernel keeps them in global scratch."""
    p = workloads.small(nx=2, ny=2, nv=32, vmax=5.0, nt=40000, seed=9)
    cav, o, h0 = make(p)
    cav.step(1)
    h_o, _ = o.step(h0, 0)
    assert f_metric(o, state(cav), h_o) < 1e-5


def test_zero_state_stays_at_rest():
    p = workloads.small(nx=4, ny=4, nv=12, vmax=4.0, nt=2000, seed=1, lid_u0=0.0)
    cav, o, h0 = make(p, h0=np.zeros((16, 12 ** 3)))
    cav.step(5)
    assert np.max(np.abs(state(cav))) < 1e-10


def test_200_steps_fp64_cavity16_v12():
    """16x16 cavity, 12^3 velocities, FP64 state: macroscopic fields after 200
    steps from rest (the lid drives the flow)."""
    p = workloads.cavity16_v12()
    cav, o, h0 = make(p, h0=np.zeros((p.nr, p.nvt)))
    cav.step(200)
    h_o, mom_o = o.run(h0, 200)
    mom_g = cav.moments().cpu().numpy()
    for k in range(5):
        rng_ = np.abs(mom_o[:, k]).max()
        assert np.max(np.abs(mom_g[:, k] - mom_o[:, k])) <= 1e-4 * rng_, k
    assert f_metric(o, state(cav), h_o) < 1e-9


def test_200_steps_fp32_v24():
    """FP32 state, 24^3 velocities on [-4.5, 4.5]^3, 10^4 samples, with the cell
    size and time step of the 64x64 Kn 0.1 cavity (8x8 cells of side 10/64)."""
    p = workloads.small(nx=8, ny=8, nv=24, vmax=4.5, nt=10000, seed=2, kn=1.0 / (8 * 10.0 / 64))
    cav, o, h0 = make(p, h0=np.zeros((p.nr, p.nvt)))
    cav.step(200)
    h_o, mom_o = o.run(h0, 200)
    mom_g = cav.moments().cpu().numpy()
    for k in range(5):
        rng_ = np.abs(mom_o[:, k]).max()
        assert np.max(np.abs(mom_g[:, k] - mom_o[:, k])) <= 1e-4 * rng_, k


@pytest.mark.parametrize("nv,vmax,nt,nxy,kn,order,tma", [(32, 5.0, 20000, 12, 0.05 * 256 / 12, "1", "0"),
                                                          (32, 5.0, 20000, 12, 0.05 * 256 / 12, "1", "1"),
                                                          (24, 4.5, 10000, 8, 0.1 * 64 / 8, None, "0")],
                         ids=["v32_ordered", "v32_ordered_tma", "v24"])
def test_200_steps_warm_start_hot_path(monkeypatch, nv, vmax, nt, nxy, kn, order, tma):
    """The benchmark's path (FP32 active-node kernel with deferred correction;
    at 32^3 with the joint bank-aware term order forced on) run for 200 steps
    from a seeded warm state, so the collision integral is non-zero from the
    first step, against the oracle running the same 200 steps on its own:
    density, velocity and temperature within 1e-4 of their range.  The cells
    have the size of the 256^2 (32^3) and 64^2 (24^3) cavities."""
    if order:
        monkeypatch.setenv("BZ_LAZY_ORDER", order)
    monkeypatch.setenv("BZ_LAZY_TMA", tma)
    p = workloads.small(nx=nxy, ny=nxy, nv=nv, vmax=vmax, nt=nt, seed=3, kn=kn, lid_u0=0.0,
                        lid_amp=0.05, lid_period=50.0)
    cav, o, h0 = make(p, seed=7)
    assert cav.get_info().kernel_variant == 2
    cav.step(200)
    h_o, mom_o = o.run(h0, 200)
    mom_g = cav.moments().cpu().numpy()
    for k in range(5):
        rng_ = np.abs(mom_o[:, k]).max()
        err = np.max(np.abs(mom_g[:, k] - mom_o[:, k])) / rng_
        print(f"moment {k}: {err:.2e} of its range after 200 steps")
        assert err <= 1e-4, k
    st = cav.stats()
    assert st[5] == 0          # no step overflowed the compact arrays


def _lz_traversal(nx, ny, G, grid, b):
    """Cells the active-node kernel's CTA b visits, in order: groups b, b +
    grid, ... of G cells in the column-strip cell order (strips of 8 columns,
    row by row inside a strip)."""
    S = 8 if nx >= 16 else nx
    full = nx // S

    def cell_of(k):
        if k < full * S * ny:
            s_, r = divmod(k, S * ny)
            return (r // S) * nx + s_ * S + r % S
        R = nx - full * S
        kk = k - full * S * ny
        return (kk // R) * nx + full * S + kk % R

    nr = nx * ny
    ngroups = (nr + G - 1) // G
    return [cell_of(grp * G + t) for grp in range(b, ngroups, grid) for t in range(G)
            if grp * G + t < nr]


def test_full_size_cavity256_v32_sampled_cells():
    """256x256 cells x 32^3 velocities, FP32, 2x10^4 samples: the launch
    configuration of the benchmark.  One step from a seeded warm state; the
    oracle recomputes, one by one from their input slabs, every cell of the
    lid row and of the left wall column, and every cell that the first and the
    last CTA of the active-node kernel visit (one CTA per SM)."""
    import torch
    from concurrent.futures import ThreadPoolExecutor
    p = workloads.cavity256_v32()
    rng = np.random.default_rng(7)
    coef = torch.from_numpy(0.3 * rng.standard_normal((p.nr, 6)).astype(np.float32)).cuda()
    a = torch.from_numpy(workloads.axis_nodes(p.nv, p.vmax).astype(np.float32)).cuda()
    vx, vy, vz = torch.meshgrid(a, a, a, indexing="ij")
    vx, vy, vz = vx.reshape(-1), vy.reshape(-1), vz.reshape(-1)
    basis = torch.stack([torch.ones_like(vx), vx, vy, vz, vx * vx + vy * vy + vz * vz - 1.5,
                         vx * vy])
    h0 = coef @ basis
    g = torch.Generator(device="cuda").manual_seed(7)
    h0 += 0.01 * torch.randn(h0.shape, generator=g, device="cuda")
    cav = binding.Cavity(p)
    assert cav.get_info().kernel_variant == 2
    cav.set_state(h0, step=3)
    cav.step(1)
    out, step = cav.get_state()
    assert step == 4
    mom = cav.moments().cpu().numpy()
    o = oracle.Oracle(**p.kwargs())
    nx, ny = p.nx, p.ny
    nsm = torch.cuda.get_device_properties(0).multi_processor_count
    grid = min((p.nr + 3) // 4, nsm)
    cells = set(range((ny - 1) * nx, ny * nx)) | set(range(0, nx * ny, nx))
    cells |= set(_lz_traversal(nx, ny, 4, grid, 0)) | set(_lz_traversal(nx, ny, 4, grid, grid - 1))
    cells = sorted(cells)
    need = sorted({cc for c in cells for cc in (c, c - 1, c + 1, c - nx, c + nx) if 0 <= cc < p.nr})
    pos = {cc: i for i, cc in enumerate(need)}
    slabs = h0[torch.tensor(need, device="cuda")].double().cpu().numpy()
    got_all = out[torch.tensor(cells, device="cuda")].double().cpu().numpy()

    def one(c):
        ix, iy = c % nx, c // nx
        sl = lambda cc: slabs[pos[cc]]
        return o.step_cell(c, sl(c), sl(c - 1) if ix > 0 else None,
                           sl(c + 1) if ix < nx - 1 else None, sl(c - nx) if iy > 0 else None,
                           sl(c + nx) if iy < ny - 1 else None, step=3)

    with ThreadPoolExecutor(max_workers=min(32, os.cpu_count() or 4)) as ex:
        refs = list(ex.map(one, cells))
    worst = 0.0
    for k, (c, (ref, m)) in enumerate(zip(cells, refs)):
        err = f_metric(o, got_all[k], ref)
        worst = max(worst, err)
        assert err < 1e-5, c
        assert np.allclose(mom[c], m, rtol=1e-4, atol=1e-5 * (1 + np.abs(m).max())), c
    print(f"full-size step: {len(cells)} cells checked, worst f error {worst:.2e}")


# ---------------------------------------------------------------- API
def test_moments_of_arbitrary_state():
    p = CASES[1]
    cav, o, h0 = make(p)
    assert np.allclose(cav.moments().cpu().numpy(), o.moments(h0), rtol=1e-5, atol=1e-6)


def test_lid_shear_matches_oracle():
    p = CASES[2]
    cav, o, h0 = make(p)
    d = cav.lid_shear().cpu().numpy()
    ref = o.lid_shear(h0, 0)
    assert np.allclose(d, ref, rtol=1e-5, atol=1e-6 * np.abs(ref).max())


def test_checkpoint_resume():
    p = CASES[1]
    a, o, h0 = make(p)
    a.step(4)
    b, _, _ = make(p)
    b.step(2)
    snap, st = b.get_state()
    c = binding.Cavity(p)
    c.set_state(snap.clone(), step=st)
    c.step(2)
    assert f_metric(o, state(a), state(c)) < 1e-6


def test_fast_kernel_is_selected_for_fp32_quads(monkeypatch):
    for nv, expect in ((32, 2), (24, 2), (16, 2), (12, 2), (10, 0), (8, 0)):
        p = workloads.small(nx=2, ny=2, nv=nv, vmax=4.0, nt=2000)
        assert binding.Cavity(p).get_info().kernel_variant == expect, nv
    assert binding.Cavity(workloads.small(nv=12, dtype="f64")).get_info().kernel_variant == 0
    monkeypatch.setenv("BZ_KERNEL", "cell4")
    assert binding.Cavity(workloads.small(nv=16, nt=2000)).get_info().kernel_variant == 1


def test_deferred_correction_is_applied_by_every_reader():
    """After steps on the active-node path the stored state carries pending
    corrections: the lid shear, the moments, a state copy, a split step and
    a restart from a copied state must all see the corrected state."""
    p = workloads.small(nx=6, ny=5, nv=16, vmax=4.0, nt=3000, seed=11, dtype="f32", eps=0.1,
                        lid_u0=0.1)
    cav, o, h0 = make(p)
    assert cav.get_info().kernel_variant == 2
    # cav takes three steps, each reading the pending corrections its
    # predecessor left; ref takes the same steps with its state read (and so
    # corrected in place) after two, and the oracle takes the third step
    # from that state.
    ref_cav, _, _ = make(p)
    ref_cav.step(2)
    h2 = state(ref_cav)
    ref_cav.step(1)
    cav.step(3)
    assert f_metric(o, state(ref_cav), state(cav)) < 1e-6
    cav, _, _ = make(p)
    cav.step(3)
    h_o, mom_o = o.step(h2, 2)
    d = cav.lid_shear().cpu().numpy()
    ref = o.lid_shear(h_o, 3)
    assert np.allclose(d, ref, rtol=1e-4, atol=1e-5 * np.abs(ref).max())
    mom = cav.moments().cpu().numpy()
    assert np.allclose(mom, mom_o, rtol=1e-4, atol=1e-5 * (1 + np.abs(mom_o).max()))
    h_g = state(cav)
    assert f_metric(o, h_g, h_o) < 1e-5
    # a split step after lazy steps, then fused steps again
    cav.step_ex(1, binding.BZ_SPLIT)
    h_o, _ = o.step(h_g, 3)
    h_g = state(cav)
    assert f_metric(o, h_g, h_o) < 1e-5
    cav.step(1)
    h4 = state(cav)
    cav.step(1)
    h_o, mom_o = o.step(h4, 5)
    snap, st = cav.get_state()
    assert st == 6 and f_metric(o, snap.double().cpu().numpy(), h_o) < 1e-5
    c2 = binding.Cavity(p)
    c2.set_state(snap.clone(), step=st)
    c2.step(1)
    cav.step(1)
    assert f_metric(o, state(c2), state(cav)) < 1e-6


def test_stats_and_info():
    p = CASES[6]
    cav, o, h0 = make(p)
    cav.step(3)
    st = cav.stats()
    assert st[0] == 3 and st[1] > 0 and st[4] >= 9
    info = cav.get_info()
    assert abs(info.dt - o.dt) <= 1e-15 * o.dt and info.nodes == p.nodes


def test_errors_are_reported():
    with pytest.raises(binding.BzError) as e:
        binding.Cavity(workloads.small(nv=48, vmax=5.0))      # 48^3 slab > shared memory
    assert e.value.status == binding.BZ_EUNSUPPORTED
    with pytest.raises(binding.BzError) as e:
        binding.Cavity(workloads.small(nt=0))
    assert e.value.status == binding.BZ_EINVAL
    cav = binding.Cavity(workloads.small())
    os.environ["BZ_FAULT"] = "launch"
    try:
        with pytest.raises(binding.BzError) as e:
            cav.step(1)
        assert e.value.status == binding.BZ_ECUDA
    finally:
        del os.environ["BZ_FAULT"]
    cav.step(1)



@pytest.mark.parametrize("kernel_env", [None, "cell4", "generic"])
def test_handles_of_different_sizes_coexist(monkeypatch, kernel_env):
    """Kernel attributes (the dynamic shared-memory limit) are shared by all
    handles of the process: creating a handle that needs less shared memory
    must not break the launches of one created before it."""
    if kernel_env:
        monkeypatch.setenv("BZ_KERNEL", kernel_env)
    probs = [workloads.small(nx=3, ny=3, nv=nv, vmax=4.0, nt=1500, seed=40 + nv, dtype="f32",
                             eps=0.1) for nv in (24, 16, 12)]
    made = [make(p) for p in probs]             # all created before any step
    for (cav, o, h0), p in zip(made, probs):
        cav.step(1)
        h_o, _ = o.step(h0, 0)
        assert f_metric(o, state(cav), h_o) < 1e-5, p.nv


@pytest.mark.parametrize("order", ["1", "0"])
def test_plans_built_ahead_match_the_per_step_chain(monkeypatch, order):
    """The sample plans built ahead in slots (BZ_LAZY_AHEAD=K, several steps
    per launch) give the steps of the per-step chain (BZ_LAZY_AHEAD=0): the
    same states to FP32 rounding (the term order runs over whole runs rather
    than chunks), the same counters of out-of-box and near-face samples,
    overflows and active nodes, across batch boundaries (K = 3), odd step
    counts (graph pairs and single steps) and a jump of the step counter."""
    for k in ("BZ_KERNEL", "BZ_LAZY_MCAP", "BZ_LAZY_ORDER", "BZ_LAZY_NOORDER", "BZ_LAZY_ORDER_CHUNK",
              "BZ_LAZY_G", "BZ_LAZY_TMA"):
        monkeypatch.delenv(k, raising=False)
    monkeypatch.setenv("BZ_LAZY_ORDER" if order == "1" else "BZ_LAZY_NOORDER", "1")
    p = workloads.small(nx=12, ny=12, nv=32, vmax=5.0, nt=20000, seed=3, kn=0.05 * 256 / 12,
                        lid_u0=0.0, lid_amp=0.05, lid_period=50.0)
    h0 = workloads.warm_state(p, seed=17).astype(np.float32)
    o = oracle.Oracle(**p.kwargs())
    runs = {}
    for K in ("0", "3"):
        monkeypatch.setenv("BZ_LAZY_AHEAD", K)
        cav = binding.Cavity(p)
        assert cav.get_info().kernel_variant == 2
        cav.set_state(h0, step=0)
        cav.step(5)
        cav.step(2)
        cav.step_ex(1, binding.BZ_DO_COLLIDE)
        mid = state(cav)
        cav.set_state(mid.astype(np.float32), step=100)
        cav.step(4)
        runs[K] = (state(cav), cav.stats())
    (ha, sa), (hb, sb) = runs["0"], runs["3"]
    assert f_metric(o, hb, ha) < 1e-6
    assert sa[0] == sb[0] == 104
    assert [sa[i] for i in (1, 2, 5, 6)] == [sb[i] for i in (1, 2, 5, 6)]
