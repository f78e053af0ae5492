"""Host logic of bench.py that needs no GPU: the kernel source hash and the
DRAM traffic it takes from the committed ncu summaries."""
import os

import bench


def test_source_hash_is_stable_and_covers_every_header():
    files = bench.CELL_KERNELS[2][2]
    h = bench.kernel_source_hash(files)
    assert h == bench.kernel_source_hash(files)
    assert len(h) == 16 and int(h, 16) >= 0
    # Each header of the list changes the hash.
    for k in range(len(files)):
        assert bench.kernel_source_hash(files[:k] + files[k + 1:]) != h


def _summary_values(name):
    vals = {}
    with open(os.path.join(bench.ROOT, "profiles", name)) as f:
        for line in f:
            if ":" in line and not line.startswith("#"):
                k, v = line.split(":", 1)
                vals[k.strip()] = v.strip().split()[0] if v.strip() else ""
    return vals


def test_profile_summary_of_the_active_node_kernel_is_complete():
    """The summary bench.py reads holds the fields it uses, and its traffic
    per cell lies between the algorithmic bytes per cell and twice that."""
    vals = _summary_values(bench.CELL_KERNELS[2][1])
    for key in ("source_hash", "workload_cells", "duration_ms", "dram_bytes_per_cell",
                "algorithmic_bytes_per_launch"):
        assert key in vals, key
    cells = int(vals["workload_cells"])
    per_cell = float(vals["dram_bytes_per_cell"])
    algo_per_cell = float(vals["algorithmic_bytes_per_launch"]) / cells
    assert algo_per_cell <= per_cell <= 2 * algo_per_cell


def test_profiled_traffic_scales_with_cells_or_is_withheld():
    """Traffic is the summary's bytes per cell times the cells, and is
    withheld (None) when the kernel headers changed after the capture or the
    kernel has no summary."""
    vals = _summary_values(bench.CELL_KERNELS[2][1])
    t1 = bench.profiled_traffic(1000, 2)
    t2 = bench.profiled_traffic(4000, 2)
    if vals["source_hash"] == bench.kernel_source_hash(bench.CELL_KERNELS[2][2]):
        assert t1 == float(vals["dram_bytes_per_cell"]) * 1000
        assert t2 == 4 * t1
    else:
        assert t1 is None and t2 is None
    assert bench.profiled_traffic(1000, 0) is None


class _FakeCavity:
    """Stands in for binding.Cavity: a plan batch of K steps built by the
    first step outside the last batch (pairs of steps, as the library's
    two-step graphs take them, never straddle one when K is even)."""

    def __init__(self, K, step=0):
        self.K, self.cur, self.lo, self.hi, self.builds = K, step, 0, 0, []

    def get_info(self):
        class I:
            pass
        i = I()
        i.plan_batch, i.step, i.plan_end = self.K, self.cur, self.hi if self.K else 0
        return i

    def step(self, n):
        k = 0
        while k < n:
            cnt = 2 if n - k >= 2 else 1
            if self.K and not (self.lo <= self.cur and self.cur + cnt <= self.hi):
                self.lo, self.hi = self.cur, self.cur + self.K
                self.builds.append(self.cur)
            self.cur += cnt
            k += cnt


def test_timed_window_starts_with_a_plan_batch():
    """After the warm-up, bench.to_plan_boundary runs the steps left in the
    current batch, so a timed window of S steps holds ceil(S / K) batch
    builds (S a multiple of K: exactly S / K, its share), for any warm-up."""
    for K in (46, 32):
        for warmup in (1, 5, 17, 46, 50):
            cav = _FakeCavity(K)
            cav.step(warmup)
            extra = bench.to_plan_boundary(cav)
            start = cav.cur
            assert start % K == 0 and extra == start - warmup
            for S in (2 * K, 40, 92):
                c2 = _FakeCavity(K)
                c2.step(start)
                n0 = len(c2.builds)
                c2.step(S)
                assert len(c2.builds) - n0 == -(-S // K), (K, warmup, S)
    # Without plans built ahead nothing is added.
    cav = _FakeCavity(0)
    cav.step(5)
    assert bench.to_plan_boundary(cav) == 0 and cav.cur == 5
