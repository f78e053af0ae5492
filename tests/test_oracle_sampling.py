"""Pins of the oracle's collision sampling (Eq. coll8Dim, Sec. 4.2)."""
import numpy as np

import oracle


def _o(**kw):
    args = dict(nx=1, ny=1, kn=1.0, nv=12, vmax=4.0, nt=20_000, seed=5, eps=0.1)
    args.update(kw)
    return oracle.Oracle(**args)


def test_kinematics_conserve_momentum_and_energy():
    """P2: v* + v1* = v + v1 and |v*|^2 + |v1*|^2 = |v|^2 + |v1|^2 exactly
    (the reading v_r = v1 - v of the post-collision map)."""
    s = _o().samples(3)
    e0 = (s["v"] ** 2).sum(1) + (s["v1"] ** 2).sum(1)
    e1 = (s["vs"] ** 2).sum(1) + (s["v1s"] ** 2).sum(1)
    assert np.max(np.abs(e1 - e0) / e0) < 1e-14
    assert np.max(np.abs(s["v"] + s["v1"] - s["vs"] - s["v1s"])) < 1e-14
    # |k . v_r| is preserved and the relative speed is preserved
    vr0 = s["v1"] - s["v"]
    vr1 = s["v1s"] - s["vs"]
    assert np.allclose(np.abs((vr0 * s["k"]).sum(1)), np.abs((vr1 * s["k"]).sum(1)), atol=1e-13)
    assert np.allclose((vr0 ** 2).sum(1), (vr1 ** 2).sum(1), rtol=1e-13)


def test_sampled_distributions():
    """v, v1 ~ Phi0 = pi^{-3/2} e^{-v^2} (variance 1/2 per component,
    E|v|^4 = 15/4) and k uniform on the unit sphere (E k_z^2 = 1/3)."""
    o = _o(nt=100_000)
    s = o.samples(0)
    n = s.size
    for key in ("v", "v1"):
        v = s[key]
        assert np.all(np.abs(v.mean(0)) < 5 * np.sqrt(0.5 / n))
        assert np.all(np.abs(v.var(0) - 0.5) < 5 * np.sqrt(0.5 / n))
        v4 = ((v ** 2).sum(1) ** 2).mean()
        assert abs(v4 - 15 / 4) < 0.1
    k = s["k"]
    assert np.max(np.abs((k ** 2).sum(1) - 1)) < 1e-14
    assert np.all(np.abs(k.mean(0)) < 5 * np.sqrt(1 / 3 / n))
    assert np.all(np.abs((k ** 2).mean(0) - 1 / 3) < 5 * np.sqrt(4 / 45 / n))
    # the two draws and the unit vector are independent of each other
    assert abs(np.corrcoef(s["v"][:, 0], s["v1"][:, 0])[0, 1]) < 5 / np.sqrt(n)
    assert abs(np.corrcoef(s["v"][:, 2], s["k"][:, 2])[0, 1]) < 5 / np.sqrt(n)
    # weight: pi K dt |s| / Nt
    cw = np.pi * oracle.K_HARD_SPHERE * o.dt / o.p.nt
    assert np.allclose(s["W"], cw * np.abs(s["s"]), rtol=1e-15)


def test_node_of_brute_force():
    o = _o(nv=7, vmax=3.0)
    dv = o.dv
    edges = -3.0 + dv * np.arange(8)
    rng = np.random.default_rng(1)
    for _ in range(2000):
        v = rng.uniform(-3.6, 3.6, size=3)
        j, _ = o.node_of(v)
        inside = np.all((v >= -3.0) & (v < 3.0))
        if not inside:
            assert j == -1
        else:
            ix, iy, iz = [int(np.searchsorted(edges, c, side="right") - 1) for c in v]
            assert j == (ix * 7 + iy) * 7 + iz
    assert o.node_of([-3.0, -3.0, -3.0])[0] == 0
    assert o.node_of([3.0, 0.0, 0.0])[0] == -1
    # a face value belongs to the upper cell
    j, near = o.node_of([edges[3], 0.1, 0.1])
    assert j // 49 == 3 and near == 1


def test_shared_and_per_cell_streams():
    o = _o(nt=64)
    a = o.samples(2)
    b = o.samples(2, cellword=0xFFFFFFFF)
    assert (a["idx"] == b["idx"]).all() and (a["v"] == b["v"]).all()
    c0 = o.samples(2, cellword=0)
    c1 = o.samples(2, cellword=1)
    assert not np.array_equal(c0["v"], c1["v"])
    d = o.samples(3)
    assert not np.array_equal(a["v"], d["v"])
