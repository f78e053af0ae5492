"""Golden fixtures: values the paper prints, and an oracle regression case."""
import os

import numpy as np

import oracle

HERE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def _paper_values():
    out = {}
    for line in open(os.path.join(HERE, "paper_values.txt")):
        if line.startswith("#") or not line.strip():
            continue
        name, val = line.split()[:2]
        out[name] = float(val)
    return out


def test_cfl_of_the_paper_gives_the_time_step():
    v = _paper_values()
    o = oracle.Oracle(nx=16, ny=16, kn=1.0, nv=12, vmax=4.0, nt=1, seed=1, cfl=v["cfl_max"])
    vtop = o.node_v()[-1]
    assert abs(vtop * o.dt / o.dx - v["cfl_max"]) < 1e-15


def test_collision_constant_uses_the_viscosity_factor():
    v = _paper_values()
    K = 5.0 * v["hs_viscosity_factor"] / 16.0 * np.sqrt(2.0 / np.pi)
    assert abs(K - oracle.K_HARD_SPHERE) < 1e-15


def test_oracle_regression_fixture():
    import sys
    sys.path.insert(0, HERE)
    import make_golden
    ref = np.load(os.path.join(HERE, "tiny_cavity.npz"))
    h0, h, mom = make_golden.make()
    assert np.array_equal(h0, ref["h0"])
    assert np.allclose(h, ref["h3"], rtol=1e-12, atol=1e-13)
    assert np.allclose(mom, ref["mom3"], rtol=1e-12, atol=1e-13)
