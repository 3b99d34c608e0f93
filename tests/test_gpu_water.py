"""Water (Sec. "Water") on the GPU against the FP64 oracle: unload fields, base
stretches, energy, gradient and HVP of a water / solid mixture (norm-relative 1e-5
in FP32, 1e-10 in FP64), and positions plus particle J after ten implicit steps of
a small dam break with a solid cube in the flow (1e-4 dx; J to 1e-5 / 1e-10)."""
import numpy as np
import pytest
import torch

import paper_2602_07853_gb300.mpml as m
from paper_2602_07853_gb300 import scenes
from tests._util import make_oracle
from tests._gpu import GpuSim, OracleSim, check

pytestmark = pytest.mark.gpu

TOL = {m.FP32: 1e-5, m.FP64: 1e-10}


@pytest.fixture(autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.set_device(0)


def mixed_scene(seed=31, n=16, count=5000):
    rng = np.random.default_rng(seed)
    sc = scenes.Scene("water_mix", (n, n, n), 1.0 / n, float(n), 1e-3, (0.0, -9.8, 0.0),
                      [scenes.Material(scenes.WATER, 1e5, 0.45),
                       scenes.Material(scenes.FIXED_COROTATED, 1e5, 0.3, rho=500.0)])
    x = rng.uniform(1.6 / n, 1 - 1.6 / n, (count, 3))
    mat = rng.integers(0, 2, count).astype(np.int64)
    sc = scenes._finish(sc, x, 0.2 * rng.standard_normal((count, 3)), mat, 8)
    J = rng.uniform(0.9, 1.1, count)
    for p in range(count):
        sc.F[p] = np.cbrt(J[p]) * np.eye(3) if mat[p] == 0 else np.eye(3) + 0.03 * rng.standard_normal((3, 3))
    sc.G = 0.5 * rng.standard_normal((count, 3, 3))
    return sc


@pytest.mark.parametrize("precision", [m.FP32, m.FP64])
def test_water_mixture_fields_energy_gradient_hvp(precision):
    sc = mixed_scene()
    g = GpuSim(sc, precision)
    inp = g.inputs()
    g.set_particles()
    o = make_oracle(sc)
    assert o.unload(**inp) == 0
    g.resample()
    tol = TOL[precision]
    for f, name in [(m.F_CELL_VOL, "V_ck"), (m.F_CELL_TAU, "tau_ck"), (m.F_NODE_MASS, "m_i"), (m.F_NODE_VEL, "v_i")]:
        check(g.field(f), o.field(name), tol, name)
    assert o.stretch() == 0
    m.mpml_stretch(g.ctx)
    V = o.field("V_ck")
    mask = V > 0
    S_g, S_o = g.field(m.F_CELL_STRETCH), o.field("S_ck")
    check(S_g[mask] - np.eye(3), S_o[mask] - np.eye(3), tol, 'S - I')
    # water slots are isotropic
    Sw = S_o[:, 0][mask[:, 0]]
    assert np.allclose(Sw, np.eye(3) * Sw[:, :1, :1], atol=1e-14)
    nn = o.count("nodes")
    rng = np.random.default_rng(32)
    v = (o.field("vhat") + 0.05 * rng.standard_normal((nn, 3))).astype(g.npdt).astype(np.float64)
    phi_o, g_o = o.eval(v)
    phi_g, g_g = m.mpml_eval(g.ctx, v)
    assert abs(phi_g - phi_o) <= tol * abs(phi_o)
    check(g_g, g_o, tol, 'gradient')
    o.linearize(v, project=True)
    p = rng.standard_normal((nn, 3)).astype(g.npdt).astype(np.float64)
    check(m.mpml_hvp(g.ctx, p), o.hvp(p), tol, 'hvp')
    g.close()


@pytest.mark.parametrize("precision", [m.FP64, m.FP32])
def test_dam_break_ten_steps(precision):
    sc = scenes.dam_break(32)
    g = GpuSim(sc, precision)
    g.set_particles()
    o = OracleSim(make_oracle(sc), g.inputs())
    for s in range(10):
        rc, _ = o.step(s * sc.dt)
        assert rc >= 0
        rc_g, _ = g.step(s * sc.dt)
        assert rc_g >= 0
    got, p_o = g.particles_by_identity(), o.particles_by_identity()
    err = np.abs(got["x"] - p_o["x"]).max()
    assert err <= 1e-4 * sc.dx, err
    water = p_o["mat"] == 0
    Fg = got["F"].reshape(-1, 3, 3)[water]
    Fo = p_o["F"].reshape(-1, 3, 3)[water]
    Jg, Jo = np.linalg.det(Fg), np.linalg.det(Fo)
    assert np.abs(Jg - Jo).max() <= 10 * TOL[precision], np.abs(Jg - Jo).max()
    assert np.allclose(Fg, np.cbrt(Jg)[:, None, None] * np.eye(3), atol=10 * TOL[precision])
    assert np.any(np.abs(Jo - 1) > 1e-4)  # the column compresses under gravity
    g.close()
