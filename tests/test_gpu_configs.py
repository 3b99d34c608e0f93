"""CUDA path vs the FP64 oracle on the other workload shapes: the stiff block
pressed by a moving Dirichlet plate (fixed-corotated, E = 1e8), a Hencky cube,
and the two-sphere collision in FP32 against the FP64 path.

Tolerances as in test_gpu_parity: positions within 1e-4 dx of the oracle after
the stated number of steps; FP32 against FP64 fields <= 1e-5 (one step).
"""
import numpy as np
import pytest
import torch

import paper_2602_07853_gb300.mpml as m
from paper_2602_07853_gb300 import scenes
from tests._util import make_oracle
from tests._gpu import GpuSim, OracleSim, check

pytestmark = pytest.mark.gpu


@pytest.fixture(autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.set_device(0)


def run_steps(sc, precision, steps):
    """Both sides step the scene; particles returned by identity (see by_identity)."""
    g = GpuSim(sc, precision)
    g.set_particles()
    o = OracleSim(make_oracle(sc), g.inputs())
    newton = []
    for s in range(steps):
        rc, st_o = o.step(s * sc.dt)
        assert rc >= 0
        rc_g, st_g = g.step(s * sc.dt)
        assert rc_g >= 0
        newton.append((st_g.newton_iters, st_o.newton_iters))
    got = g.particles_by_identity()
    g.close()
    return got, o.particles_by_identity(), newton


@pytest.mark.parametrize("precision", [m.FP64, m.FP32])
def test_pressed_block_with_moving_plate(precision):
    """Config-3 shape at 32^3: 20,480 particles, plate moving down at 0.1 m/s, 3 steps."""
    sc = scenes.pressed_block(32)
    got, ref, newton = run_steps(sc, precision, 3)
    assert all(ng >= 1 for ng, _ in newton)  # the plate loads the block every step
    err = np.abs(got["x"] - ref["x"]).max()
    assert err <= 1e-4 * sc.dx, err
    # the plate pushed the top layer down
    top = ref["x"][:, 1] > np.percentile(ref["x"][:, 1], 99)
    assert np.mean(got["v"][top, 1]) < -0.05


@pytest.mark.parametrize("precision", [m.FP64, m.FP32])
def test_hencky_cube_ten_steps(precision):
    """StVK with Hencky strain (Sec. 4.3.1) on the pre-stretched config-1 cube."""
    sc = scenes.elastic_cube("stretched")
    sc.materials = [scenes.Material(scenes.HENCKY, 1e5, 0.3)]
    got, ref, newton = run_steps(sc, precision, 10)
    assert sum(ng for ng, _ in newton) >= 10
    err = np.abs(got["x"] - ref["x"]).max()
    assert err <= 1e-4 * sc.dx, err


def test_two_spheres_fp32_against_fp64_path():
    """Config 2 (64^3, 59k particles, at contact): one step of the FP32 path (FP32 HVP and
    transfers, FP64 reductions) against the FP64 path, field by field."""
    sc = scenes.two_spheres(64, gap=1.0 / 64)
    out = {}
    p_in = sc.particles(np.float32)  # both paths read the same (FP32-representable) particles
    for prec in (m.FP64, m.FP32):
        g = GpuSim(sc, prec)
        g.set_particles(p_in)
        rc, st = g.step(0.0)
        assert rc == 0 and st.newton_iters >= 1
        out[prec] = (g.particles(), g.field(m.F_NODE_VNEW), st)
        g.close()
    p64, v64, st64 = out[m.FP64]
    p32, v32, st32 = out[m.FP32]
    check(v32, v64, 1e-4, 'v_new fp32 vs fp64')  # both Newton solves stop at 1e-6
    assert np.abs(p32["x"] - p64["x"]).max() <= 1e-4 * sc.dx
    assert abs(st32.newton_iters - st64.newton_iters) <= 1


@pytest.mark.parametrize("precision", [m.FP64, m.FP32])
def test_slab_on_sand_plasticity(precision):
    """Config-5 shape at 32^3 (31,784 particles): a von Mises slab above a Drucker-Prager
    sand box, Hencky elasticity, two materials; 3 steps with the return maps in G2P."""
    sc = scenes.slab_on_sand(32)
    got, ref, newton = run_steps(sc, precision, 3)
    err = np.abs(got["x"] - ref["x"]).max()
    assert err <= 1e-4 * sc.dx, err
    F_err = np.abs(got["F"] - ref["F"]).max()
    assert F_err <= (1e-5 if precision == m.FP32 else 1e-10), F_err
    # the sand settles under gravity: some particles sit at the apex (pure rotation)
    sand = ref["mat"] == 1
    Fs = ref["F"][sand].reshape(-1, 3, 3)
    ortho = np.abs(np.einsum("nij,nkj->nik", Fs, Fs) - np.eye(3)).max(axis=(1, 2)) < 1e-12
    assert ortho.any()


@pytest.mark.parametrize("precision,tol", [(m.FP64, 1e-12), (m.FP32, 1e-6)])
def test_linear_momentum_of_colliding_cubes(precision, tol):
    """Sec. 6.6: two cubes colliding head-on without gravity or walls in reach keep their
    total linear momentum (the paper reports ~1e-14); 20 implicit steps through the impact."""
    sc = scenes.colliding_cubes(64, speed=1.0)
    g = GpuSim(sc, precision)
    g.set_particles()
    p0 = g.particles()
    mom0 = (p0["mp"][:, None] * p0["v"]).sum(axis=0)
    scale = (p0["mp"] * np.abs(p0["v"][:, 0])).sum()
    newton = 0
    for s in range(20):
        rc, st = g.step(s * sc.dt)
        assert rc == 0
        newton += st.newton_iters
    p = g.particles()
    mom = (p["mp"][:, None] * p["v"]).sum(axis=0)
    assert newton > 0                                   # the impact needed Newton solves
    assert np.abs(mom - mom0).max() <= tol * scale, (mom, mom0)
    g.close()
