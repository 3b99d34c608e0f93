"""The error of every FP32 result against the FP64 oracle, per workload shape.

FP32 storage and arithmetic for the transfers, the HVP and the CG vectors, FP64 for the
reductions, the Newton iterate, the gradient, the energy and the stretch eigen-solves: each
result below is compared with the FP64 oracle on the same (FP32-representable) particles,
element by element (norm-relative and largest-element errors, both recorded in the precision
report written by conftest.py when MPML_PRECISION_REPORT is set):
  transfers (m_c, v_c, G_c, V_ck, tau_ck, m_i, v_i), stretch S - I, energy and gradient at the
  Newton start, HVP of a random direction, Newton solution v_new - vhat, and positions after
  three steps (in units of dx, compared particle by particle).
Workloads: config 1 (pre-stretched elastic cube, 8^3 voxels), config 2 (two Neo-Hookean
spheres at contact, 64^3), config 3 (stiff pressed block, 64^3) and config 5 (slab on sand at
impact, 64^3; two plastic materials, mixed cells).
"""
import numpy as np
import pytest
import torch

import oracle
import paper_2602_07853_gb300.mpml as m
from paper_2602_07853_gb300 import scenes
from tests._util import make_oracle
from tests._gpu import GpuSim, OracleSim, check, record

pytestmark = pytest.mark.gpu

WORKLOADS = {
    "config1_cube_stretched": lambda: scenes.elastic_cube("stretched"),
    "config2_two_spheres_64": lambda: scenes.two_spheres(64, gap=1.0 / 64),
    "config3_pressed_block_64": lambda: scenes.pressed_block(64),
    "config5_slab_on_sand_64_impact": lambda: scenes.slab_on_sand(64, impact=True),
}


@pytest.fixture(autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.set_device(0)


@pytest.mark.parametrize("name", list(WORKLOADS))
def test_fp32_results_against_the_fp64_oracle(name):
    sc = WORKLOADS[name]()
    g = GpuSim(sc, m.FP32)
    inp = g.inputs()
    g.set_particles()
    o = make_oracle(sc)
    assert o.unload(**inp) == 0
    g.resample()
    for f, key in ((m.F_CELL_MASS, "m_c"), (m.F_CELL_VEL, "v_c"), (m.F_CELL_VGRAD, "G_c"), (m.F_CELL_VOL, "V_ck"),
                   (m.F_CELL_TAU, "tau_ck"), (m.F_NODE_MASS, "m_i"), (m.F_NODE_VEL, "v_i")):
        check(g.field(f), o.field(key), 1e-5, f"{name}: {key}")
    assert o.stretch() == 0
    m.mpml_stretch(g.ctx)
    mask = o.field("V_ck") > 0
    check(g.field(m.F_CELL_STRETCH)[mask] - np.eye(3), o.field("S_ck")[mask] - np.eye(3), 1e-5, f"{name}: S - I")
    # the Newton start v0 (vhat with the Dirichlet values), energy and gradient there
    _, st0 = o.newton(oracle.default_solver(newton_max=0))
    v0 = o.field("v_new")
    phi_o, g_o = o.eval(v0)
    phi_g, g_g = m.mpml_eval(g.ctx, v0)
    check(np.array([phi_g]), np.array([phi_o]), 1e-5, f"{name}: energy at v0")
    check(g_g, g_o, 1e-5, f"{name}: gradient at v0")
    o.linearize(v0)
    rng = np.random.default_rng(5)
    p = rng.standard_normal(v0.shape).astype(np.float32).astype(np.float64)
    check(m.mpml_hvp(g.ctx, p), o.hvp(p), 1e-5, f"{name}: HVP")
    # Newton solutions (both stop at relative residual 1e-6)
    rc_o, _ = o.newton(oracle.default_solver())
    assert rc_o == 0
    g.resample()  # restores the Newton start (mpml_eval moved the context's iterate)
    rc, st = g.newton()
    assert rc == 0
    vhat = o.field("vhat")
    check(g.field(m.F_NODE_VNEW) - vhat, o.field("v_new") - vhat, 1e-4, f"{name}: v_new - vhat")
    g.close()
    # positions after three steps, particle by particle
    g = GpuSim(sc, m.FP32)
    g.set_particles()
    os_ = OracleSim(make_oracle(sc), g.inputs())
    for s in range(3):
        assert os_.step(s * sc.dt)[0] >= 0
        assert g.step(s * sc.dt)[0] >= 0
    got, ref = g.particles_by_identity(), os_.particles_by_identity()
    record(f"{name}: positions after 3 steps / dx", np.abs(got["x"] - ref["x"]).max() / sc.dx, 1e-4)
    check(got["v"], ref["v"], 1e-4, f"{name}: particle v after 3 steps")
    g.close()
