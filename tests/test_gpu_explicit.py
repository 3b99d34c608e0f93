"""Explicit integrator (mpml_explicit_step) against the FP64 oracle's explicit branch.

Tolerances as in test_gpu_parity: node velocities <= 1e-5 (FP32) / 1e-10 (FP64)
norm-relative after one step, positions after 10 steps within 1e-4 dx.
"""
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


@pytest.mark.parametrize("precision", [m.FP32, m.FP64])
def test_explicit_node_velocities(precision):
    sc = scenes.elastic_cube("stretched")
    g = GpuSim(sc, precision)
    inp = g.inputs()
    g.set_particles()
    g.resample()
    m.mpml_explicit_step(g.ctx)
    o = make_oracle(sc)
    assert o.unload(**inp) == 0
    o.explicit()
    v_o = o.field("v_new")
    v_g = g.field(m.F_NODE_VNEW)
    check(v_g - o.field("vhat"), v_o - o.field("vhat"), TOL[precision], 'v_new - vhat')
    g.close()


@pytest.mark.parametrize("precision", [m.FP32, m.FP64])
def test_explicit_ten_steps(precision):
    sc = scenes.elastic_cube("stretched")
    g = GpuSim(sc, precision)
    g.set_particles()
    o = OracleSim(make_oracle(sc), g.inputs())
    for s in range(10):
        rc, _ = o.step(s * sc.dt, explicit=True)
        assert rc == 0
        m.mpml_set_time(g.ctx, s * sc.dt)
        g.resample()
        m.mpml_explicit_step(g.ctx)
        g.g2p()
    err = np.abs(g.particles_by_identity()["x"] - o.particles_by_identity()["x"]).max()
    assert err <= 1e-4 * sc.dx, err
    g.close()
