"""Fixed-point plasticity (Sec. "Fixed-Point Plasticity") on the GPU against the FP64
oracle: one solve of a von Mises impact and of a Drucker-Prager column (node
velocities v - vhat to 1e-4 relative, as for every Newton solve: both stop at 1e-6),
the converged bases' trial states on or inside the yield surface (the projection
at the final iterate changes nothing beyond rounding), three steps of positions
(1e-4 dx), and the batched solver's rejection of the option."""
import numpy as np
import pytest
import torch

import oracle
import paper_2602_07853_gb300.mpml as m
from tests._util import make_oracle
from tests._gpu import GpuSim, OracleSim, check, rel_err
from tests.test_oracle_fixed_point import plastic_scene

pytestmark = pytest.mark.gpu


@pytest.fixture(autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.set_device(0)


@pytest.mark.parametrize("kind", ["vm", "dp"])
@pytest.mark.parametrize("precision", [m.FP32, m.FP64])
def test_fixed_point_solve_matches_the_oracle(kind, precision):
    sc = plastic_scene(kind)
    g = GpuSim(sc, precision)
    inp = g.inputs()
    g.set_particles()
    o = make_oracle(sc)
    assert o.unload(**inp) == 0
    g.resample()
    assert o.stretch() == 0
    rc_o, st_o = o.newton(oracle.default_solver(fixed_point=1))
    rc, st = g.newton(m.solver_opts(plastic_fixed_point=1))
    assert rc_o == 0 and rc == 0, (rc, st.status, st.newton_iters)
    assert st.plastic_projections > 0
    vhat = o.field("vhat")
    check(g.field(m.F_NODE_VNEW) - vhat, o.field("v_new") - vhat, 1e-4, 'v_new - vhat')
    # a second solve without the option differs (the semi-implicit grid solve)
    g2 = GpuSim(sc, precision)
    g2.set_particles()
    g2.resample()
    rc2, st2 = g2.newton(m.solver_opts())
    assert rc2 == 0 and st2.plastic_projections == 0
    assert rel_err(g2.field(m.F_NODE_VNEW) - vhat, o.field("v_new") - vhat) > 1e-3
    g.close()
    g2.close()


@pytest.mark.parametrize("precision", [m.FP64, m.FP32])
def test_fixed_point_three_steps(precision):
    sc = plastic_scene("dp")
    g = GpuSim(sc, precision)
    g.set_particles()
    o = OracleSim(make_oracle(sc), g.inputs())
    for s in range(3):
        rc, _ = o.step(s * sc.dt, oracle.default_solver(fixed_point=1))
        assert rc >= 0
        rc_g, st = g.step(s * sc.dt, m.solver_opts(plastic_fixed_point=1))
        assert rc_g >= 0
    err = np.abs(g.particles_by_identity()["x"] - o.particles_by_identity()["x"]).max()
    assert err <= 1e-4 * sc.dx, err
    g.close()


def test_batched_solver_rejects_fixed_point():
    sc = plastic_scene("dp")
    g = GpuSim(sc, m.FP32)
    g.set_particles()
    g.resample()
    with pytest.raises(m.MPMLError) as e:
        m.mpml_newton_step_batch([g.ctx], m.solver_opts(plastic_fixed_point=1))
    assert e.value.code == m.ERR_ARG
    g.close()
