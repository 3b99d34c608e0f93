"""Batched implicit solve (mpml_newton_step_batch): several independent scenes in
lockstep, every CG round one persistent launch, against the same scenes solved
one by one with mpml_newton_step and against the FP64 oracle.

Tolerances: both solvers stop at relative residual 1e-6, so the node velocities
agree to ~1e-6 relative (checked at 1e-4 as in test_gpu_parity); positions
after 3 steps within 1e-4 dx of the oracle.  Iteration counts are not unique:
the two copies of a scene drift apart by FP32 rounding (atomic sums in a
different order) over the steps, and with CG and Newton both stopping at 1e-6
the residual after a Newton iteration sits near the Newton threshold, so the
Newton counts are not compared and the first CG counts agree within 25%.
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


# default solver options: a shape in free fall starts from g(v0) = 0 up to rounding, which
# the library's rounding floor (1e-12 ||M vhat||) accepts as converged
OPTS = dict()


def small_batch(count=5):
    # scenes of uneven size on 32^3 domains (extents 6..14 voxels, all three shapes)
    return [scenes.batch_scene(i, n=32, extent=6 + 2 * i) for i in range(count)]


def test_batch_matches_single_scene_solves():
    scs = small_batch()
    sims = [GpuSim(sc, m.FP32) for sc in scs]
    for g in sims:
        g.set_particles()
    # step the scenes until they touch the floor, one by one and batched side by side
    ref = [GpuSim(sc, m.FP32) for sc in scs]
    for g in ref:
        g.set_particles()
    for step in range(10):
        for g in sims + ref:
            m.mpml_set_time(g.ctx, step * g.sc.dt)
            g.resample()
        rc, stats = m.mpml_newton_step_batch([g.ctx for g in sims], m.solver_opts(**OPTS))
        assert rc >= 0
        for i, (g, sb) in enumerate(zip(ref, stats)):
            rc1, s1 = g.newton(m.solver_opts(**OPTS))
            info = (step, i, s1.status, sb.status, s1.newton_iters, sb.newton_iters, s1.g0_norm, sb.g0_norm,
                    s1.g_norm, sb.g_norm, list(s1.alpha[:s1.newton_iters]), list(sb.alpha[:sb.newton_iters]),
                    list(s1.cg_iters[:s1.newton_iters]), list(sb.cg_iters[:sb.newton_iters]))
            assert s1.status == 0 and sb.status == 0, info
            # nearly the same first Newton system: Jacobi-PCG counts agree within the
            # FP32 drift.  The Newton counts are not compared: the residual after one
            # Newton step sits at the 1e-6 threshold, so rounding decides between one
            # step and a few more (both converged; the solutions are compared below)
            if s1.newton_iters and sb.newton_iters:
                assert abs(s1.cg_iters[0] - sb.cg_iters[0]) <= max(2, 0.25 * s1.cg_iters[0]), info
            assert sb.g_norm <= max(1e-6 * sb.g0_norm, 1e-11)
        for g, gr in zip(sims, ref):
            v_b, v_1 = g.field(m.F_NODE_VNEW), gr.field(m.F_NODE_VNEW)
            check(v_b, v_1, 1e-4, 'v_new batch vs single')
            g.g2p()
            gr.g2p()
    # the shapes reached the sticky floor: some scene needed Newton iterations with contact
    assert any(s.newton_iters >= 1 for s in stats)
    for g in sims + ref:
        g.close()


def test_batch_scene_against_oracle():
    sc = scenes.batch_scene(2, n=32, extent=10)
    other = scenes.batch_scene(1, n=32, extent=8)
    g, h = GpuSim(sc, m.FP32), GpuSim(other, m.FP32)
    g.set_particles()
    h.set_particles()
    o = OracleSim(make_oracle(sc), g.inputs())
    for step in range(3):
        t = step * sc.dt
        rc, _ = o.step(t)
        assert rc >= 0
        for s in (g, h):
            m.mpml_set_time(s.ctx, t)
            s.resample()
        rc, _ = m.mpml_newton_step_batch([g.ctx, h.ctx], m.solver_opts(**OPTS))
        assert rc >= 0
        g.g2p()
        h.g2p()
    err = np.abs(g.particles_by_identity()["x"] - o.particles_by_identity()["x"]).max()
    assert err <= 1e-4 * sc.dx, err
    g.close()
    h.close()


def test_batch_rejects_mixed_contexts():
    sc = scenes.batch_scene(0, n=32, extent=6)
    a, b = GpuSim(sc, m.FP32), GpuSim(sc, m.FP64)
    a.set_particles()
    b.set_particles()
    a.resample()
    b.resample()
    with pytest.raises(m.MPMLError) as e:
        m.mpml_newton_step_batch([a.ctx, b.ctx])
    assert e.value.code == m.ERR_ARG
    with pytest.raises(m.MPMLError):
        m.mpml_newton_step_batch([a.ctx, a.ctx])
    a.close()
    b.close()


def test_batch_on_separate_streams_with_batched_resample():
    """Contexts on their own streams, Algorithm 2 through mpml_resample_batch: the same
    per-scene results as scene-by-scene steps on one stream."""
    scs = small_batch(4)
    streams = [torch.cuda.Stream() for _ in scs]
    ctxs, parts, keep = [], [], []
    for sc, st in zip(scs, streams):
        mats = [m.material(mt.model, *m.lame_parameters(mt.E, mt.nu)) for mt in sc.materials]
        desc = m.scene_desc(sc.n, sc.dx, sc.dt, sc.gravity, m.FP32, sc.wall_layers, sc.plate, sc.inv_dx)
        ctxs.append(m.mpml_create(desc, mats, st.cuda_stream))
        p = {k: torch.from_numpy(np.ascontiguousarray(v)).cuda() for k, v in sc.particles(np.float32).items()}
        keep.append(p)
        parts.append(m.particles_from_tensors(p["x"], p["v"], p["F"], p["G"], p["mp"], p["Vp"], p["mat"]))
    torch.cuda.synchronize()
    ref = [GpuSim(sc, m.FP32) for sc in scs]
    for g in ref:
        g.set_particles()
    for step in range(8):
        for c in ctxs:
            m.mpml_set_time(c, step * scs[0].dt)
        m.mpml_resample_batch(ctxs, parts)
        rc, stats = m.mpml_newton_step_batch(ctxs)
        assert rc == 0
        for c, pp in zip(ctxs, parts):
            m.mpml_g2p(c, pp)
        for g in ref:
            g.step(step * g.sc.dt)
        torch.cuda.synchronize()
    for p, g in zip(keep, ref):
        got = p["x"].cpu().numpy().astype(np.float64)
        want = g.particles()["x"]
        assert np.abs(got - want).max() <= 1e-4 * g.sc.dx
    for c in ctxs:
        m.mpml_destroy(c)
    for g in ref:
        g.close()
