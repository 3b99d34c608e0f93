"""The solver paths the large workloads run, and the solver's failure reports, on the GPU.

- Every launch shape of the persistent Jacobi-PCG kernel (tangent block staged in shared
  memory or streamed from global memory with the CTA on one brick, one or two CTAs per SM;
  one brick per 64-thread group, two to four CTAs per SM), forced through
  mpml_set_pcg_config, on both tangent formats, against the FP64 oracle's Newton solution
  (both stop at relative residual 1e-6: compared at 1e-4 on v - vhat, element by element),
  and the persistent-solver autotuner's choice.
- Full-size solves of the 3-8M pressed block (1,051,200 active cells, about 2,100 cell bricks:
  the column-group and streamed kernels) and of the 256^3 slab on sand at impact (19.2M
  particles, 2.5M cells: the column-group kernel and the staged 45-number kernel with 16+ bricks
  per CTA): the oracle's own FP64 gradient at the GPU solution is within the Newton tolerance of
  its gradient at the start.
- The slab on sand at impact, reduced to 64^3 (mixed slab / sand cells from the first step,
  plastic flow in both materials), stepped through the impact against the oracle.
- A batch of 16 scenes of uneven size in one lockstep solve against per-scene oracle steps.
- Failure reports (Algorithm 3's solve must report them): a grid-barrier wait that runs out
  (MPML_ERR_TIMEOUT, context usable afterwards), a stress that no stretch can produce
  (MPML_ERR_STRETCH, as the oracle reports), a Newton cap that is too small
  (MPML_WARN_NOT_CONVERGED).
"""
import numpy as np
import pytest
import torch

import oracle
import paper_2602_07853_gb300.mpml as m
from paper_2602_07853_gb300 import scenes
from tests._util import make_oracle
from tests._gpu import GpuSim, OracleSim, check

pytestmark = pytest.mark.gpu

SHAPES = [tuple(sh) for sh in m.PCG_SHAPE_TABLE]


@pytest.fixture(autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.set_device(0)


def oracle_solution(sc):
    o = make_oracle(sc)
    inp = {k: (v.astype(np.float64) if k != "mat" else v) for k, v in sc.particles(np.float32).items()}
    assert o.unload(**inp) == 0
    assert o.stretch() == 0
    rc, st = o.newton(oracle.default_solver())
    assert rc == 0
    return o, st


@pytest.mark.parametrize("name", ["pressed_block_32", "stretched_cube", "slab_on_sand_32_impact"])
def test_every_persistent_shape_matches_the_oracle(name):
    sc = {"pressed_block_32": lambda: scenes.pressed_block(32),
          "stretched_cube": lambda: scenes.elastic_cube("stretched"),
          "slab_on_sand_32_impact": lambda: scenes.slab_on_sand(32, impact=True)}[name]()
    o, st_o = oracle_solution(sc)
    assert st_o.newton_iters >= 1
    vhat, v_o = o.field("vhat"), o.field("v_new")
    for staging, ctas in SHAPES:
        g = GpuSim(sc, m.FP32)
        g.set_particles()
        m.mpml_set_pcg_config(g.ctx, staging, ctas)
        g.resample()
        rc, st = g.newton()
        assert rc == 0, (staging, ctas, rc)
        _, last_staging, last_ctas = m.mpml_get_pcg_config(g.ctx)
        assert (last_staging, last_ctas) == (staging, ctas)
        check(g.field(m.F_NODE_VNEW) - vhat, v_o - vhat, 1e-4, f"v_new - vhat ({name}, staging {staging}, {ctas}/SM)")
        g.close()


def full_size_gradient_check(sc, expect_staging, force=None, opts=None):
    """GPU Newton solve at full size; the oracle's FP64 gradient at the GPU solution."""
    g = GpuSim(sc, m.FP32)
    g.set_particles()
    if force is not None:
        m.mpml_set_pcg_config(g.ctx, *force)
    o = make_oracle(sc)
    assert o.unload(**g.inputs()) == 0
    g.resample()
    assert np.array_equal(g.keys(m.KEYS_CELLS), o.cell_keys())
    assert o.stretch() == 0
    # the oracle's gradient norm at the Newton start v0 (vhat with the Dirichlet values imposed)
    _, st0 = o.newton(oracle.default_solver(newton_max=0))
    g0 = st0.g0_norm
    assert g0 > 0
    rc, st = g.newton(opts)
    assert rc == 0, (rc, st.newton_iters, list(st.cg_iters[:st.newton_iters]))
    assert st.newton_iters >= 1
    _, last_staging, _ = m.mpml_get_pcg_config(g.ctx)
    assert last_staging == expect_staging
    v_g = g.field(m.F_NODE_VNEW)
    g.close()
    _, g1 = o.eval(v_g)
    ratio = np.linalg.norm(g1) / g0
    assert ratio <= 2e-6, ratio
    return st


@pytest.mark.parametrize("force", [None, (m.PCG_STREAMED, 2)])
def test_full_size_pressed_block_236(force):
    """Config 3 at dx = 1/236 (7.9M particles, about 2,100 cell bricks): without a tuned shape,
    above eight cell bricks per SM the column-group solver runs the compressed tangent (the fixed
    rule); and the CTA-per-brick solver with streamed rows and many bricks per CTA."""
    full_size_gradient_check(scenes.pressed_block(236), force[0] if force else m.PCG_COLUMNS, force)


@pytest.mark.parametrize("force", [None, (m.PCG_STAGED, 2)])
def test_full_size_slab_on_sand_256_at_impact(force):
    """Config 5 (256^3, 19.2M particles, two plastic materials) at impact: the column-group
    solver (fixed rule for the 45-number tangent above eight cell bricks per SM), and the
    staged solver with many bricks per CTA."""
    full_size_gradient_check(scenes.slab_on_sand(256, impact=True), force[0] if force else m.PCG_COLUMNS, force)


@pytest.mark.parametrize("name", ["two_spheres_48", "slab_on_sand_48_impact"])
def test_pcg_autotuner_picks_the_fastest_shape(name):
    """mpml_autotune_pcg times every shape on the current system; its choice is the fastest
    it measured, later solves of the context (and of another context of the same format and
    size class) run it, and their solutions match the oracle."""
    sc = {"two_spheres_48": lambda: scenes.two_spheres(48, gap=1.0 / 48),
          "slab_on_sand_48_impact": lambda: scenes.slab_on_sand(48, impact=True)}[name]()
    m.mpml_tile_cache_clear()
    o, _ = oracle_solution(sc)
    vhat, v_o = o.field("vhat"), o.field("v_new")
    g = GpuSim(sc, m.FP32)
    g.set_particles()
    g.resample()
    m.mpml_stretch(g.ctx)
    m.mpml_linearize(g.ctx, g.field(m.F_NODE_VHAT))
    shape, ms = m.mpml_autotune_pcg(g.ctx, 20, 2)
    timed = [t for t in ms if t >= 0]
    assert len(timed) >= 4 and ms[shape] == min(timed), ms
    for ctx_owner in (g, None):
        h = g if ctx_owner is g else GpuSim(sc, m.FP32)
        if h is not g:
            h.set_particles()
        # resample: mpml_newton_step starts from the context's current node velocities, which
        # mpml_linearize set to its argument
        h.resample()
        rc, st = h.newton()
        assert rc == 0
        _, staging, ctas = m.mpml_get_pcg_config(h.ctx)
        assert (staging, ctas) == tuple(m.PCG_SHAPE_TABLE[shape])
        check(h.field(m.F_NODE_VNEW) - vhat, v_o - vhat, 1e-4, f"v_new - vhat (tuned shape {shape})")
        h.close()
    m.mpml_tile_cache_clear()


def test_full_size_slab_on_sand_256_inexact_newton():
    """Config 5 at impact with the inexact-Newton forcing (cg_forcing 0.3): every CG solve stops
    at its forcing term (none below cg_rtol, the first at the cap), and Newton's own FP64 test
    still holds -- the oracle's gradient at the GPU solution is within 2e-6 of its initial norm."""
    st = full_size_gradient_check(scenes.slab_on_sand(256, impact=True), m.PCG_COLUMNS,
                                  opts=m.solver_opts(cg_forcing=0.3))
    rel = [st.cg_rel_resid[k] for k in range(st.newton_iters)]
    assert all(r <= 0.5 for r in rel), rel
    assert 0.1 <= rel[0] <= 0.3 * (1 + 1e-6), rel  # the first solve stops at eta_0 = 0.3
    assert st.g_norm <= 1e-6 * st.g0_norm


@pytest.mark.parametrize("precision", [m.FP32, m.FP64])
def test_slab_on_sand_impact_inexact_newton_against_the_oracle(precision):
    """Config 5 reduced to 64^3 from the moment of impact, 4 steps with the inexact-Newton forcing
    (cg_forcing 0.3) against the oracle's exact-solve steps: positions within 1e-4 dx, F and v
    element by element -- both stop Newton at 1e-6 of the initial FP64 gradient, so the forcing
    changes the work, not the result."""
    sc = scenes.slab_on_sand(64, impact=True)
    g = GpuSim(sc, precision)
    g.set_particles()
    o = OracleSim(make_oracle(sc), g.inputs())
    opts = m.solver_opts(cg_forcing=0.3)
    cg_g = cg_o = 0
    for s in range(4):
        rc, st_o = o.step(s * sc.dt)
        assert rc >= 0
        rc_g, st_g = g.step(s * sc.dt, opts)
        assert rc_g == 0
        assert st_g.g_norm <= 1e-6 * st_g.g0_norm
        cg_g += st_g.cg_iters_total
        cg_o += st_o.cg_iters_total
    assert cg_g < cg_o, (cg_g, cg_o)
    got, ref = g.particles_by_identity(), o.particles_by_identity()
    err = np.abs(got["x"] - ref["x"]).max()
    assert err <= 1e-4 * sc.dx, err
    # both sides stop Newton at 1e-6 of the initial gradient along different iterate paths, so the
    # bar is that of the FP32 path in both precisions (the Newton tolerance, not the rounding)
    check(got["F"] - np.eye(3), ref["F"] - np.eye(3), 1e-4, "F - I after 4 steps")
    check(got["v"], ref["v"], 1e-4, "v after 4 steps")
    g.close()


def test_cg_forcing_out_of_range_is_rejected():
    """cg_forcing outside [0, 0.5] (or NaN) is MPML_ERR_ARG, for the single-scene and the batched
    solver; in range, both converge to Newton's tolerance."""
    sc = scenes.elastic_cube("stretched")
    g = GpuSim(sc, m.FP32)
    g.set_particles()
    g.resample()
    for bad in (-0.1, 0.6, float("nan")):
        rc = m.load().mpml_newton_step(g.ctx, m.C.byref(m.solver_opts(cg_forcing=bad)), None)
        assert rc == m.ERR_ARG, (bad, rc)
    rc, _ = g.newton(m.solver_opts(cg_forcing=0.5))
    assert rc == 0
    g.close()
    scs = [scenes.random_state(scenes.batch_scene(i, n=32, extent=6 + i), 100 + i, v_scale=0.05, G_scale=0.5,
                               F_scale=0.01) for i in range(2)]
    sims = [GpuSim(s, m.FP32) for s in scs]
    for s in sims:
        s.set_particles()
        s.resample()
    ptrs = [s.ctx.value if isinstance(s.ctx, m.C.c_void_p) else s.ctx for s in sims]
    rc = m.load().mpml_newton_step_batch((m.C.c_void_p * 2)(*ptrs), 2,
                                         m.C.byref(m.solver_opts(cg_forcing=0.7)), None)
    assert rc == m.ERR_ARG
    rc, stats = m.mpml_newton_step_batch([s.ctx for s in sims], m.solver_opts(cg_forcing=0.3))
    assert rc == 0
    for st in stats:
        assert st.newton_iters >= 1 and st.g_norm <= 1e-6 * st.g0_norm
    for s in sims:
        s.close()


@pytest.mark.parametrize("precision", [m.FP32, m.FP64])
def test_slab_on_sand_through_the_impact(precision):
    """Config 5 reduced to 64^3 (288,608 particles) from the moment of impact: 4 steps with
    mixed slab / sand cells, Newton with line search, and the von Mises / Drucker-Prager
    return maps in G2P; positions within 1e-4 dx of the oracle and F element by element."""
    sc = scenes.slab_on_sand(64, impact=True)
    g = GpuSim(sc, precision)
    g.set_particles()
    o = OracleSim(make_oracle(sc), g.inputs())
    newton = 0
    for s in range(4):
        rc, st_o = o.step(s * sc.dt)
        assert rc >= 0
        rc_g, st_g = g.step(s * sc.dt)
        assert rc_g == 0
        assert st_g.newton_iters == st_o.newton_iters
        newton += st_g.newton_iters
    assert newton >= 4
    V = o.o.field("V_ck")
    assert ((V > 0).sum(axis=1) == 2).any()  # mixed slab / sand cells
    got, ref = g.particles_by_identity(), o.particles_by_identity()
    err = np.abs(got["x"] - ref["x"]).max()
    assert err <= 1e-4 * sc.dx, err
    check(got["F"] - np.eye(3), ref["F"] - np.eye(3), 1e-4 if precision == m.FP32 else 1e-9, "F - I after 4 steps")
    check(got["v"], ref["v"], 1e-4 if precision == m.FP32 else 1e-9, "v after 4 steps")
    g.close()


def test_batch_of_16_uneven_scenes_against_the_oracle():
    """16 scenes of extents 6..21 voxels (boxes, spheres, tori; ~200 to ~80k particles) on their
    own 32^3 grids with seeded random velocity, velocity gradient and deformation (so every
    scene solves a nonlinear system from the first step), two lockstep batched steps against
    each scene's oracle steps."""
    scs = [scenes.random_state(scenes.batch_scene(i, n=32, extent=6 + i), 100 + i, v_scale=0.05, G_scale=0.5,
                               F_scale=0.01) for i in range(16)]
    sims = [GpuSim(sc, m.FP32) for sc in scs]
    for g in sims:
        g.set_particles()
    orcs = [OracleSim(make_oracle(sc), g.inputs()) for sc, g in zip(scs, sims)]
    for step in range(2):
        for o, sc in zip(orcs, scs):
            rc, _ = o.step(step * sc.dt)
            assert rc >= 0
        for g in sims:
            m.mpml_set_time(g.ctx, step * g.sc.dt)
            g.resample()
        rc, stats = m.mpml_newton_step_batch([g.ctx for g in sims])
        assert rc == 0
        assert all(s.newton_iters >= 1 for s in stats)
        for g in sims:
            g.g2p()
    for g, o, sc in zip(sims, orcs, scs):
        got, p = g.particles_by_identity(), o.particles_by_identity()
        err = np.abs(got["x"] - p["x"]).max()
        assert err <= 1e-4 * sc.dx, (sc.name, err)
        check(got["v"], p["v"], 1e-4, f"v ({sc.name})")
        g.close()


def test_grid_barrier_timeout_is_reported_and_the_context_recovers():
    """A bound of one poll per grid-barrier wait: CTAs give up waiting for the others, the
    persistent solve ends early, and mpml_newton_step reports MPML_ERR_TIMEOUT.  After the next
    resample (which clears the latched status) the default bound solves normally."""
    sc = scenes.two_spheres(64, gap=1.0 / 64)
    g = GpuSim(sc, m.FP32)
    g.set_particles()
    g.resample()
    m.mpml_set_pcg_config(g.ctx, barrier_spins=1)
    with pytest.raises(m.MPMLError) as e:
        g.newton()
    assert e.value.code == m.ERR_TIMEOUT
    m.mpml_set_pcg_config(g.ctx)
    g.resample()
    rc, st = g.newton()
    assert rc == 0 and st.newton_iters >= 1
    g.close()


def test_batched_grid_barrier_timeout_is_reported():
    scs = [scenes.random_state(scenes.batch_scene(i, n=32, extent=6 + i), 200 + i, v_scale=0.05) for i in range(3)]
    sims = [GpuSim(sc, m.FP32) for sc in scs]
    for g in sims:
        g.set_particles()
        g.resample()
    m.mpml_set_pcg_config(sims[0].ctx, barrier_spins=1)
    with pytest.raises(m.MPMLError) as e:
        m.mpml_newton_step_batch([g.ctx for g in sims])
    assert e.value.code == m.ERR_TIMEOUT
    for g in sims:
        g.close()


@pytest.mark.parametrize("precision", [m.FP32, m.FP64])
def test_unrecoverable_compression_reports_stretch_error(precision):
    """Fixed-corotated particles compressed to F = 0.6 I (J = 0.216): the cell stress has no
    stretch on the admissible branch (J >= 1/2).  The device latches the error and
    mpml_newton_step returns MPML_ERR_STRETCH, as the oracle's stretch reconstruction does."""
    sc = scenes.elastic_cube("fall")
    sc.F = np.tile(0.6 * np.eye(3), (sc.num_particles, 1, 1))
    o = make_oracle(sc)
    assert o.unload(**{k: (v.astype(np.float64) if k != "mat" else v)
                       for k, v in sc.particles(np.float32).items()}) == 0
    assert o.stretch() == m.ERR_STRETCH
    g = GpuSim(sc, precision)
    g.set_particles()
    g.resample()
    with pytest.raises(m.MPMLError) as e:
        g.newton()
    assert e.value.code == m.ERR_STRETCH
    g.close()


def test_newton_cap_reports_not_converged():
    """The pressed block needs more than one Newton iteration per step: with newton_max = 1
    the step returns MPML_WARN_NOT_CONVERGED (a warning: the iterate is still usable)."""
    sc = scenes.pressed_block(32)
    g = GpuSim(sc, m.FP32)
    g.set_particles()
    g.resample()
    rc, st = g.newton(m.solver_opts(newton_max=1))
    assert rc == m.WARN_NOT_CONVERGED
    assert st.newton_iters == 1 and st.g_norm > 1e-6 * st.g0_norm
    g.close()
