"""Pins for the oracle's fixed-point plasticity (Sec. "Fixed-Point Plasticity"; CPU only).

With the projection inside Newton, the converged grid state is a fixed point:
every plastic slot's F_c(v) = (I + dt G_c(v)) B_c at the final velocities lies on
or inside its yield surface (the return map leaves it unchanged), and the
gradient criterion holds with those bases.  Without yielding the fixed-point
solve equals the semi-implicit one exactly; with yielding they differ (the
semi-implicit solve's F_c(v) lies outside the surface).
"""
import numpy as np
import pytest

import oracle
from paper_2602_07853_gb300 import scenes
from tests._util import make_oracle


def plastic_scene(kind, n=16, seed=40):
    rng = np.random.Generator(np.random.PCG64(seed))
    if kind == "vm":
        mats = [scenes.Material(scenes.HENCKY, 5e5, 0.3, 1000.0, scenes.VON_MISES, 1e3, 0.0)]
        vox = scenes._grid_voxels((5, 1, 5), (11, 7, 11))
        v0 = np.array([0.0, -2.0, 0.0])
    else:
        mats = [scenes.Material(scenes.HENCKY, 1e6, 0.3, 2000.0, scenes.DRUCKER_PRAGER, 0.0,
                                float(np.radians(30.0)))]
        vox = scenes._grid_voxels((5, 1, 5), (11, 11, 11))
        v0 = np.zeros(3)
    sc = scenes.Scene("fp_" + kind, (n, n, n), 1.0 / n, float(n), 2e-3, (0.0, -9.8, 0.0), mats)
    x = scenes.seed_voxels(vox, sc.dx, 8, rng)
    return scenes._finish(sc, x, np.tile(v0, (len(x), 1)), np.zeros(len(x), np.int64), 8)


def solve(sc, fixed_point, particles=None):
    o = make_oracle(sc)
    p = particles if particles is not None else sc.particles()
    assert o.unload(**p) == 0
    assert o.stretch() == 0
    rc, st = o.newton(oracle.default_solver(fixed_point=fixed_point))
    return o, rc, st


def final_F(o):
    """F_c(v) = (I + dt G_c(v)) B_c of every occupied slot at the final velocities."""
    rc, _ = o.load()  # computes G_c at the solved node velocities
    assert rc == 0
    G = o.field("G_c_new")
    B = o.field("S_ck")[:, 0]
    V = o.field("V_ck")[:, 0]
    F = (np.eye(3) + o.scene.dt * G) @ B
    return F[V > 0]


@pytest.mark.parametrize("kind", ["vm", "dp"])
def test_fixed_point_state_is_on_or_inside_the_yield_surface(kind):
    sc = plastic_scene(kind)
    mat = sc.materials[0]
    mu, lam = oracle.lame(mat.E, mat.nu)
    o, rc, st = solve(sc, 1)
    assert rc == 0 and st.status == 0
    assert st.g_norm <= max(1e-6 * st.g0_norm, 1e-12)
    outside = 0
    for F in final_F(o):
        k, Fn = oracle.return_map(mat.plastic, mu, lam, mat.yield_stress, mat.friction_angle, F)
        if k != 0:
            # at most a rounding-level correction
            assert np.abs(Fn - F).max() <= 1e-7, (k, np.abs(Fn - F).max())
            outside += 1
    # the semi-implicit solve of the same step leaves trial states outside the surface
    o2, rc2, _ = solve(sc, 0)
    assert rc2 == 0
    far = 0
    for F in final_F(o2):
        k, Fn = oracle.return_map(mat.plastic, mu, lam, mat.yield_stress, mat.friction_angle, F)
        far += int(k != 0 and np.abs(Fn - F).max() > 1e-5)
    assert far > 0
    v_fp, v_si = o.field("v_new"), o2.field("v_new")
    assert np.abs(v_fp - v_si).max() > 1e-6


def test_without_yielding_fixed_point_equals_semi_implicit():
    sc = scenes.elastic_cube("stretched")
    o1, rc1, st1 = solve(sc, 1)
    o0, rc0, st0 = solve(sc, 0)
    assert rc1 == rc0 == 0
    assert st1.newton_iters == st0.newton_iters
    assert np.array_equal(o1.field("v_new"), o0.field("v_new"))
