"""Pins for the oracle's implicit Integrate (Algorithm 3) and whole steps (CPU only).

Against: central finite differences of the incremental potential and its
gradient; symmetry; translation invariance (sum of grad w_ic = 0, App. A);
the explicit force of Algorithm 3 at G_c(v) = 0 (which checks the stretch
reconstruction independently, P(S) S^T = tau); a dense numpy solve of the
assembled Hessian; the discrete free-fall closed form; a uniform-stretch
patch test; momentum conservation (Sec. 6.6).
"""
import json
import os

import numpy as np
import pytest

import oracle
from paper_2602_07853_gb300 import scenes
from tests._util import make_oracle

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def stressed_state(model=scenes.FIXED_COROTATED, seed=0, E=1e5, nu=0.3):
    """Cube of 4^3 voxels in a 16^3 grid with a random smooth deformation and velocity."""
    n = 16
    sc = scenes.Scene("stressed", (n, n, n), 1 / n, float(n), 1e-2, (0.0, -9.8, 0.0),
                      [scenes.Material(model, E, nu)])
    rng = np.random.Generator(np.random.PCG64(seed))
    vox = np.mgrid[6:10, 6:10, 6:10].reshape(3, -1).T
    x = scenes.seed_voxels(vox, sc.dx, 8, rng)
    sc = scenes._finish(sc, x, np.zeros_like(x), np.zeros(len(x), np.int64), 8)
    sc.F = sc.F + 0.03 * rng.standard_normal(sc.F.shape)
    sc.v = 0.2 * rng.standard_normal(sc.v.shape)
    return sc


@pytest.mark.parametrize("model", [scenes.FIXED_COROTATED, scenes.NEO_HOOKEAN, scenes.HENCKY, scenes.WATER])
def test_gradient_and_hvp_by_finite_differences(model):
    sc = stressed_state(model, seed=model)
    o = make_oracle(sc)
    assert o.unload(**sc.particles()) == 0
    assert o.stretch() == 0
    nn = o.count("nodes")
    rng = np.random.default_rng(1)
    fixed = o.field("fixed").astype(bool)
    v = o.field("vhat") + 0.05 * rng.standard_normal((nn, 3))
    phi, g = o.eval(v)
    d = rng.standard_normal((nn, 3))
    d[fixed] = 0
    h = 1e-6
    fd = (o.eval(v + h * d, grad=False)[0] - o.eval(v - h * d, grad=False)[0]) / (2 * h)
    assert np.isclose(np.sum(g * d), fd, rtol=1e-7)
    # unprojected Hessian == derivative of the gradient
    o.linearize(v, project=False)
    Hd = o.hvp(d)
    fdg = (o.eval(v + h * d)[1] - o.eval(v - h * d)[1]) / (2 * h)
    assert np.linalg.norm(Hd - fdg) <= 1e-6 * np.linalg.norm(Hd)
    # symmetry u^T H w = w^T H u (projected)
    o.linearize(v, project=True)
    u, w = rng.standard_normal((nn, 3)), rng.standard_normal((nn, 3))
    u[fixed] = 0
    w[fixed] = 0
    assert np.isclose(np.sum(u * o.hvp(w)), np.sum(w * o.hvp(u)), rtol=1e-12)
    assert np.sum(u * o.hvp(u)) > 0


@pytest.mark.parametrize("model", [scenes.NEO_HOOKEAN, scenes.WATER])
def test_elastic_gradient_translation_invariant_and_explicit_force(model):
    """With no fixed nodes: sum_i (g_i - m_i (v_i - vhat_i)) = 0.  At v = 0
    (G_c(0) = 0, F_c = S_c) the elastic gradient equals -dt f_i with f_i the
    explicit force of Algorithm 3 built from the transferred tau_c: this holds
    only if P(S_c) S_c^T = tau_c, an independent pin of the stretch step."""
    sc = stressed_state(model, seed=3)
    sc.wall_layers = 0
    o = make_oracle(sc)
    assert o.unload(**sc.particles()) == 0
    assert o.stretch() == 0
    nn = o.count("nodes")
    m, vhat = o.field("m_i"), o.field("vhat")
    v = np.zeros((nn, 3))
    _, g = o.eval(v)
    ge = g - m[:, None] * (v - vhat)
    f = o.explicit_force()
    assert np.allclose(ge, -sc.dt * f, atol=1e-9 * np.abs(ge).max())
    v = 0.1 * np.random.default_rng(0).standard_normal((nn, 3))
    _, g = o.eval(v)
    ge = g - m[:, None] * (v - vhat)
    assert np.allclose(ge.sum(0), 0, atol=1e-10 * np.abs(ge).sum())


def test_pcg_matches_dense_solve():
    sc = stressed_state(scenes.FIXED_COROTATED, seed=4, E=1e6)
    o = make_oracle(sc)
    assert o.unload(**sc.particles()) == 0
    assert o.stretch() == 0
    nn = o.count("nodes")
    v = o.field("vhat")
    o.linearize(v)
    free = ~o.field("fixed").astype(bool)
    idx = np.nonzero(np.repeat(free, 3))[0]
    H = np.zeros((3 * nn, 3 * nn))
    for j in idx:
        e = np.zeros(3 * nn)
        e[j] = 1
        H[:, j] = o.hvp(e.reshape(nn, 3)).ravel()
    Hf = H[np.ix_(idx, idx)]
    assert np.allclose(Hf, Hf.T, atol=1e-12 * np.abs(Hf).max())
    assert np.linalg.eigvalsh(Hf).min() > 0
    b = np.random.default_rng(5).standard_normal(3 * nn)
    x, it, rr = o.pcg(b.reshape(nn, 3), rtol=1e-12)
    xref = np.linalg.solve(Hf, b[idx])
    assert np.allclose(x.ravel()[idx], xref, rtol=1e-8, atol=1e-9 * np.abs(xref).max())
    d = o.diag().ravel()
    assert np.allclose(d[idx], np.diag(Hf), rtol=1e-12)


def run_steps(sc, steps, solver=None):
    o = make_oracle(sc)
    p = sc.particles()
    stats = []
    for s in range(steps):
        o.set_time(s * sc.dt)
        rc, p, st = o.step(p, solver)
        assert rc >= 0, rc
        stats.append(st)
    return p, stats


def test_free_fall_discrete_closed_form():
    """Unstressed free fall: G_c(vhat) = 0 so Newton takes no iteration and the
    centre of mass follows y_k = y_0 + g dt^2 k (k + 1) / 2 (vhat = v + dt g, then
    x += dt v^{n+1}); within 1e-4 dx of it, and O(dt) from g t^2 / 2."""
    sc = scenes.elastic_cube("fall")
    y0 = np.average(sc.x[:, 1], weights=sc.mp)
    p, stats = run_steps(sc, 10)
    assert all(st.newton_iters == 0 for st in stats)
    k = 10
    y = np.average(p["x"][:, 1], weights=p["mp"])
    ref = y0 + 0.5 * (-9.8) * sc.dt ** 2 * k * (k + 1)
    assert abs(y - ref) < 1e-4 * sc.dx
    t = k * sc.dt
    assert abs(y - (y0 - 0.5 * 9.8 * t * t)) < 1.1 * 0.5 * 9.8 * sc.dt * t
    assert np.allclose(p["F"], np.eye(3), atol=1e-13)


def test_uniform_stretch_patch():
    """All particles with the same symmetric F0: every fully covered centre gets
    tau_c = tau(F0) and S_c = F0, and the elastic force vanishes at nodes whose
    8 neighbouring centres are all fully covered."""
    sc = scenes.elastic_cube("stretched")
    sc.gravity = (0.0, 0.0, 0.0)

    class _Mid:  # regular 2x2x2 lattice (no jitter) so that V_c is uniform inside
        def random(self, shape):
            return np.full(shape, 0.5)

    vox = np.mgrid[12:20, 16:24, 12:20].reshape(3, -1).T
    sc.x = scenes.seed_voxels(vox, sc.dx, 8, _Mid())
    o = make_oracle(sc)
    assert o.unload(**sc.particles()) == 0
    assert o.stretch() == 0
    S = o.field("S_ck")[:, 0]
    ijk = oracle.decode_keys(o.cell_keys(), sc.n)
    inner = np.all((ijk >= [12, 16, 12]) & (ijk < [19, 23, 19]), axis=1)
    F0 = np.diag([1.05, 0.97, 1.0])
    assert np.allclose(S[inner], F0, atol=1e-12)
    f = o.explicit_force()
    nijk = oracle.decode_keys(o.node_keys(), sc.n)
    # cells 13..18 (y: 17..22) collect the full 2x2x2 lattice weight; nodes between them
    interior = np.all((nijk >= [14, 18, 14]) & (nijk <= [18, 22, 18]), axis=1)
    assert np.abs(f[interior]).max() < 1e-9 * np.abs(f).max()


def test_newton_converges_and_meets_tolerances():
    sc = scenes.elastic_cube("stretched")
    o = make_oracle(sc)
    assert o.unload(**sc.particles()) == 0
    assert o.stretch() == 0
    rc, st = o.newton(oracle.default_solver())
    assert rc == 0
    assert st.newton_iters >= 1
    assert st.g_norm <= 1e-6 * st.g0_norm
    assert st.phi <= st.phi0


def test_linear_momentum_conserved():
    """Two cubes colliding without gravity and away from the walls: the transfers
    conserve momentum exactly and the solve to its tolerance, so with tight
    tolerances the total momentum stays at round-off (Sec. 6.6 reports
    max |P| = 7.11e-15 kg m/s for its pair of cubes)."""
    with open(os.path.join(GOLDEN, "paper_momentum.json")) as fh:
        gold = json.load(fh)
    sc = scenes.colliding_cubes(n=32, speed=1.0)
    P0 = (sc.mp[:, None] * sc.v).sum(0)
    scale = (sc.mp * np.abs(sc.v[:, 0])).sum()
    p, stats = run_steps(sc, 8, oracle.default_solver(cg_rtol=1e-13, newton_rtol=1e-12))
    P = (p["mp"][:, None] * p["v"]).sum(0)
    assert np.abs(P - P0).max() <= gold["our_bound_relative"] * scale
    assert any(st.newton_iters > 0 for st in stats)


@pytest.mark.slow
def test_angular_momentum_rotating_rod():
    """Rotating rod (Sec. 6.6): L_z relative drift is small (the paper reports 1.02e-4
    over its run; here 10 steps with 64^3 cells)."""
    sc = scenes.rotating_rod(n=64)
    L0 = np.sum(sc.mp * (sc.x[:, 0] - 0.5) * sc.v[:, 1] - sc.mp * (sc.x[:, 1] - 0.5) * sc.v[:, 0])
    p, _ = run_steps(sc, 10, oracle.default_solver(cg_rtol=1e-10, newton_rtol=1e-10))
    x, v, m = p["x"], p["v"], p["mp"]
    L = np.sum(m * (x[:, 0] - 0.5) * v[:, 1] - m * (x[:, 1] - 0.5) * v[:, 0])
    assert abs(L - L0) / abs(L0) < 2e-3
