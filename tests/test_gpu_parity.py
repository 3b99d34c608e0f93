"""CUDA path vs the FP64 oracle, element by element, through the C ABI.

Tolerances:
  - integer work (keys, sort order, active cells, DOF nodes): bit-exact;
  - FP32 transfers / stretch / energy / gradient / HVP: <= 1e-5 per field, both
    norm-relative and as the largest element error relative to the field's
    largest element (FP32 sums of at most 64 weighted terms round to about
    64 * 2^-24 = 4e-6 of their largest term; 1e-5 is also the workload's
    gradient / HVP bound);
  - FP64 path: <= 1e-10;
  - positions after 10 steps: <= 1e-4 dx.
"""
import numpy as np
import pytest
import torch

import oracle
import paper_2602_07853_gb300.mpml as m
from paper_2602_07853_gb300 import scenes
from tests._util import make_oracle
from tests._gpu import GpuSim, OracleSim, check, rel_err

pytestmark = pytest.mark.gpu

TOL = {m.FP32: 1e-5, m.FP64: 1e-10}


def random_scene(seed=0, n=16, count=300):
    rng = np.random.default_rng(seed)
    sc = scenes.Scene("random", (n, n, n), 1.0 / n, float(n), 1e-3, (0.0, -9.8, 0.0),
                      [scenes.Material(scenes.FIXED_COROTATED, 1e5, 0.3),
                       scenes.Material(scenes.NEO_HOOKEAN, 3e4, 0.4, rho=2000.0)])
    x = rng.uniform(1.6 / n, 1 - 1.6 / n, (count, 3))
    x[:10, 0] = (np.floor(x[:10, 0] * n) + 0.5) / n  # f == 0 on one axis
    sc.x = x
    sc.v = rng.standard_normal((count, 3))
    sc.G = rng.standard_normal((count, 3, 3))
    sc.F = np.eye(3) + 0.05 * rng.standard_normal((count, 3, 3))
    sc.Vp = np.full(count, sc.dx ** 3 / 8)
    sc.mat = rng.integers(0, 2, count).astype(np.int32)
    sc.mp = np.array([1000.0, 2000.0])[sc.mat] * sc.Vp
    return sc


def both(sc, precision):
    g = GpuSim(sc, precision)
    inp = g.inputs()
    g.set_particles()
    o = make_oracle(sc)
    assert o.unload(**inp) == 0
    g.resample()
    return g, o, inp


@pytest.fixture(autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.set_device(0)


@pytest.mark.parametrize("precision", [m.FP32, m.FP64])
def test_sort_and_sets_bit_exact(precision):
    for seed, count in ((0, 300), (1, 5000)):
        g, o, _ = both(random_scene(seed, count=count), precision)
        assert np.array_equal(g.keys(m.KEYS_PARTICLES), o.particle_keys())
        assert np.array_equal(g.t["perm"].cpu().numpy().astype(np.int64), o.perm())
        assert np.array_equal(g.keys(m.KEYS_CELLS), o.cell_keys())
        assert np.array_equal(g.keys(m.KEYS_NODES), o.node_keys())
        assert np.array_equal(g.field(m.F_NODE_FIXED), o.field("fixed"))
        g.close()


@pytest.mark.parametrize("precision", [m.FP32, m.FP64])
def test_unload_fields(precision):
    g, o, _ = both(random_scene(2, count=3000), precision)
    tol = TOL[precision]
    pairs = [(m.F_CELL_MASS, "m_c"), (m.F_CELL_VEL, "v_c"), (m.F_CELL_VGRAD, "G_c"), (m.F_CELL_VOL, "V_ck"),
             (m.F_CELL_TAU, "tau_ck"), (m.F_NODE_MASS, "m_i"), (m.F_NODE_VEL, "v_i"), (m.F_NODE_VHAT, "vhat")]
    for f, name in pairs:
        check(g.field(f), o.field(name), tol, name)
    g.close()


@pytest.mark.parametrize("precision", [m.FP32, m.FP64])
def test_stretch_energy_gradient_hvp(precision):
    sc = random_scene(3, count=4000)
    sc.F = np.eye(3) + 0.02 * np.random.default_rng(4).standard_normal(sc.F.shape)
    g, o, _ = both(sc, precision)
    tol = TOL[precision]
    assert o.stretch() == 0
    m.mpml_stretch(g.ctx)
    S_g, S_o = g.field(m.F_CELL_STRETCH), o.field("S_ck")
    V = o.field("V_ck")
    mask = V > 0
    check(S_g[mask] - np.eye(3), S_o[mask] - np.eye(3), tol, 'S - I')
    nn = o.count("nodes")
    rng = np.random.default_rng(5)
    v = o.field("vhat") + 0.05 * rng.standard_normal((nn, 3))
    v = v.astype(g.npdt).astype(np.float64)
    phi_o, g_o = o.eval(v)
    phi_g, g_g = m.mpml_eval(g.ctx, v)
    assert abs(phi_g - phi_o) <= tol * abs(phi_o)
    check(g_g, g_o, tol, 'gradient')
    o.linearize(v, project=True)
    p = rng.standard_normal((nn, 3)).astype(g.npdt).astype(np.float64)
    check(m.mpml_hvp(g.ctx, p), o.hvp(p), tol, 'hvp')
    g.close()


def _rotation(rng):
    q = rng.standard_normal(4)
    w, x, y, z = q / np.linalg.norm(q)
    return np.array([[1 - 2 * (y * y + z * z), 2 * (x * y - z * w), 2 * (x * z + y * w)],
                     [2 * (x * y + z * w), 1 - 2 * (x * x + z * z), 2 * (y * z - x * w)],
                     [2 * (x * z - y * w), 2 * (y * z + x * w), 1 - 2 * (x * x + y * y)]])


@pytest.mark.parametrize("precision", [m.FP32, m.FP64])
@pytest.mark.parametrize("kind", ["rest", "isotropic", "double", "near_double"])
@pytest.mark.parametrize("model", [scenes.FIXED_COROTATED, scenes.NEO_HOOKEAN, scenes.HENCKY])
def test_stretch_degenerate_stress(precision, kind, model):
    """Stretch reconstruction where the cell-averaged Kirchhoff stress has repeated or
    nearly repeated eigenvalues (and zero stress at rest): the symmetric eigen-solve must
    still reach the oracle's FP64 stretch (Sec. 4.2)."""
    n = 16
    rng = np.random.default_rng(11)
    count = 3000
    sc = scenes.Scene("degenerate", (n, n, n), 1.0 / n, float(n), 1e-3, (0.0, -9.8, 0.0),
                      [scenes.Material(model, 1e5, 0.3)])
    sc.x = rng.uniform(1.6 / n, 1 - 1.6 / n, (count, 3))
    sc.v = rng.standard_normal((count, 3))
    sc.G = np.zeros((count, 3, 3))
    R = _rotation(rng)
    diag = {"rest": (1.0, 1.0, 1.0), "isotropic": (1.01, 1.01, 1.01), "double": (1.01, 1.01, 0.98),
            "near_double": (1.01, 1.01 + 1e-9, 0.98)}[kind]
    F = R @ np.diag(diag) @ R.T
    sc.F = np.broadcast_to(F, (count, 3, 3)).copy()
    sc.Vp = np.full(count, sc.dx ** 3 / 8)
    sc.mat = np.zeros(count, np.int32)
    sc.mp = 1000.0 * sc.Vp
    g, o, _ = both(sc, precision)
    assert o.stretch() == 0
    m.mpml_stretch(g.ctx)
    S_g, S_o = g.field(m.F_CELL_STRETCH), o.field("S_ck")
    mask = o.field("V_ck") > 0
    ref = S_o[mask] - np.eye(3)
    err = np.linalg.norm(S_g[mask] - S_o[mask]) / max(np.linalg.norm(ref), 1e-30)
    if kind == "rest":
        # S = I: the absolute error in units of the FP32 / FP64 rounding of S
        assert np.max(np.abs(S_g[mask] - np.eye(3))) <= {m.FP32: 1e-6, m.FP64: 1e-14}[precision]
    else:
        assert err <= TOL[precision], err
    g.close()


def node_only_brick_scene(seed=9):
    """Particles filling cells 8..15 on every axis of a 32^3 grid: the DOF nodes of
    layer 16 live in bricks that contain no active cell (node-only bricks)."""
    n = 32
    sc = scenes.Scene("node_only", (n, n, n), 1.0 / n, float(n), 1e-3, (0.0, -9.8, 0.0),
                      [scenes.Material(scenes.NEO_HOOKEAN, 1e5, 0.3)])
    rng = np.random.default_rng(seed)
    x = rng.uniform(8.6 / n, 15.4 / n, (6000, 3))
    sc = scenes._finish(sc, x, 0.1 * rng.standard_normal((6000, 3)), np.zeros(6000, np.int64), 8)
    sc.F = np.eye(3) + 0.02 * rng.standard_normal(sc.F.shape)
    return sc


@pytest.mark.parametrize("precision", [m.FP32, m.FP64])
def test_hvp_and_solve_with_node_only_bricks(precision):
    sc = node_only_brick_scene()
    g, o, _ = both(sc, precision)
    keys = g.keys(m.KEYS_NODES)
    assert np.array_equal(keys, o.node_keys())
    assert (oracle.decode_keys(keys, sc.n) == 16).any()  # nodes in bricks without cells
    assert o.stretch() == 0
    m.mpml_stretch(g.ctx)
    nn = o.count("nodes")
    v = o.field("vhat")
    o.linearize(v)
    m.mpml_linearize(g.ctx, v)
    p = np.random.default_rng(1).standard_normal((nn, 3)).astype(g.npdt).astype(np.float64)
    check(m.mpml_hvp(g.ctx, p), o.hvp(p), TOL[precision], 'hvp')
    rc_o, st_o = o.newton(oracle.default_solver())
    rc, st = g.newton(m.solver_opts())
    assert rc == 0 and rc_o == 0
    # Jacobi-PCG iteration counts of the first Newton system agree closely
    assert abs(st.cg_iters[0] - st_o.cg_iters[0]) <= 2 + 0.02 * st_o.cg_iters[0]
    g.close()


@pytest.mark.parametrize("precision", [m.FP32, m.FP64])
def test_newton_step_solution(precision):
    sc = scenes.elastic_cube("stretched")
    g, o, _ = both(sc, precision)
    assert o.stretch() == 0
    rc_o, st_o = o.newton(oracle.default_solver())
    rc, st = g.newton(m.solver_opts())
    assert rc == 0 and rc_o == 0
    assert st.newton_iters >= 1
    v_g, v_o = g.field(m.F_NODE_VNEW), o.field("v_new")
    # both solves stop at relative residual 1e-6: the solutions agree to that order
    check(v_g - o.field("vhat"), v_o - o.field("vhat"), 1e-4, 'v_new - vhat')
    g.close()


@pytest.mark.parametrize("precision", [m.FP32, m.FP64])
def test_load_given_same_node_velocity(precision):
    sc = random_scene(6, count=3000)
    g, o, _ = both(sc, precision)
    nn = o.count("nodes")
    v = np.random.default_rng(7).standard_normal((nn, 3)).astype(g.npdt).astype(np.float64)
    o.set_node_velocity(v)
    m.mpml_set_node_velocity(g.ctx, v)
    rc, out = o.load()
    g.g2p()
    got = g.particles()
    tol = TOL[precision]
    check(g.field(m.F_CELL_VEL_NEW), o.field("v_c_new"), tol, 'v_c_new')
    check(g.field(m.F_CELL_VGRAD_NEW), o.field("G_c_new"), tol, 'G_c_new')
    for k in ("v", "G", "F"):
        check(got[k], out[k], tol, k)
    assert np.abs(got["x"] - out["x"]).max() <= (1e-6 if precision == m.FP32 else 1e-14)
    assert np.array_equal(got["mat"], out["mat"])
    g.close()


@pytest.mark.parametrize("variant", ["fall", "rest", "stretched"])
@pytest.mark.parametrize("precision", [m.FP64, m.FP32])
def test_ten_steps_positions(variant, precision):
    """Elastic cube of 8^3 voxels, 4096 particles, dt = 1e-3: positions after 10
    implicit steps within 1e-4 dx of the FP64 oracle."""
    sc = scenes.elastic_cube(variant)
    g = GpuSim(sc, precision)
    g.set_particles()
    o = OracleSim(make_oracle(sc), g.inputs())
    for s in range(10):
        rc, st_o = o.step(s * sc.dt)
        assert rc >= 0
        rc_g, st_g = g.step(s * sc.dt)
        assert rc_g >= 0
    got, ref = g.particles_by_identity(), o.particles_by_identity()
    err = np.abs(got["x"] - ref["x"]).max()
    assert err <= 1e-4 * sc.dx, err
    g.close()


def test_host_memory_path_matches_device():
    sc = scenes.elastic_cube("stretched")
    a = GpuSim(sc, m.FP32)
    a.set_particles()
    a.step()
    b = GpuSim(sc, m.FP32)
    b.set_particles(host=True)
    b.step()
    pa, pb = a.particles(), b.particles()
    for k in ("x", "v", "F", "G"):
        assert np.array_equal(pa[k], pb[k]) or rel_err(pb[k], pa[k]) < 1e-6, k
    assert np.array_equal(pa["perm"], pb["perm"])
    a.close()
    b.close()


def test_edge_cases():
    sc = random_scene(8, count=50)
    # empty particle set
    g = GpuSim(sc, m.FP32)
    g.set_particles({k: v[:0] for k, v in sc.particles(np.float32).items()})
    g.step()
    assert m.mpml_counts(g.ctx)["cells"] == 0
    g.close()
    # out of the grid / non-finite / bad material
    for mutate, code in ((lambda p: p["x"].__setitem__((3, 1), 0.5 / 16 - 1e-4), m.ERR_OUT_OF_DOMAIN),
                         (lambda p: p["x"].__setitem__((3, 1), np.nan), m.ERR_NONFINITE),
                         (lambda p: p["mat"].__setitem__(3, 7), m.ERR_ARG)):
        p = sc.particles(np.float32)
        mutate(p)
        g = GpuSim(sc, m.FP32)
        g.set_particles(p)
        with pytest.raises(m.MPMLError) as ei:
            g.resample()
            m.mpml_sync(g.ctx)
        assert ei.value.code == code
        g.close()
    # a single particle in a large sparse grid (many empty bricks)
    big = scenes.Scene("one", (256, 256, 256), 1 / 256, 256.0, 1e-3, (0, -9.8, 0),
                       [scenes.Material(scenes.FIXED_COROTATED, 1e5, 0.3)])
    big = scenes._finish(big, np.array([[0.5, 0.5, 0.5]]), np.zeros((1, 3)), np.zeros(1, np.int64), 8)
    g, o, _ = both(big, m.FP32)
    assert np.array_equal(g.keys(m.KEYS_CELLS), o.cell_keys())
    g.close()


def test_full_size_two_spheres():
    """Two Neo-Hookean spheres on 168^3 (~1.07M particles) at contact: bit-exact
    sets, unload fields, and the Newton solution satisfies the oracle's own
    optimality (its FP64 gradient at the GPU solution is small)."""
    sc = scenes.two_spheres(168, gap=1.0 / 168)
    g, o, _ = both(sc, m.FP32)
    assert np.array_equal(g.keys(m.KEYS_CELLS), o.cell_keys())
    assert np.array_equal(g.keys(m.KEYS_NODES), o.node_keys())
    for f, name in ((m.F_CELL_MASS, "m_c"), (m.F_NODE_MASS, "m_i"), (m.F_NODE_VEL, "v_i")):
        check(g.field(f), o.field(name), 1e-5, name)
    assert o.stretch() == 0
    m.mpml_stretch(g.ctx)
    # operator parity at full size, linearised at vhat
    vhat = o.field("vhat")
    phi_o, g_o = o.eval(vhat)
    phi_g, g_g = m.mpml_eval(g.ctx, vhat)
    check(g_g, g_o, 1e-5, 'gradient')
    o.linearize(vhat)
    p = np.random.default_rng(3).standard_normal(vhat.shape).astype(np.float32).astype(np.float64)
    check(m.mpml_hvp(g.ctx, p), o.hvp(p), 1e-5, 'hvp')
    rc, st = g.newton(m.solver_opts())
    assert rc == 0, (rc, st.newton_iters, list(st.cg_iters[:st.newton_iters]))
    v_g = g.field(m.F_NODE_VNEW)
    phi1, g1 = o.eval(v_g)
    assert phi1 <= phi_o
    # the oracle's own FP64 gradient at the GPU solution meets the Newton tolerance
    assert np.linalg.norm(g1) <= 2e-6 * np.linalg.norm(g_o)
    g.close()


def mixture_scene(nmat, seed=11, n=16, count=4000):
    """Random particles of nmat materials (all three models), so most cells mix them (Sec. 4.4)."""
    rng = np.random.default_rng(seed)
    mats = [scenes.Material(scenes.FIXED_COROTATED, 1e5, 0.3), scenes.Material(scenes.NEO_HOOKEAN, 3e4, 0.4, rho=2000.0),
            scenes.Material(scenes.HENCKY, 5e4, 0.25, rho=1500.0), scenes.Material(scenes.FIXED_COROTATED, 2e5, 0.35)]
    sc = scenes.Scene("mixture", (n, n, n), 1.0 / n, float(n), 1e-3, (0.0, -9.8, 0.0), mats[:nmat])
    x = rng.uniform(2.6 / n, 1 - 2.6 / n, (count, 3))
    sc.x = x
    sc.v = 0.1 * rng.standard_normal((count, 3))
    sc.G = 0.1 * rng.standard_normal((count, 3, 3))
    sc.F = np.eye(3) + 0.02 * rng.standard_normal((count, 3, 3))
    sc.Vp = np.full(count, sc.dx ** 3 / 8)
    sc.mat = rng.integers(0, nmat, count).astype(np.int32)
    sc.mp = np.array([mt.rho for mt in sc.materials])[sc.mat] * sc.Vp
    return sc


@pytest.mark.parametrize("precision,nmat", [(m.FP32, 4), (m.FP64, 3)])
def test_material_mixtures_up_to_the_slot_limit(precision, nmat):
    """Four materials in FP32 and three in FP64 (the P2Q shared-memory budget): unload fields,
    stretches, energy, gradient and HVP against the oracle."""
    sc = mixture_scene(nmat)
    g, o, _ = both(sc, precision)
    tol = TOL[precision]
    for f, name in [(m.F_CELL_VOL, "V_ck"), (m.F_CELL_TAU, "tau_ck"), (m.F_NODE_MASS, "m_i"), (m.F_NODE_VEL, "v_i")]:
        check(g.field(f), o.field(name), tol, name)
    assert o.stretch() == 0
    m.mpml_stretch(g.ctx)
    V = o.field("V_ck")
    mask = V > 0
    assert (mask.sum(axis=1) >= 3).any()  # cells that hold three or more materials
    S_g, S_o = g.field(m.F_CELL_STRETCH), o.field("S_ck")
    check(S_g[mask] - np.eye(3), S_o[mask] - np.eye(3), tol, 'S - I')
    nn = o.count("nodes")
    rng = np.random.default_rng(12)
    v = (o.field("vhat") + 0.05 * rng.standard_normal((nn, 3))).astype(g.npdt).astype(np.float64)
    phi_o, g_o = o.eval(v)
    phi_g, g_g = m.mpml_eval(g.ctx, v)
    assert abs(phi_g - phi_o) <= tol * abs(phi_o)
    check(g_g, g_o, tol, 'gradient')
    o.linearize(v, project=True)
    p = rng.standard_normal((nn, 3)).astype(g.npdt).astype(np.float64)
    check(m.mpml_hvp(g.ctx, p), o.hvp(p), tol, 'hvp')
    g.close()


@pytest.mark.parametrize("precision", [m.FP32, m.FP64])
def test_neo_hookean_energy_at_small_strain(precision):
    """Strains of 1e-6: the elastic energy is second order in the strain, and the
    line search near convergence compares energies of that size.  GPU against the
    oracle (both evaluate it without first-order cancellation): 1e-8 relative in FP64;
    in FP32 the FP32 transfers of the tiny stresses bound it (1e-5, the FP32 bound)."""
    sc = node_only_brick_scene(seed=12)
    rng = np.random.default_rng(13)
    sc.F = np.eye(3) + 1e-6 * rng.standard_normal(sc.F.shape)
    sc.v = np.zeros_like(sc.v)
    sc.G = np.zeros_like(sc.G)
    g, o, _ = both(sc, precision)
    assert o.stretch() == 0
    m.mpml_stretch(g.ctx)
    nn = o.count("nodes")
    v = (o.field("vhat") + 1e-7 * rng.standard_normal((nn, 3))).astype(g.npdt).astype(np.float64)
    phi_o, _ = o.eval(v)
    phi_g, _ = m.mpml_eval(g.ctx, v)
    assert phi_o > 0
    tol = 1e-8 if precision == m.FP64 else 1e-5
    assert abs(phi_g - phi_o) <= tol * abs(phi_o), (phi_g, phi_o)
    g.close()
