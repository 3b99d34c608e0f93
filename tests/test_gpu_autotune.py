"""HVP launch-shape autotuner on the GPU: every launch shape of both tangent
formats against the FP64 oracle's HVP (norm-relative 1e-5, the FP32 HVP bound),
the tuner's choice (the fastest measured shape, recorded in the cache), and a
graph-driven Newton solve that picks its shape automatically and agrees with
the persistent solver."""
import numpy as np
import pytest
import torch

import paper_2602_07853_gb300.mpml as m
from paper_2602_07853_gb300 import scenes
from tests._util import make_oracle
from tests._gpu import GpuSim, check

pytestmark = pytest.mark.gpu


@pytest.fixture(autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.set_device(0)
    m.mpml_tile_cache_clear()
    yield
    m.mpml_tile_cache_clear()


def scene(kind, seed=21, count=6000, n=24):
    rng = np.random.default_rng(seed)
    mats = [scenes.Material(scenes.FIXED_COROTATED, 1e5, 0.3)]
    if kind == "k45":
        mats.append(scenes.Material(scenes.NEO_HOOKEAN, 3e4, 0.4, rho=2000.0))
    sc = scenes.Scene(kind, (n, n, n), 1.0 / n, float(n), 1e-3, (0.0, -9.8, 0.0), mats)
    x = rng.uniform(1.6 / n, 1 - 1.6 / n, (count, 3))
    sc = scenes._finish(sc, x, 0.1 * rng.standard_normal((count, 3)),
                        rng.integers(0, len(mats), count).astype(np.int64), 8)
    sc.F = np.eye(3) + 0.03 * rng.standard_normal(sc.F.shape)
    return sc


@pytest.mark.parametrize("kind", ["cmp", "k45"])
def test_every_tile_matches_the_oracle_and_the_tuner_picks_the_fastest(kind, tmp_path):
    sc = scene(kind)
    g = GpuSim(sc, m.FP32)
    inp = g.inputs()
    g.set_particles()
    o = make_oracle(sc)
    assert o.unload(**inp) == 0
    g.resample()
    assert o.stretch() == 0
    m.mpml_stretch(g.ctx)
    nn = o.count("nodes")
    rng = np.random.default_rng(22)
    v = (o.field("vhat") + 0.05 * rng.standard_normal((nn, 3))).astype(np.float32).astype(np.float64)
    o.linearize(v, project=True)
    m.mpml_linearize(g.ctx, v)
    p = rng.standard_normal((nn, 3)).astype(np.float32).astype(np.float64)
    want = o.hvp(p)
    for t in range(m.HVP_TILES):
        m.mpml_set_hvp_tile(g.ctx, t)
        tile, desc = m.mpml_get_hvp_tile(g.ctx)
        assert tile == t and desc
        check(m.mpml_hvp(g.ctx, p), want, 1e-5, (t, desc))
    m.mpml_set_hvp_tile(g.ctx, -1)
    tile, ms = m.mpml_autotune_hvp(g.ctx, 3)
    assert 0 <= tile < m.HVP_TILES
    assert all(t > 0 for t in ms) and ms[tile] == min(ms)
    assert m.mpml_get_hvp_tile(g.ctx)[0] == tile
    # the autotuner leaves the linearisation and the solver vectors usable
    check(m.mpml_hvp(g.ctx, p), want, 1e-5, 'hvp')
    path = tmp_path / "tiles.txt"
    m.mpml_tile_cache_save(path)
    rows = [l.split() for l in open(path)]
    assert len(rows) == 1 and int(rows[0][0]) == (25 if kind == "cmp" else 45) and int(rows[0][2]) == tile
    g.close()


def test_graph_solve_autotunes_and_matches_the_persistent_solver():
    sc = scenes.two_spheres(48, gap=1.0 / 48)
    a, b = GpuSim(sc, m.FP32), GpuSim(sc, m.FP32)
    for s in (a, b):
        s.set_particles()
        s.resample()
    assert m.mpml_get_hvp_tile(a.ctx)[0] == -1
    rc_a, st_a = a.newton(m.solver_opts(use_graph=1))
    rc_b, st_b = b.newton(m.solver_opts(use_graph=2))
    assert rc_a == 0 and rc_b == 0
    tile, _ = m.mpml_get_hvp_tile(a.ctx)
    assert 0 <= tile < m.HVP_TILES  # chosen on the first graph-driven solve
    va, vb = a.field(m.F_NODE_VNEW), b.field(m.F_NODE_VNEW)
    vhat = a.field(m.F_NODE_VHAT)
    check(va - vhat, vb - vhat, 1e-4, 'v_new - vhat')
    # a second context of the same format and size takes the cached choice
    c = GpuSim(sc, m.FP32)
    c.set_particles()
    c.resample()
    rc_c, _ = c.newton(m.solver_opts(use_graph=1))
    assert rc_c == 0 and m.mpml_get_hvp_tile(c.ctx)[0] == tile
    for s in (a, b, c):
        s.close()
