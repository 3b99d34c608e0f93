"""Pins for the oracle's explicit integrator (CPU only).

Against: free fall (no stress: v^{n+1} = v^n + dt g exactly, positions follow the
discrete free-fall law); linear-momentum balance of the internal force (the
forces of every cell sum to zero, so sum m v changes only by dt g sum m when no
node is fixed); a uniform stretch field (interior nodes feel no force); the
implicit step's gradient at G = 0 (dt times the explicit force is minus the
elastic gradient, App. B), i.e. one explicit step equals one Newton-free update
from the same stress.
"""
import numpy as np

import oracle
from paper_2602_07853_gb300 import scenes
from tests._util import make_oracle


def test_free_fall_is_exact():
    sc = scenes.elastic_cube("fall")
    o = make_oracle(sc)
    p = {k: (v.astype(np.float64) if k != "mat" else v) for k, v in sc.particles().items()}
    y0 = p["x"][:, 1].mean()
    for k in range(5):
        o.set_time(k * sc.dt)
        rc, p = o.explicit_step(p)
        assert rc == 0
    y = p["x"][:, 1].mean()
    n = 5
    assert abs(y - (y0 + 0.5 * sc.gravity[1] * sc.dt ** 2 * n * (n + 1))) < 1e-12
    assert np.allclose(p["v"][:, 1], n * sc.dt * sc.gravity[1], atol=1e-12)


def test_internal_forces_balance_linear_momentum():
    """Stretched cube away from walls: the internal force changes no momentum."""
    sc = scenes.elastic_cube("stretched")
    sc.gravity = (0.0, 0.0, 0.0)
    o = make_oracle(sc)
    p = {k: (v.astype(np.float64) if k != "mat" else v) for k, v in sc.particles().items()}
    assert o.unload(**p) == 0
    f = np.zeros((o.count("nodes"), 3))
    oracle.lib().orc_explicit_force(o._h, oracle._dp(f))
    assert np.abs(f).max() > 1e-3                      # the stretch does load the nodes
    assert np.abs(f.sum(axis=0)).max() < 1e-10 * np.abs(f).sum()
    o.explicit()
    m = o.field("m_i")[:, None]
    fixed = o.field("fixed") > 0
    assert not fixed[m[:, 0] > 0].any()               # no loaded node is on a wall
    assert np.allclose((m * o.field("v_new")).sum(axis=0), (m * o.field("v_i")).sum(axis=0), atol=1e-14)


def test_explicit_force_is_minus_the_elastic_gradient_over_dt():
    """At G = 0 (v = vhat with vhat uniform) F_c = S_c, so dt f_i = -(g_i - m_i (v_i - vhat_i))
    with S reconstructed from the same stress (Sec. 4.2)."""
    sc = scenes.elastic_cube("stretched")
    sc.gravity = (0.0, 0.0, 0.0)
    sc.wall_layers = 0
    o = make_oracle(sc)
    p = {k: (v.astype(np.float64) if k != "mat" else v) for k, v in sc.particles().items()}
    p["v"][:] = 0.0
    assert o.unload(**p) == 0
    assert o.stretch() == 0
    vhat = o.field("vhat")
    _, g = o.eval(vhat)
    f = np.zeros_like(g)
    oracle.lib().orc_explicit_force(o._h, oracle._dp(f))
    fixed = o.field("fixed") > 0
    assert np.allclose(sc.dt * f[~fixed], -g[~fixed], rtol=1e-8, atol=1e-12 * np.abs(g).max())
