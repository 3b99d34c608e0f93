"""Pins for the oracle's Unload (Algorithm 2) and Load (Algorithm 4) (CPU only).

Against: brute-force binning in numpy; the partition-of-unity / linear
reproduction identities of App. A (affine fields are transferred exactly);
conservation of mass, momentum and extensive stress (Sec. 3.2); the
hourglass filter of Sec. 7.
"""
import numpy as np
import pytest

import oracle
from paper_2602_07853_gb300 import scenes
from tests._util import brute_force_sets, make_oracle


def small_scene(seed=0, n=16, count=300):
    """A few hundred random particles in a 16^3 grid, several 8^3 bricks, random v/G/F."""
    rng = np.random.default_rng(seed)
    sc = scenes.Scene("random", (n, n, n), 1.0 / n, float(n), 1e-3, (0.0, -9.8, 0.0),
                      [scenes.Material(scenes.FIXED_COROTATED, 1e5, 0.3),
                       scenes.Material(scenes.NEO_HOOKEAN, 3e4, 0.4, rho=2000.0)])
    x = rng.uniform(1.6 / n, 1 - 1.6 / n, (count, 3))
    # a few particles exactly on centre lines (f == 0) to exercise the active rule
    x[:10, 0] = (np.floor(x[:10, 0] * n) + 0.5) / n
    sc.x = x
    sc.v = rng.standard_normal((count, 3))
    sc.G = rng.standard_normal((count, 3, 3))
    sc.F = np.eye(3) + 0.05 * rng.standard_normal((count, 3, 3))
    sc.Vp = np.full(count, sc.dx ** 3 / 8)
    sc.mat = rng.integers(0, 2, count).astype(np.int32)
    sc.mp = np.array([1000.0, 2000.0])[sc.mat] * sc.Vp
    return sc


def test_sort_and_active_sets_brute_force():
    sc = small_scene()
    o = make_oracle(sc)
    assert o.unload(**sc.particles()) == 0
    keys, perm, ckeys, nkeys = brute_force_sets(sc.x, sc.inv_dx, sc.n)
    assert np.array_equal(o.particle_keys(), keys)
    assert np.array_equal(o.perm(), perm)
    assert np.array_equal(o.cell_keys(), ckeys)
    assert np.array_equal(o.node_keys(), nkeys)


def test_out_of_domain_rejected():
    sc = small_scene(count=20)
    sc.x[3, 1] = 0.5 / 16 - 1e-9  # base centre index -1
    o = make_oracle(sc)
    assert o.unload(**sc.particles()) == oracle.ERR_OUT_OF_DOMAIN
    sc.x[3, 1] = np.nan
    assert make_oracle(sc).unload(**sc.particles()) == oracle.ERR_NONFINITE


def test_affine_field_reproduced_exactly():
    """v(x) = a + B x with G_p = B: the kinematic unload gives v_c = a + B x_c,
    G_c = B, and the centre-to-node gather v_i = a + B x_i (linear reproduction)."""
    sc = small_scene(1)
    rng = np.random.default_rng(2)
    a, B = rng.standard_normal(3), rng.standard_normal((3, 3))
    sc.v = a + sc.x @ B.T
    sc.G = np.tile(B, (sc.num_particles, 1, 1))
    o = make_oracle(sc)
    assert o.unload(**sc.particles()) == 0
    xc = (oracle.decode_keys(o.cell_keys(), sc.n) + 0.5) * sc.dx
    xi = oracle.decode_keys(o.node_keys(), sc.n) * sc.dx
    assert np.allclose(o.field("v_c"), a + xc @ B.T, atol=1e-12)
    assert np.allclose(o.field("G_c"), B, atol=1e-12)
    assert np.allclose(o.field("v_i"), a + xi @ B.T, atol=1e-12)


def test_unload_conserves_mass_momentum_stress():
    sc = small_scene(3)
    o = make_oracle(sc)
    assert o.unload(**sc.particles()) == 0
    m_c, v_c = o.field("m_c"), o.field("v_c")
    m_i, v_i = o.field("m_i"), o.field("v_i")
    P = (sc.mp[:, None] * sc.v).sum(0)
    assert np.isclose(m_c.sum(), sc.mp.sum(), rtol=1e-13)
    assert np.allclose((m_c[:, None] * v_c).sum(0), P, atol=1e-13 * np.abs(sc.mp[:, None] * sc.v).sum())
    assert np.isclose(m_i.sum(), m_c.sum(), rtol=1e-13)
    assert np.allclose((m_i[:, None] * v_i).sum(0), P, atol=1e-13 * np.abs(sc.mp[:, None] * sc.v).sum())
    # sum_c V_c tau_c = sum_p V_p tau_p per material (Sec. 3.2)
    V_ck, tau_ck = o.field("V_ck"), o.field("tau_ck")
    sc_o = o.scene
    for k in range(2):
        ref = np.zeros((3, 3))
        for p in np.nonzero(sc.mat == k)[0]:
            ref += sc.Vp[p] * oracle.kirchhoff(sc_o.model[k], sc_o.mu[k], sc_o.lam[k], sc.F[p])
        got = (V_ck[:, k, None, None] * tau_ck[:, k]).sum(0)
        assert np.allclose(got, ref, rtol=1e-12, atol=1e-12 * np.abs(ref).max())
        assert np.isclose(V_ck[:, k].sum(), sc.Vp[sc.mat == k].sum(), rtol=1e-13)


def test_load_reproduces_affine_node_field():
    """Nodal v_i = a + B x_i: v_c = a + B x_c, G_c = B, then v_p = a + B x_p, G_p = B,
    x += dt v_p and F <- (I + dt B) F (Algorithm 4)."""
    sc = small_scene(4)
    o = make_oracle(sc)
    assert o.unload(**sc.particles()) == 0
    rng = np.random.default_rng(5)
    a, B = rng.standard_normal(3), rng.standard_normal((3, 3))
    xi = oracle.decode_keys(o.node_keys(), sc.n) * sc.dx
    o.set_node_velocity(a + xi @ B.T)
    rc, out = o.load()
    assert rc == 0
    perm = o.perm()
    x0, F0 = sc.x[perm], sc.F[perm]
    xc = (oracle.decode_keys(o.cell_keys(), sc.n) + 0.5) * sc.dx
    assert np.allclose(o.field("v_c_new"), a + xc @ B.T, atol=1e-12)
    assert np.allclose(o.field("G_c_new"), B, atol=1e-11)
    assert np.allclose(out["v"], a + x0 @ B.T, atol=1e-12)
    assert np.allclose(out["G"], B, atol=1e-11)
    assert np.allclose(out["x"], x0 + sc.dt * (a + x0 @ B.T), atol=1e-14)
    assert np.allclose(out["F"], np.einsum("ij,pjk->pik", np.eye(3) + sc.dt * B, F0), atol=1e-13)
    assert np.array_equal(out["mat"], sc.mat[perm])


def test_hourglass_mode_filtered():
    """v_i = (-1)^(i+j+k) e gives v_c = 0 and G_c = 0 at every centre (Sec. 7)."""
    sc = small_scene(6)
    o = make_oracle(sc)
    assert o.unload(**sc.particles()) == 0
    ijk = oracle.decode_keys(o.node_keys(), sc.n)
    sgn = (-1.0) ** ijk.sum(1)
    o.set_node_velocity(np.outer(sgn, [0.3, -1.2, 2.0]))
    o.load()
    assert np.abs(o.field("v_c_new")).max() < 1e-14
    assert np.abs(o.field("G_c_new")).max() < 1e-10


def test_load_conserves_momentum():
    """sum_p m_p v_p^{n+1} = sum_i m_i v_i^{n+1} for any nodal field."""
    sc = small_scene(7)
    o = make_oracle(sc)
    assert o.unload(**sc.particles()) == 0
    rng = np.random.default_rng(8)
    v = rng.standard_normal((o.count("nodes"), 3))
    o.set_node_velocity(v)
    rc, out = o.load()
    m_i = o.field("m_i")
    assert np.allclose((out["mp"][:, None] * out["v"]).sum(0), (m_i[:, None] * v).sum(0),
                       atol=1e-13 * np.abs(m_i[:, None] * v).sum())
