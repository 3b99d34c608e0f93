"""Learned preconditioner: CUDA (BF16 tensor-core convolutions) vs the FP64 oracle.

Tolerances: BF16 keeps 8 significant bits, so one product carries a relative
rounding of 2^-9 ~ 2e-3; the three layers and the sums over 27 taps x 16
channels give an expected norm-relative error of ~1e-2 for the network
correction and its weight gradients.  Bounds below: 3e-2 (application, loss),
6e-2 (gradients).
"""
import numpy as np
import pytest
import torch

import oracle
from oracle import nn as onn
import paper_2602_07853_gb300.mpml as m
from paper_2602_07853_gb300 import scenes
from tests._gpu import GpuSim, check
from tests._util import make_oracle

pytestmark = pytest.mark.gpu


@pytest.fixture(autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.set_device(0)


def linearized_pair(sc):
    """GPU (FP32) and oracle, unloaded, stretched and linearised at vhat."""
    g = GpuSim(sc, m.FP32)
    inp = g.inputs()
    g.set_particles()
    g.resample()
    o = make_oracle(sc)
    assert o.unload(**inp) == 0
    assert o.stretch() == 0
    m.mpml_stretch(g.ctx)
    vhat = o.field("vhat")
    o.linearize(vhat)
    m.mpml_linearize(g.ctx, vhat)
    return g, o, vhat


def dense(o, sc, values):
    ijk = oracle.decode_keys(o.node_keys(), sc.n)
    shape = tuple(np.array(sc.n) + 1)
    return onn.to_grid(values, ijk, shape), ijk, shape


def masks(o, sc):
    fixed = o.field("fixed")
    ones = np.ones((len(fixed), 1))
    dof, ijk, shape = dense(o, sc, ones)
    free, _, _ = dense(o, sc, (1 - fixed)[:, None])
    return dof[..., 0], free[..., 0], ijk, shape


def small_scene():
    sc = scenes.elastic_cube("stretched")
    return sc


def test_apply_matches_oracle():
    sc = small_scene()
    g, o, vhat = linearized_pair(sc)
    dof, free, ijk, shape = masks(o, sc)
    d = o.diag()
    dinv = np.where(d > 0, 1.0 / np.where(d > 0, d, 1), 0.0)
    Ws = m.nn_init_weights(3)
    Ws32 = [np.asarray(W, np.float32).astype(np.float64) for W in Ws]
    m.mpml_nn_set_weights(g.ctx, Ws)
    rng = np.random.default_rng(4)
    r = (rng.standard_normal(vhat.shape) * (d > 0)).astype(np.float32).astype(np.float64)
    z_gpu = m.mpml_nn_apply(g.ctx, r)
    zg, _, _ = dense(o, sc, r)
    dg, _, _ = dense(o, sc, dinv)
    z_or, _ = onn.precondition(zg, dg, Ws32, dof, free)
    z_or = onn.from_grid(z_or, ijk)
    jac = dinv * r
    check(z_gpu - jac, z_or - jac, 3e-2, 'network correction')
    check(z_gpu, z_or, 1e-2, 'z')
    # returned weights are the ones set (FP32 master copy)
    back = m.mpml_nn_get_weights(g.ctx)
    for a, b in zip(back, Ws32):
        assert np.array_equal(a, b)
    g.close()


def test_loss_and_gradient_match_oracle():
    sc = small_scene()
    g, o, vhat = linearized_pair(sc)
    dof, free, ijk, shape = masks(o, sc)
    d = o.diag()
    dinv = np.where(d > 0, 1.0 / np.where(d > 0, d, 1), 0.0)
    Ws = m.nn_init_weights(5, gain=0.5)
    Ws32 = [np.asarray(W, np.float32).astype(np.float64) for W in Ws]
    m.mpml_nn_set_weights(g.ctx, Ws)
    rng = np.random.default_rng(6)
    r = (rng.standard_normal(vhat.shape) * (d > 0)).astype(np.float32).astype(np.float64)
    e = (rng.standard_normal(vhat.shape) * (d > 0)).astype(np.float32).astype(np.float64)
    loss_g, grads_g = m.mpml_nn_loss_grad(g.ctx, r, e)

    def hvp_grid(vg):
        return onn.to_grid(o.hvp(onn.from_grid(vg, ijk)), ijk, shape)

    rg, _, _ = dense(o, sc, r)
    eg, _, _ = dense(o, sc, e)
    dg, _, _ = dense(o, sc, dinv)
    loss_o, grads_o = onn.loss_and_grad(rg, eg, dg, Ws32, dof, free, hvp_grid)
    assert abs(loss_g - loss_o) <= 3e-2 * abs(loss_o)
    for l in range(3):
        check(grads_g[l], grads_o[l], 6e-2, l)
    g.close()


def test_zero_network_fcg_equals_jacobi_pcg():
    """Flexible CG with NN = 0 is Jacobi-PCG (a fixed symmetric preconditioner)."""
    sc = scenes.two_spheres(64, gap=1.0 / 64)
    g = GpuSim(sc, m.FP32)
    g.set_particles()
    g.resample()
    rc_j, st_j = g.newton(m.solver_opts(newton_max=2))
    m.mpml_nn_set_weights(g.ctx, [np.zeros(s) for s in m.NN_SHAPES])
    g.resample()
    rc_l, st_l = g.newton(m.solver_opts(newton_max=2, precond=m.PRECOND_LEARNED))
    assert st_l.fcg_fallbacks == 0
    for k in range(st_j.newton_iters):
        assert abs(st_l.cg_iters[k] - st_j.cg_iters[k]) <= 2, (list(st_l.cg_iters[:2]), list(st_j.cg_iters[:2]))
    assert abs(st_l.g_norm - st_j.g_norm) <= 1e-3 * st_j.g0_norm
    g.close()


def test_training_reduces_loss_and_learned_solve_converges():
    sc = scenes.two_spheres(64, gap=1.0 / 64)
    g = GpuSim(sc, m.FP32)
    g.set_particles()
    g.resample()
    rc_j, st_j = g.newton(m.solver_opts())
    m.mpml_nn_set_weights(g.ctx, m.nn_init_weights(7, gain=0.1))
    g.resample()
    tr = m.mpml_nn_train(g.ctx, m.train_opts(samples=16, epochs=10, batch=4, lr=2e-3))
    assert tr.samples == 16
    assert tr.loss_last < tr.loss_first
    g.resample()
    rc_l, st_l = g.newton(m.solver_opts(precond=m.PRECOND_LEARNED))
    assert rc_l == 0
    # the converged Newton solution does not depend on the preconditioner
    assert st_l.g_norm <= 1e-6 * st_l.g0_norm
    print(f"Jacobi-PCG CG iterations {st_j.cg_iters_total}, learned FCG {st_l.cg_iters_total}, "
          f"fallbacks {st_l.fcg_fallbacks}, loss {tr.loss_first:.3f} -> {tr.loss_last:.3f}")
    g.close()


def test_trained_network_gains_over_jacobi_on_an_unseen_system():
    """What the trained network gains over the method without it: on residual / error pairs
    of a Newton system it was not trained on (the next time step), its preconditioned
    residual is closer to the error in the H-angle than the Jacobi one (lower mean loss
    1 - cos_H).  Wall-clock is reported by bench.py (learned_precond)."""
    sc = scenes.two_spheres(64, gap=1.0 / 64)
    g = GpuSim(sc, m.FP32)
    g.set_particles()
    g.resample()
    m.mpml_nn_set_weights(g.ctx, m.nn_init_weights(7, gain=0.1))
    m.mpml_nn_train(g.ctx, m.train_opts(samples=32, epochs=20, batch=4, lr=1e-3))
    trained = m.mpml_nn_get_weights(g.ctx)
    # advance one time step with plain Jacobi-PCG, then look at the next Newton system
    g.resample()
    rc, st = g.newton(m.solver_opts())
    assert rc == 0
    g.g2p()
    m.mpml_set_time(g.ctx, sc.dt)
    g.resample()
    ev_learned = m.mpml_nn_train(g.ctx, m.train_opts(samples=16, epochs=1, batch=4, lr=0.0))
    m.mpml_nn_set_weights(g.ctx, [np.zeros(s) for s in m.NN_SHAPES])
    ev_jacobi = m.mpml_nn_train(g.ctx, m.train_opts(samples=16, epochs=1, batch=4, lr=0.0))
    back = m.mpml_nn_get_weights(g.ctx)
    assert all(np.array_equal(b, np.zeros_like(b)) for b in back)  # evaluation left the weights alone
    print(f"unseen system: mean 1 - cos_H  learned {ev_learned.loss_first:.4f}  Jacobi {ev_jacobi.loss_first:.4f}")
    assert ev_learned.loss_first < ev_jacobi.loss_first
    del trained
    g.close()


def test_adam_step_on_caller_pairs():
    """mpml_nn_adam_step applies the gradient of mpml_nn_loss_grad and zeroes it; a few steps
    on one pair lower that pair's loss."""
    sc = small_scene()
    g, o, vhat = linearized_pair(sc)
    m.mpml_nn_set_weights(g.ctx, m.nn_init_weights(5, gain=0.5))
    rng = np.random.default_rng(9)
    d = o.diag()
    r = rng.standard_normal(vhat.shape) * (d > 0)
    e = rng.standard_normal(vhat.shape) * (d > 0)
    l0, grad0 = m.mpml_nn_loss_grad(g.ctx, r, e)
    w0 = m.mpml_nn_get_weights(g.ctx)
    m.mpml_nn_adam_step(g.ctx, 1e-3)
    assert all(np.abs(x).max() == 0 for x in m.mpml_nn_get_grad(g.ctx))
    assert any(not np.array_equal(a, b) for a, b in zip(w0, m.mpml_nn_get_weights(g.ctx)))
    for _ in range(20):
        m.mpml_nn_loss_grad(g.ctx, r, e)
        m.mpml_nn_adam_step(g.ctx, 1e-3)
    l1, _ = m.mpml_nn_loss_grad(g.ctx, r, e)
    assert l1 < l0
    g.close()
