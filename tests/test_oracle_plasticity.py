"""Pins for the oracle's plastic return maps (CPU only).

Independent of the oracle's SVD: principal stretches from numpy's eigh of
F^T F, rotations from scipy's polar decomposition.  Checked: admissible states
are untouched; returned states lie on the yield surface with the volumetric
strain and the polar rotation kept; a closed-form von Mises case; the
Drucker-Prager apex for tension; idempotence.
"""
import numpy as np
import pytest
from scipy.linalg import polar

import oracle

MU, LAM = oracle.lame(5e5, 0.3)


def hencky(F):
    """Principal Hencky strains (ascending by eigh) and the right stretch basis."""
    w, V = np.linalg.eigh(F.T @ F)
    return 0.5 * np.log(w), V


def kirchhoff_principal(eps):
    return 2 * MU * eps + LAM * eps.sum()


def rot(seed):
    q, _ = np.linalg.qr(np.random.default_rng(seed).standard_normal((3, 3)))
    return q * np.sign(np.linalg.det(q))


def make_F(eps, seed):
    R, Q = rot(seed), rot(seed + 100)
    return R @ Q @ np.diag(np.exp(eps)) @ Q.T  # rotation R, symmetric stretch along Q


def dev_norm(tau):
    return np.linalg.norm(tau - tau.mean())


@pytest.mark.parametrize("seed", range(4))
def test_von_mises_inside_is_unchanged(seed):
    sy = 2e3
    F = make_F(np.array([1e-4, -5e-4, 2e-4]), seed)
    kind, Fn = oracle.return_map(oracle.VON_MISES, MU, LAM, sy, 0.0, F)
    assert kind == 0 and np.array_equal(Fn, F)


@pytest.mark.parametrize("seed", range(4))
def test_von_mises_return_lies_on_the_surface(seed):
    sy = 2e3
    eps = np.array([0.03, -0.01, -0.005])
    F = make_F(eps, seed)
    kind, Fn = oracle.return_map(oracle.VON_MISES, MU, LAM, sy, 0.0, F)
    assert kind == 1
    e_new, _ = hencky(Fn)
    tau = kirchhoff_principal(e_new)
    assert abs(dev_norm(tau) - np.sqrt(2 / 3) * sy) <= 1e-9 * sy
    assert abs(e_new.sum() - eps.sum()) <= 1e-12          # volume kept
    assert np.allclose(polar(Fn)[0], polar(F)[0], atol=1e-12)  # rotation kept
    kind2, Fn2 = oracle.return_map(oracle.VON_MISES, MU, LAM, sy, 0.0, Fn)
    assert kind2 == 0 or np.allclose(Fn2, Fn, atol=1e-14)  # idempotent


def test_von_mises_closed_form_pure_shear():
    """eps = (a, -a, 0): radial return gives (t, -t, 0) / sqrt(2) with
    t = sqrt(2/3) sigma_y / (2 mu), i.e. F = diag(e^(t/sqrt2), e^(-t/sqrt2), 1)."""
    sy, a = 2e3, 0.05
    F = np.diag([np.exp(a), np.exp(-a), 1.0])
    kind, Fn = oracle.return_map(oracle.VON_MISES, MU, LAM, sy, 0.0, F)
    t = np.sqrt(2 / 3) * sy / (2 * MU)
    assert kind == 1
    assert np.allclose(Fn, np.diag([np.exp(t / np.sqrt(2)), np.exp(-t / np.sqrt(2)), 1.0]), atol=1e-14)


@pytest.mark.parametrize("seed", range(3))
def test_drucker_prager_tension_goes_to_the_apex(seed):
    F = make_F(np.array([0.02, 0.01, -0.005]), seed)  # tr(eps) > 0
    kind, Fn = oracle.return_map(oracle.DRUCKER_PRAGER, MU, LAM, 0.0, np.radians(30), F)
    assert kind == 2
    assert np.allclose(Fn, polar(F)[0], atol=1e-12)  # stretch-free: the rotation alone


def test_drucker_prager_hydrostatic_compression_is_admissible():
    F = 0.97 * rot(7)
    kind, Fn = oracle.return_map(oracle.DRUCKER_PRAGER, MU, LAM, 0.0, np.radians(30), F)
    assert kind == 0 and np.array_equal(Fn, F)


@pytest.mark.parametrize("seed", range(4))
def test_drucker_prager_cone_return(seed):
    phi = np.radians(30)
    sp = np.sin(phi)
    alpha = np.sqrt(2 / 3) * 2 * sp / (3 - sp)
    eps = np.array([0.02, -0.03, -0.01])  # compressive, strong shear
    F = make_F(eps, seed)
    tau0 = kirchhoff_principal(hencky(F)[0])
    assert dev_norm(tau0) + alpha * tau0.sum() > 0  # outside the cone
    kind, Fn = oracle.return_map(oracle.DRUCKER_PRAGER, MU, LAM, 0.0, phi, F)
    assert kind == 3
    e_new, _ = hencky(Fn)
    tau = kirchhoff_principal(e_new)
    assert abs(dev_norm(tau) + alpha * tau.sum()) <= 1e-9 * abs(tau.sum())  # on the cone
    assert abs(e_new.sum() - eps.sum()) <= 1e-12
    assert np.allclose(polar(Fn)[0], polar(F)[0], atol=1e-12)
    kind2, Fn2 = oracle.return_map(oracle.DRUCKER_PRAGER, MU, LAM, 0.0, phi, Fn)
    assert kind2 == 0 or np.allclose(Fn2, Fn, atol=1e-14)


def test_load_applies_the_map_per_material():
    """A particle of a von Mises material with a large shear F comes out of Load on the
    yield surface; an elastic material's particle keeps its updated F."""
    n = 16
    mats = [(oracle.HENCKY, 5e5, 0.3), (oracle.HENCKY, 5e5, 0.3, oracle.VON_MISES, 2e3, 0.0)]
    o = oracle.Oracle(oracle.make_scene(n, 1.0 / n, 1e-3, (0.0, 0.0, 0.0), mats))
    x = np.array([[0.41, 0.52, 0.47], [0.63, 0.38, 0.55]])
    F = np.stack([np.diag([np.exp(0.05), np.exp(-0.05), 1.0])] * 2)
    p = dict(x=x, v=np.zeros((2, 3)), F=F.reshape(2, 9), G=np.zeros((2, 9)), mp=np.ones(2) * 1e-3,
             Vp=np.ones(2) * 1e-6, mat=np.array([0, 1], np.int32))
    assert o.unload(**p) == 0
    assert o.stretch() == 0
    o.set_node_velocity(np.zeros((o.count("nodes"), 3)))
    rc, res = o.load()
    assert rc == 0
    Fo = res["F"].reshape(-1, 3, 3)
    mat = res["mat"]
    t = np.sqrt(2 / 3) * 2e3 / (2 * MU)
    assert np.allclose(Fo[mat == 0][0], F[0], atol=1e-14)
    assert np.allclose(Fo[mat == 1][0], np.diag([np.exp(t / np.sqrt(2)), np.exp(-t / np.sqrt(2)), 1.0]),
                       atol=1e-12)
