"""Pins for the oracle's water model (Sec. "Water"; CPU only).

Checked against things other than the model's own formulas: the energy and the
Kirchhoff stress depend on det F only (rotations and isochoric stretches leave
them unchanged), the pressure equals J dpsi/dJ by central differences of the
energy along J, the stretch reconstruction inverts the stress (and picks the
J >= 1/2 root, which carries the same pressure as its mirror 1 - J), and the
particle update of Load follows the divergence of an affine node velocity field
(linear reproduction gives G_c exactly).
"""
import numpy as np
import pytest

import oracle

E, NU = 2e5, 0.45
MU, LAM = oracle.lame(E, NU)
KAP = LAM + 2.0 / 3.0 * MU
W = oracle.WATER


def rand_rot(rng):
    q, r = np.linalg.qr(rng.standard_normal((3, 3)))
    q = q @ np.diag(np.sign(np.diag(r)))
    if np.linalg.det(q) < 0:
        q[:, 0] = -q[:, 0]
    return q


def iso(J):
    return np.cbrt(J) * np.eye(3)


@pytest.mark.parametrize("seed", range(5))
def test_energy_and_stress_depend_on_J_only(seed):
    rng = np.random.default_rng(seed)
    a, b = np.exp(rng.uniform(-0.3, 0.3, 2))
    J = rng.uniform(0.6, 1.5)
    F = rand_rot(rng) @ np.diag([a, b, J / (a * b)]) @ rand_rot(rng).T  # det F = J
    assert np.isclose(np.linalg.det(F), J)
    psi = oracle.psi(W, MU, LAM, F)
    assert psi == pytest.approx(oracle.psi(W, MU, LAM, iso(J)), rel=1e-12, abs=1e-12 * KAP)
    tau = oracle.kirchhoff(W, MU, LAM, F)
    # isotropic: no shear strength
    assert np.allclose(tau, np.trace(tau) / 3 * np.eye(3), atol=1e-9 * KAP)
    # pressure = J dpsi/dJ (central difference of psi along J at fixed isochoric part)
    h = 1e-6
    dpsi = (oracle.psi(W, MU, LAM, iso(J + h)) - oracle.psi(W, MU, LAM, iso(J - h))) / (2 * h)
    assert np.trace(tau) / 3 == pytest.approx(J * dpsi, rel=1e-7, abs=1e-7 * KAP)


def test_energy_is_zero_at_rest_and_undefined_when_inverted():
    assert oracle.psi(W, MU, LAM, np.eye(3)) == 0.0
    assert not np.isfinite(oracle.psi(W, MU, LAM, np.diag([1.0, 1.0, -0.5])))


@pytest.mark.parametrize("J", [0.55, 0.8, 1.0, 1.25, 2.0])
def test_stretch_reconstruction_inverts_the_pressure(J):
    R = rand_rot(np.random.default_rng(7))
    tau = oracle.kirchhoff(W, MU, LAM, R @ iso(J))
    S = oracle.stretch_from_tau(W, MU, LAM, tau)
    assert np.allclose(S, iso(J), rtol=1e-12, atol=1e-12)


@pytest.mark.parametrize("J", [0.1, 0.3, 0.45])
def test_reconstruction_takes_the_root_above_one_half(J):
    tau = oracle.kirchhoff(W, MU, LAM, iso(J))
    S = oracle.stretch_from_tau(W, MU, LAM, tau)
    Jb = np.linalg.det(S)
    assert Jb >= 0.5 and Jb == pytest.approx(1 - J, rel=1e-12)
    assert np.allclose(oracle.kirchhoff(W, MU, LAM, S), tau, atol=1e-9 * KAP)  # same pressure
    assert np.allclose(S, np.cbrt(Jb) * np.eye(3), atol=1e-14)


def test_reconstruction_rejects_pressure_below_the_minimum():
    with pytest.raises(Exception):
        oracle.stretch_from_tau(W, MU, LAM, -0.3 * KAP * np.eye(3))  # pi < -kappa/4


def test_load_updates_J_by_the_velocity_divergence():
    """Affine node velocities v = A x + c: G_c = A in every cell (linear reproduction),
    so each water particle's J becomes (1 + dt tr A) J and F stays isotropic, while a
    solid particle takes F <- (I + dt A) F."""
    n, dt = 16, 1e-3
    mats = [(W, E, NU), (oracle.FIXED_COROTATED, 1e5, 0.3)]
    o = oracle.Oracle(oracle.make_scene(n, 1.0 / n, dt, (0.0, 0.0, 0.0), mats))
    rng = np.random.default_rng(3)
    npart = 40
    x = rng.uniform(0.3, 0.7, (npart, 3))
    J0 = rng.uniform(0.9, 1.1, npart)
    mat = (np.arange(npart) % 2).astype(np.int32)
    F = np.stack([iso(j) if k == 0 else np.eye(3) + 0.01 * rng.standard_normal((3, 3))
                  for j, k in zip(J0, mat)])
    p = dict(x=x, v=np.zeros((npart, 3)), F=F.reshape(npart, 9), G=np.zeros((npart, 9)),
             mp=np.full(npart, 1e-3), Vp=np.full(npart, 1e-6), mat=mat)
    assert o.unload(**p) == 0
    A = np.array([[0.3, 0.1, -0.2], [0.05, -0.4, 0.1], [0.2, 0.0, 0.6]])
    c = np.array([0.1, -0.2, 0.05])
    ijk = oracle.decode_keys(o.node_keys(), n)
    xn = ijk * (1.0 / n)
    o.set_node_velocity(xn @ A.T + c)
    rc, res = o.load()
    assert rc == 0
    perm = o.perm()
    Fo = res["F"].reshape(-1, 3, 3)
    for q in range(npart):
        src = perm[q]
        if res["mat"][q] == 0:
            Jn = (1 + dt * np.trace(A)) * J0[src]
            assert np.allclose(Fo[q], iso(Jn), rtol=1e-12, atol=1e-13)
        else:
            assert np.allclose(Fo[q], (np.eye(3) + dt * A) @ F[src], rtol=1e-12, atol=1e-13)
