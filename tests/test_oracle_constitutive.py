"""Pins for the oracle's constitutive pieces (CPU only).

Each test checks the oracle against something other than itself: finite
differences, the paper's closed forms retyped from the text in numpy,
scipy's polar / matrix square root, numpy's eigh and polynomial roots.
"""
import numpy as np
import pytest
import scipy.linalg

import oracle

MODELS = [oracle.FIXED_COROTATED, oracle.NEO_HOOKEAN, oracle.HENCKY, oracle.WATER]
MU, LAM = oracle.lame(1e5, 0.3)


def rand_rot(rng):
    q, r = np.linalg.qr(rng.standard_normal((3, 3)))
    q = q @ np.diag(np.sign(np.diag(r)))
    if np.linalg.det(q) < 0:
        q[:, 0] = -q[:, 0]
    return q


def rand_F(rng, scale):
    return np.eye(3) + scale * rng.standard_normal((3, 3))


@pytest.mark.parametrize("scale", [1e-3, 0.1, 0.4])
def test_svd_signed(scale):
    rng = np.random.default_rng(0)
    for _ in range(50):
        F = rand_F(rng, scale)
        if rng.random() < 0.3:
            F[:, 2] *= -1  # inverted
        U, s, V = oracle.svd3(F)
        assert np.allclose(U @ np.diag(s) @ V.T, F, atol=1e-12)
        assert np.allclose(U.T @ U, np.eye(3), atol=1e-12)
        assert np.allclose(V.T @ V, np.eye(3), atol=1e-12)
        assert np.isclose(np.linalg.det(U), 1) and np.isclose(np.linalg.det(V), 1)
        assert s[0] >= s[1] >= abs(s[2]) - 1e-12
        assert np.sign(s[2]) == np.sign(np.linalg.det(F))


def test_sym_eigen_matches_numpy():
    rng = np.random.default_rng(1)
    for n in (3, 9):
        A = rng.standard_normal((n, n))
        A = A + A.T
        ev, Q = oracle.sym_eigen(A)
        assert np.allclose(np.sort(ev), np.linalg.eigvalsh(A), atol=1e-12)
        assert np.allclose(Q @ np.diag(ev) @ Q.T, A, atol=1e-12)


@pytest.mark.parametrize("model", MODELS)
@pytest.mark.parametrize("scale", [1e-2, 0.2])
def test_piola_is_energy_gradient(model, scale):
    """P = dpsi/dF by central differences."""
    rng = np.random.default_rng(2 + model)
    h = 1e-6
    for _ in range(10):
        F = rand_F(rng, scale)
        if np.linalg.det(F) <= 0.2:
            continue
        P = oracle.piola(model, MU, LAM, F)
        fd = np.zeros((3, 3))
        for a in range(3):
            for b in range(3):
                E = np.zeros((3, 3))
                E[a, b] = h
                fd[a, b] = (oracle.psi(model, MU, LAM, F + E) - oracle.psi(model, MU, LAM, F - E)) / (2 * h)
        assert np.allclose(P, fd, rtol=1e-6, atol=1e-6 * np.abs(P).max())


@pytest.mark.parametrize("model", MODELS)
@pytest.mark.parametrize("scale", [1e-2, 0.2])
def test_tangent_is_piola_derivative(model, scale):
    """Unprojected dP/dF by central differences of P, and symmetric."""
    rng = np.random.default_rng(10 + model)
    h = 1e-6
    for _ in range(10):
        F = rand_F(rng, scale)
        if np.linalg.det(F) <= 0.2:
            continue
        A = oracle.tangent(model, MU, LAM, F, project=False)
        fd = np.zeros((9, 9))
        for c in range(9):
            E = np.zeros(9)
            E[c] = h
            fd[:, c] = ((oracle.piola(model, MU, LAM, F + E.reshape(3, 3)) -
                         oracle.piola(model, MU, LAM, F - E.reshape(3, 3))) / (2 * h)).ravel()
        assert np.allclose(A, A.T, atol=1e-9 * np.abs(A).max())
        assert np.allclose(A, fd, rtol=1e-5, atol=1e-6 * np.abs(A).max())


@pytest.mark.parametrize("model", MODELS)
def test_tangent_equal_singular_values(model):
    """The closed-form pair terms stay finite and continuous at s_i == s_j."""
    R = rand_rot(np.random.default_rng(3))
    F = R @ np.diag([1.1, 1.1, 0.9])
    A = oracle.tangent(model, MU, LAM, F)
    A2 = oracle.tangent(model, MU, LAM, R @ np.diag([1.1 + 1e-7, 1.1, 0.9]))
    assert np.all(np.isfinite(A))
    assert np.allclose(A, A2, rtol=1e-5, atol=1e-5 * np.abs(A).max())


@pytest.mark.parametrize("model", MODELS)
def test_projection_is_eigen_clamp(model):
    """Projected tangent == numpy eigh with negative eigenvalues set to 0."""
    rng = np.random.default_rng(20 + model)
    for scale in (0.05, 0.5):
        for _ in range(10):
            F = rand_F(rng, scale)
            if np.linalg.det(F) <= 0.1:
                continue
            A = oracle.tangent(model, MU, LAM, F, project=False)
            Ap = oracle.tangent(model, MU, LAM, F, project=True)
            w, Q = np.linalg.eigh(A)
            ref = (Q * np.maximum(w, 0)) @ Q.T
            assert np.allclose(Ap, ref, atol=1e-9 * np.abs(A).max())
            assert np.linalg.eigvalsh(Ap).min() >= -1e-9 * np.abs(A).max()


def test_kirchhoff_neo_hookean_split_form():
    """Eq. for the split Neo-Hookean Kirchhoff stress, retyped in numpy:
    tau = mu J^{-2/d} dev(b) + kappa/2 (J^2 - 1) I (Sec. 4.3.2)."""
    rng = np.random.default_rng(4)
    kap = 2 / 3 * MU + LAM
    for _ in range(20):
        F = rand_F(rng, 0.2)
        J = np.linalg.det(F)
        if J <= 0.2:
            continue
        b = F @ F.T
        ref = MU * J ** (-2 / 3) * (b - np.trace(b) / 3 * np.eye(3)) + kap / 2 * (J * J - 1) * np.eye(3)
        assert np.allclose(oracle.kirchhoff(oracle.NEO_HOOKEAN, MU, LAM, F), ref, rtol=1e-10,
                           atol=1e-10 * np.abs(ref).max())


def test_kirchhoff_hencky_principal_form():
    """Principal Kirchhoff stress of Hencky-StVK: tau_i = 2 mu log s_i + lam sum log s_j
    (Sec. 4.3.1), directions = eigenvectors of b = F F^T (numpy eigh)."""
    rng = np.random.default_rng(5)
    for _ in range(20):
        F = rand_F(rng, 0.2)
        if np.linalg.det(F) <= 0.2:
            continue
        w, Q = np.linalg.eigh(F @ F.T)
        e = 0.5 * np.log(w)
        ref = Q @ np.diag(2 * MU * e + LAM * e.sum()) @ Q.T
        assert np.allclose(oracle.kirchhoff(oracle.HENCKY, MU, LAM, F), ref, rtol=1e-10,
                           atol=1e-10 * np.abs(ref).max())


def test_kirchhoff_fixed_corotated_polar_form():
    """Fixed-corotated: P = 2 mu (F - R) + lam (J - 1) J F^{-T} with R from scipy's polar."""
    rng = np.random.default_rng(6)
    for _ in range(20):
        F = rand_F(rng, 0.2)
        J = np.linalg.det(F)
        if J <= 0.2:
            continue
        R, _ = scipy.linalg.polar(F)
        P = 2 * MU * (F - R) + LAM * (J - 1) * J * np.linalg.inv(F).T
        assert np.allclose(oracle.piola(oracle.FIXED_COROTATED, MU, LAM, F), P, rtol=1e-9,
                           atol=1e-9 * np.abs(P).max())
        assert np.allclose(oracle.kirchhoff(oracle.FIXED_COROTATED, MU, LAM, F), P @ F.T, rtol=1e-9,
                           atol=1e-9 * np.abs(P).max())


# water keeps J only (its reconstruction is J^(1/3) I, pinned in test_oracle_water)
@pytest.mark.parametrize("model", [m for m in MODELS if m != oracle.WATER])
@pytest.mark.parametrize("scale", [1e-4, 1e-2, 0.15])
def test_stretch_round_trip(model, scale):
    """tau = P(F) F^T then reconstruct: S = sqrtm(F F^T) (the left stretch; scipy), and
    P(S) S^T = tau (Sec. 4.2, the defining relation of the rotation-free base)."""
    rng = np.random.default_rng(30 + model)
    for _ in range(20):
        F = rand_rot(rng) @ (np.eye(3) + scale * rng.standard_normal((3, 3)))
        # fixed-corotated is inverted on its unique branch J >= 1/2 only
        if np.linalg.det(F) <= (0.5 if model == oracle.FIXED_COROTATED else 0.3):
            continue
        tau = oracle.kirchhoff(model, MU, LAM, F)
        S = oracle.stretch_from_tau(model, MU, LAM, tau)
        Vl = np.real(scipy.linalg.sqrtm(F @ F.T))
        assert np.allclose(S, Vl, atol=1e-9)
        tau2 = oracle.piola(model, MU, LAM, S) @ S.T
        assert np.allclose(tau2, tau, atol=1e-8 * max(1.0, np.abs(tau).max()))
        assert np.allclose(S @ tau, tau @ S, atol=1e-8 * max(1.0, np.abs(tau).max()))


@pytest.mark.parametrize("model", MODELS)
def test_stretch_zero_stress_is_identity(model):
    assert np.allclose(oracle.stretch_from_tau(model, MU, LAM, np.zeros((3, 3))), np.eye(3), atol=1e-13)


def test_hencky_inverse_matches_root_solve():
    """Closed-form Hencky inverse (Sec. 4.3.1) vs scipy's root finder on tau_i(e)."""
    import scipy.optimize
    rng = np.random.default_rng(7)
    for _ in range(10):
        t = 1e4 * rng.standard_normal(3)
        fun = lambda e: 2 * MU * e + LAM * e.sum() - t
        e = scipy.optimize.fsolve(fun, np.zeros(3), xtol=1e-14)
        S = oracle.stretch_from_tau(oracle.HENCKY, MU, LAM, np.diag(t))
        assert np.allclose(np.diag(S), np.exp(e), rtol=1e-10)


def test_neo_hookean_cardano_matches_polynomial_roots():
    """App. C root choice: beta_i = m + delta_i with m the largest real root of
    m^3 + S2 m + S3 - J^2 (numpy.roots) reproduces the sampled stretches."""
    rng = np.random.default_rng(8)
    kap = 2 / 3 * MU + LAM
    for _ in range(30):
        s = np.exp(0.2 * rng.standard_normal(3))
        J = s.prod()
        beta = s ** 2
        # principal Kirchhoff stresses from the split form
        t = MU * J ** (-2 / 3) * (beta - beta.mean()) + kap / 2 * (J * J - 1)
        S = oracle.stretch_from_tau(oracle.NEO_HOOKEAN, MU, LAM, np.diag(t))
        assert np.allclose(np.diag(S), s, rtol=1e-9)
        alpha = t.mean()
        Jr = np.sqrt(1 + 2 * alpha / kap)
        d = (t - alpha) / (MU * Jr ** (-2 / 3))
        S2 = d[0] * d[1] + d[1] * d[2] + d[2] * d[0]
        roots = np.roots([1, 0, S2, d.prod() - Jr * Jr])
        m = max(r.real for r in roots if abs(r.imag) < 1e-9)
        assert np.allclose(np.sqrt(m + d), s, rtol=1e-7)


def test_fixed_corotated_inverse_unique_branch():
    """tau_i = 2 mu s_i (s_i - 1) + lam J (J - 1) with J = prod s_i, checked in numpy."""
    rng = np.random.default_rng(9)
    for _ in range(30):
        s = np.exp(0.15 * rng.standard_normal(3))
        J = s.prod()
        t = 2 * MU * s * (s - 1) + LAM * J * (J - 1)
        S = oracle.stretch_from_tau(oracle.FIXED_COROTATED, MU, LAM, np.diag(t))
        assert np.allclose(np.diag(S), s, rtol=1e-10)


def test_fixed_corotated_rejects_below_half_volume():
    """J < 1/2 lies off the branch on which the inverse is unique: ERR_STRETCH."""
    s = np.array([1.0233, 0.9507, 0.5005])
    J = s.prod()
    t = 2 * MU * s * (s - 1) + LAM * J * (J - 1)
    with pytest.raises(ValueError):
        oracle.stretch_from_tau(oracle.FIXED_COROTATED, MU, LAM, np.diag(t))


@pytest.mark.parametrize("scale", [1e-7, 1e-5, 1e-3, 3e-2, 0.2])
def test_neo_hookean_energy_keeps_relative_accuracy_at_small_strain(scale):
    """The split Neo-Hookean energy of Sec. 4.3.2 against a 50-digit evaluation of the
    same formula (mpmath): second order in the strain, so a direct FP64 evaluation of
    J^(-2/3) I1 - 3 loses about eps / strain^2 of relative accuracy; the oracle's form
    keeps it (1e-12 relative here), which the line search needs near convergence."""
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 50
    rng = np.random.default_rng(int(1e3 * scale) + 7)
    for _ in range(20):
        F = np.eye(3) + scale * rng.standard_normal((3, 3))
        Fm = mp.matrix([[mp.mpf(float(F[i, j])) for j in range(3)] for i in range(3)])
        J = mp.det(Fm)
        I1 = sum(Fm[i, j] ** 2 for i in range(3) for j in range(3))
        kap = mp.mpf(2) / 3 * MU + LAM
        ref = MU / 2 * (J ** (mp.mpf(-2) / 3) * I1 - 3) + kap / 4 * (J ** 2 - 1 - 2 * mp.log(J))
        got = oracle.psi(oracle.NEO_HOOKEAN, MU, LAM, F)
        assert abs(got - float(ref)) <= 1e-12 * abs(float(ref)), (scale, got, float(ref))
