"""FP64 CPU oracle for the MPM Lite implicit step (arXiv 2602.07853).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and
``bench.py``'s cpu_baseline / reference arm may import this package.  It
shares no code with the CUDA library (``paper_2602_07853_gb300``) and never
imports it.

The arithmetic lives in ``mpml_oracle.c`` (plain double-precision loops,
built with ``-O2 -ffp-contract=off``).  This module only compiles it,
marshals numpy arrays and gives the steps the paper's names:

* :meth:`Oracle.unload`   Algorithm 2 (Sec. 3.1-3.3)
* :meth:`Oracle.stretch`  Algorithm 3, stretch reconstruction (Sec. 4.3)
* :meth:`Oracle.newton`   Algorithm 3, minimise the incremental potential
* :meth:`Oracle.load`     Algorithm 4

Every function here is pinned by a ``-m "not gpu"`` test (finite
differences, closed forms, brute force, conservation laws) except the
long-horizon trajectories of contact scenes (parity unpinned: compared as
statistics only).
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "mpml_oracle.c")
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

FIXED_COROTATED, NEO_HOOKEAN, HENCKY, WATER = 0, 1, 2, 3
OK, WARN_NOT_CONVERGED, ERR_ARG, ERR_OUT_OF_DOMAIN, ERR_NONFINITE, ERR_STRETCH = 0, 1, -1, -2, -3, -4
MAX_MATS = 4


def build(force: bool = False) -> str:
    """Compile ``liboracle.so`` next to the source (x86 here, aarch64 on the GPU machine)."""
    with _lock:
        stale = (not os.path.exists(_LIB_PATH)) or (
            os.path.getmtime(_LIB_PATH) < max(os.path.getmtime(_SRC),
                                              os.path.getmtime(os.path.join(_HERE, "mpml_oracle.h"))))
        if force or stale:
            tmp = _LIB_PATH + f".tmp{os.getpid()}"
            subprocess.check_call(["gcc", "-O2", "-std=c99", "-ffp-contract=off", "-fPIC", "-shared",
                                   "-o", tmp, _SRC, "-lm"])
            os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class Scene(C.Structure):
    _fields_ = [("n", C.c_int * 3), ("dx", C.c_double), ("inv_dx", C.c_double), ("dt", C.c_double),
                ("gravity", C.c_double * 3), ("n_mats", C.c_int), ("model", C.c_int * MAX_MATS),
                ("mu", C.c_double * MAX_MATS), ("lam", C.c_double * MAX_MATS),
                ("wall_layers", C.c_int), ("has_plate", C.c_int), ("plate_lo", C.c_double * 3),
                ("plate_hi", C.c_double * 3), ("plate_vel", C.c_double * 3), ("time", C.c_double),
                ("plastic", C.c_int * MAX_MATS), ("yield_stress", C.c_double * MAX_MATS),
                ("friction_angle", C.c_double * MAX_MATS)]


class Solver(C.Structure):
    _fields_ = [("cg_rtol", C.c_double), ("cg_max", C.c_int), ("newton_rtol", C.c_double),
                ("newton_atol", C.c_double), ("newton_max", C.c_int), ("ls_c1", C.c_double),
                ("ls_max", C.c_int), ("fixed_point", C.c_int)]


class Stats(C.Structure):
    _fields_ = [("status", C.c_int), ("newton_iters", C.c_int), ("cg_iters_total", C.c_int),
                ("cg_iters", C.c_int * 64), ("alpha", C.c_double * 64), ("g0_norm", C.c_double),
                ("g_norm", C.c_double), ("phi0", C.c_double), ("phi", C.c_double)]


_D = C.POINTER(C.c_double)
_I = C.POINTER(C.c_int)
_L = C.POINTER(C.c_long)
_LL = C.POINTER(C.c_longlong)
_VP = C.c_void_p


def lib():
    global _lib
    if _lib is None:
        build()
        L = C.CDLL(_LIB_PATH)
        sig = {
            "orc_create": (_VP, [C.POINTER(Scene)]),
            "orc_destroy": (None, [_VP]),
            "orc_set_time": (None, [_VP, C.c_double]),
            "orc_unload": (C.c_int, [_VP, C.c_long, _D, _D, _D, _D, _D, _D, _I]),
            "orc_stretch": (C.c_int, [_VP]),
            "orc_newton": (C.c_int, [_VP, C.POINTER(Solver), C.POINTER(Stats)]),
            "orc_explicit": (C.c_int, [_VP]),
            "orc_load": (C.c_int, [_VP, _D, _D, _D, _D, _D, _D, _I]),
            "orc_count": (C.c_long, [_VP, C.c_int]),
            "orc_get_perm": (None, [_VP, _L]),
            "orc_get_particle_keys": (None, [_VP, _LL]),
            "orc_get_cell_keys": (None, [_VP, _LL]),
            "orc_get_node_keys": (None, [_VP, _LL]),
            "orc_get_field": (None, [_VP, C.c_int, _D]),
            "orc_set_node_velocity": (None, [_VP, _D]),
            "orc_eval": (C.c_int, [_VP, _D, _D, _D]),
            "orc_linearize": (C.c_int, [_VP, _D, C.c_int]),
            "orc_hvp": (None, [_VP, _D, _D]),
            "orc_diag": (None, [_VP, _D]),
            "orc_explicit_force": (None, [_VP, _D]),
            "orc_pcg": (C.c_int, [_VP, _D, _D, C.c_double, C.c_int, _D]),
            "orc_psi": (C.c_int, [C.c_int, C.c_double, C.c_double, _D, _D]),
            "orc_piola": (C.c_int, [C.c_int, C.c_double, C.c_double, _D, _D]),
            "orc_tangent": (C.c_int, [C.c_int, C.c_double, C.c_double, _D, C.c_int, _D]),
            "orc_kirchhoff": (C.c_int, [C.c_int, C.c_double, C.c_double, _D, _D]),
            "orc_stretch_from_tau": (C.c_int, [C.c_int, C.c_double, C.c_double, _D, _D]),
            "orc_svd3": (None, [_D, _D, _D, _D]),
            "orc_sym_eigen": (None, [C.c_int, _D, _D, _D]),
            "orc_return_map": (C.c_int, [C.c_int, C.c_double, C.c_double, C.c_double, C.c_double, _D]),
        }
        for name, (res, args) in sig.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def _dp(a):
    return a.ctypes.data_as(_D)


def _f64(a, shape=None):
    a = np.ascontiguousarray(a, dtype=np.float64)
    if shape is not None:
        a = a.reshape(shape)
    return a


# ----------------------------------------------------------------------------
# constitutive pieces
# ----------------------------------------------------------------------------
def psi(model, mu, lam, F):
    F = _f64(F, (3, 3))
    out = C.c_double()
    rc = lib().orc_psi(model, mu, lam, _dp(F), C.byref(out))
    return out.value if rc == 0 else np.inf


def piola(model, mu, lam, F):
    F = _f64(F, (3, 3))
    P = np.zeros((3, 3))
    if lib().orc_piola(model, mu, lam, _dp(F), _dp(P)):
        raise ValueError("energy undefined at F")
    return P


def tangent(model, mu, lam, F, project=False):
    F = _f64(F, (3, 3))
    A = np.zeros((9, 9))
    if lib().orc_tangent(model, mu, lam, _dp(F), int(project), _dp(A)):
        raise ValueError("energy undefined at F")
    return A


def kirchhoff(model, mu, lam, F):
    F = _f64(F, (3, 3))
    t = np.zeros((3, 3))
    if lib().orc_kirchhoff(model, mu, lam, _dp(F), _dp(t)):
        raise ValueError("energy undefined at F")
    return t


def stretch_from_tau(model, mu, lam, tau):
    tau = _f64(tau, (3, 3))
    S = np.zeros((3, 3))
    rc = lib().orc_stretch_from_tau(model, mu, lam, _dp(tau), _dp(S))
    if rc:
        raise ValueError(f"stretch reconstruction failed ({rc})")
    return S


def svd3(F):
    F = _f64(F, (3, 3))
    U, s, V = np.zeros((3, 3)), np.zeros(3), np.zeros((3, 3))
    lib().orc_svd3(_dp(F), _dp(U), _dp(s), _dp(V))
    return U, s, V


def sym_eigen(A):
    A = _f64(A)
    n = A.shape[0]
    ev, Q = np.zeros(n), np.zeros((n, n))
    lib().orc_sym_eigen(n, _dp(A), _dp(ev), _dp(Q))
    return ev, Q


ELASTIC, VON_MISES, DRUCKER_PRAGER = 0, 1, 2


def return_map(plastic, mu, lam, yield_stress, friction_angle, F):
    """Plastic return map of one deformation gradient; returns (kind, F_new)."""
    Fn = np.ascontiguousarray(np.asarray(F, dtype=np.float64).reshape(9).copy())
    kind = lib().orc_return_map(int(plastic), float(mu), float(lam), float(yield_stress),
                                float(friction_angle), _dp(Fn))
    return kind, Fn.reshape(3, 3)


def lame(E, nu):
    """mu = E / (2 (1 + nu)), lam = E nu / ((1 + nu)(1 - 2 nu)) (standard; not stated in the paper)."""
    return E / (2 * (1 + nu)), E * nu / ((1 + nu) * (1 - 2 * nu))


# ----------------------------------------------------------------------------
# whole-step state
# ----------------------------------------------------------------------------
def make_scene(n, dx, dt, gravity=(0.0, -9.8, 0.0), materials=((FIXED_COROTATED, 1e5, 0.3),),
               wall_layers=1, plate=None, inv_dx=None, time=0.0):
    """materials: sequence of (model, E, nu) or (model, E, nu, plastic, yield_stress,
    friction_angle_radians).  plate: (lo3, hi3, vel3) or None."""
    sc = Scene()
    n = (n, n, n) if np.isscalar(n) else tuple(n)
    for a in range(3):
        sc.n[a] = int(n[a])
        sc.gravity[a] = float(gravity[a])
    sc.dx = float(dx)
    sc.inv_dx = float(inv_dx if inv_dx is not None else 1.0 / dx)
    sc.dt = float(dt)
    sc.n_mats = len(materials)
    for k, mt in enumerate(materials):
        model, E, nu = mt[:3]
        mu, lam = lame(E, nu)
        sc.model[k], sc.mu[k], sc.lam[k] = int(model), mu, lam
        if len(mt) > 3:
            sc.plastic[k], sc.yield_stress[k], sc.friction_angle[k] = int(mt[3]), float(mt[4]), float(mt[5])
    sc.wall_layers = int(wall_layers)
    if plate is not None:
        sc.has_plate = 1
        for a in range(3):
            sc.plate_lo[a], sc.plate_hi[a], sc.plate_vel[a] = plate[0][a], plate[1][a], plate[2][a]
    sc.time = float(time)
    return sc


def default_solver(cg_rtol=1e-6, cg_max=10000, newton_rtol=1e-6, newton_atol=0.0, newton_max=50,
                   ls_c1=1e-4, ls_max=30, fixed_point=0):
    s = Solver()
    s.cg_rtol, s.cg_max, s.newton_rtol, s.newton_atol = cg_rtol, cg_max, newton_rtol, newton_atol
    s.newton_max, s.ls_c1, s.ls_max, s.fixed_point = newton_max, ls_c1, ls_max, int(fixed_point)
    return s


class Oracle:
    """One MPM Lite time step at a time, in FP64, on the CPU."""

    def __init__(self, scene: Scene):
        self.scene = scene
        self._h = lib().orc_create(C.byref(scene))

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            lib().orc_destroy(h)
            self._h = None

    def set_time(self, t):
        self.scene.time = t
        lib().orc_set_time(self._h, float(t))

    # Algorithm 2
    def unload(self, x, v, F, G, mp, Vp, mat):
        np_ = int(np.asarray(x).shape[0])
        self._p = dict(x=_f64(x, (np_, 3)), v=_f64(v, (np_, 3)), F=_f64(F, (np_, 3, 3)),
                       G=_f64(G, (np_, 3, 3)), mp=_f64(mp, (np_,)), Vp=_f64(Vp, (np_,)),
                       mat=np.ascontiguousarray(mat, dtype=np.int32).reshape(np_))
        p = self._p
        rc = lib().orc_unload(self._h, np_, _dp(p["x"]), _dp(p["v"]), _dp(p["F"]), _dp(p["G"]),
                              _dp(p["mp"]), _dp(p["Vp"]), p["mat"].ctypes.data_as(_I))
        return rc

    def stretch(self):
        return lib().orc_stretch(self._h)

    def newton(self, solver=None):
        st = Stats()
        solver = solver or default_solver()
        rc = lib().orc_newton(self._h, C.byref(solver), C.byref(st))
        return rc, st

    def explicit(self):
        """Algorithm 3, explicit branch: node velocities from the explicit internal force."""
        return lib().orc_explicit(self._h)

    def explicit_step(self, particles):
        """Algorithm 1 with the explicit integrator: (status, new particles (sorted))."""
        rc = self.unload(**particles)
        if rc:
            return rc, None
        self.explicit()
        return self.load()

    def load(self):
        n = self.count("particles")
        x, v = np.zeros((n, 3)), np.zeros((n, 3))
        F, G = np.zeros((n, 3, 3)), np.zeros((n, 3, 3))
        mp, Vp, mat = np.zeros(n), np.zeros(n), np.zeros(n, dtype=np.int32)
        rc = lib().orc_load(self._h, _dp(x), _dp(v), _dp(F), _dp(G), _dp(mp), _dp(Vp),
                            mat.ctypes.data_as(_I))
        return rc, dict(x=x, v=v, F=F, G=G, mp=mp, Vp=Vp, mat=mat)

    def step(self, particles, solver=None):
        """Algorithm 1: returns (status, new particle dict (sorted), stats)."""
        rc = self.unload(**particles)
        if rc:
            return rc, None, None
        rc = self.stretch()
        if rc:
            return rc, None, None
        rc, st = self.newton(solver)
        if rc < 0:
            return rc, None, st
        rc2, out = self.load()
        return (rc if rc else rc2), out, st

    # introspection
    def count(self, what):
        return int(lib().orc_count(self._h, {"particles": 0, "cells": 1, "nodes": 2}[what]))

    def perm(self):
        out = np.zeros(self.count("particles"), dtype=np.int64)
        lib().orc_get_perm(self._h, out.ctypes.data_as(_L))
        return out

    def particle_keys(self):
        out = np.zeros(self.count("particles"), dtype=np.int64)
        lib().orc_get_particle_keys(self._h, out.ctypes.data_as(_LL))
        return out

    def cell_keys(self):
        out = np.zeros(self.count("cells"), dtype=np.int64)
        lib().orc_get_cell_keys(self._h, out.ctypes.data_as(_LL))
        return out

    def node_keys(self):
        out = np.zeros(self.count("nodes"), dtype=np.int64)
        lib().orc_get_node_keys(self._h, out.ctypes.data_as(_LL))
        return out

    _FIELDS = {"m_c": (0, "c", 1), "v_c": (1, "c", 3), "G_c": (2, "c", 9), "V_ck": (3, "c", -1),
               "tau_ck": (4, "c", -9), "S_ck": (5, "c", -9), "v_c_new": (6, "c", 3),
               "G_c_new": (7, "c", 9), "m_i": (10, "n", 1), "v_i": (11, "n", 3),
               "vhat": (12, "n", 3), "fixed": (13, "n", 1), "v_new": (14, "n", 3)}

    def field(self, name):
        fid, where, w = self._FIELDS[name]
        K = self.scene.n_mats
        n = self.count("cells" if where == "c" else "nodes")
        width = w if w > 0 else K * (-w)
        out = np.zeros(n * width)
        lib().orc_get_field(self._h, fid, _dp(out))
        if w == 1:
            return out
        if w == 3:
            return out.reshape(n, 3)
        if w == 9:
            return out.reshape(n, 3, 3)
        if w == -1:
            return out.reshape(n, K)
        return out.reshape(n, K, 3, 3)

    def set_node_velocity(self, v):
        v = _f64(v, (self.count("nodes"), 3))
        lib().orc_set_node_velocity(self._h, _dp(v))

    def eval(self, v, grad=True):
        v = _f64(v, (self.count("nodes"), 3))
        phi = C.c_double()
        g = np.zeros_like(v)
        lib().orc_eval(self._h, _dp(v), C.byref(phi), _dp(g) if grad else None)
        return phi.value, g

    def linearize(self, v, project=True):
        v = _f64(v, (self.count("nodes"), 3))
        return lib().orc_linearize(self._h, _dp(v), int(project))

    def hvp(self, p):
        p = _f64(p, (self.count("nodes"), 3))
        y = np.zeros_like(p)
        lib().orc_hvp(self._h, _dp(p), _dp(y))
        return y

    def diag(self):
        d = np.zeros((self.count("nodes"), 3))
        lib().orc_diag(self._h, _dp(d))
        return d

    def explicit_force(self):
        f = np.zeros((self.count("nodes"), 3))
        lib().orc_explicit_force(self._h, _dp(f))
        return f

    def pcg(self, b, rtol=1e-6, maxit=10000):
        b = _f64(b, (self.count("nodes"), 3))
        x = np.zeros_like(b)
        rr = C.c_double()
        it = lib().orc_pcg(self._h, _dp(b), _dp(x), rtol, maxit, C.byref(rr))
        return x, it, rr.value


def decode_keys(keys, n):
    """Brick-major key (8^3 bricks) -> integer (i, j, k) grid coordinates."""
    n = (n, n, n) if np.isscalar(n) else tuple(n)
    keys = np.asarray(keys, dtype=np.int64)
    nbx, nby = (n[0] >> 3) + 1, (n[1] >> 3) + 1
    b, l = keys // 512, keys % 512
    i = (b % nbx) * 8 + l % 8
    j = ((b // nbx) % nby) * 8 + (l // 8) % 8
    k = (b // (nbx * nby)) * 8 + l // 64
    return np.stack([i, j, k], axis=1)
