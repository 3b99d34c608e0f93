"""Thin ctypes binding of ``include/mpml.h`` (argument marshalling only).

Every function keeps the C name (``mpml_create``, ``mpml_resample``,
``mpml_newton_step``, ``mpml_g2p`` ...).  All computation happens in
``libmpml.so`` (CUDA, sm_103a); this module never computes anything itself
and raises if the library cannot be loaded.  Torch is only used to hand
device pointers and streams over.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import build as _build

MAX_MATS = 4
OK, WARN_NOT_CONVERGED = 0, 1
ERR_ARG, ERR_OUT_OF_DOMAIN, ERR_NONFINITE, ERR_STRETCH, ERR_TIMEOUT, ERR_CUDA, ERR_NOMEM = -1, -2, -3, -4, -5, -6, -7
ERR_TOO_LARGE = -8
NOALLOC_MAX_SLOTS = 1 << 21
FIXED_COROTATED, NEO_HOOKEAN, HENCKY, WATER = 0, 1, 2, 3
ELASTIC, VON_MISES, DRUCKER_PRAGER = 0, 1, 2
FP32, FP64 = 0, 1
MEM_DEVICE, MEM_HOST = 0, 1
PRECOND_JACOBI, PRECOND_LEARNED = 0, 1
PCG_AUTO, PCG_STAGED, PCG_STREAMED, PCG_COLUMNS = 0, 1, 2, 3
PCG_SHAPES = 7  # MPML_PCG_SHAPES
PCG_SHAPE_TABLE = ((1, 1), (1, 2), (2, 1), (2, 2), (3, 2), (3, 3), (3, 4))
KEYS_PARTICLES, KEYS_CELLS, KEYS_NODES = 0, 1, 2
F_CELL_MASS, F_CELL_VEL, F_CELL_VGRAD, F_CELL_VOL, F_CELL_TAU, F_CELL_STRETCH = 0, 1, 2, 3, 4, 5
F_CELL_VEL_NEW, F_CELL_VGRAD_NEW = 6, 7
F_NODE_MASS, F_NODE_VEL, F_NODE_VHAT, F_NODE_FIXED, F_NODE_VNEW = 10, 11, 12, 13, 14


class mpml_material(C.Structure):
    _fields_ = [("model", C.c_int), ("mu", C.c_double), ("lambda_", C.c_double), ("plastic", C.c_int),
                ("yield_stress", C.c_double), ("friction_angle", C.c_double)]


class mpml_scene_desc(C.Structure):
    _fields_ = [("n", C.c_int * 3), ("dx", C.c_double), ("inv_dx", C.c_double), ("dt", C.c_double),
                ("gravity", C.c_double * 3), ("precision", C.c_int), ("wall_layers", C.c_int),
                ("has_plate", C.c_int), ("plate_lo", C.c_double * 3), ("plate_hi", C.c_double * 3),
                ("plate_vel", C.c_double * 3)]


class mpml_particles(C.Structure):
    _fields_ = [("n", C.c_int64), ("mem", C.c_int), ("x", C.c_void_p), ("v", C.c_void_p), ("F", C.c_void_p),
                ("G", C.c_void_p), ("mass", C.c_void_p), ("volume", C.c_void_p),
                ("mat", C.c_void_p), ("perm", C.c_void_p)]


class mpml_solver_opts(C.Structure):
    _fields_ = [("cg_rtol", C.c_double), ("cg_max", C.c_int), ("newton_rtol", C.c_double),
                ("newton_atol", C.c_double), ("newton_max", C.c_int), ("ls_c1", C.c_double),
                ("ls_max", C.c_int), ("precond", C.c_int), ("check_every", C.c_int), ("use_graph", C.c_int),
                ("plastic_fixed_point", C.c_int), ("cg_forcing", C.c_double)]


class mpml_solve_stats(C.Structure):
    _fields_ = [("status", C.c_int), ("newton_iters", C.c_int), ("cg_iters_total", C.c_int),
                ("cg_iters", C.c_int * 64), ("alpha", C.c_double * 64), ("cg_rel_resid", C.c_double * 64),
                ("g0_norm", C.c_double), ("g_norm", C.c_double), ("phi0", C.c_double), ("phi", C.c_double),
                ("n_particles", C.c_int64), ("n_cells", C.c_int64), ("n_nodes", C.c_int64),
                ("n_bricks", C.c_int64), ("fcg_fallbacks", C.c_int), ("plastic_projections", C.c_int)]


class mpml_pcg_config(C.Structure):
    _fields_ = [("tangent_staging", C.c_int), ("ctas_per_sm", C.c_int), ("barrier_spins", C.c_uint)]


class mpml_train_opts(C.Structure):
    _fields_ = [("samples", C.c_int), ("rtol", C.c_double), ("cg_max", C.c_int), ("epochs", C.c_int),
                ("batch", C.c_int), ("lr", C.c_float)]


class mpml_train_stats(C.Structure):
    _fields_ = [("samples", C.c_int), ("loss_first", C.c_double), ("loss_last", C.c_double)]


_D = C.POINTER(C.c_double)
_I64 = C.POINTER(C.c_int64)
_lib = None

EXPORTS = {
    "mpml_create": (C.c_int, [C.POINTER(mpml_scene_desc), C.POINTER(mpml_material), C.c_int, C.c_void_p,
                              C.POINTER(C.c_void_p)]),
    "mpml_destroy": (C.c_int, [C.c_void_p]),
    "mpml_status_str": (C.c_char_p, [C.c_int]),
    "mpml_set_time": (C.c_int, [C.c_void_p, C.c_double]),
    "mpml_sync": (C.c_int, [C.c_void_p]),
    "mpml_resample": (C.c_int, [C.c_void_p, C.POINTER(mpml_particles)]),
    "mpml_newton_step": (C.c_int, [C.c_void_p, C.POINTER(mpml_solver_opts), C.POINTER(mpml_solve_stats)]),
    "mpml_g2p": (C.c_int, [C.c_void_p, C.POINTER(mpml_particles)]),
    "mpml_explicit_step": (C.c_int, [C.c_void_p]),
    "mpml_newton_step_batch": (C.c_int, [C.POINTER(C.c_void_p), C.c_int, C.POINTER(mpml_solver_opts),
                                         C.POINTER(mpml_solve_stats)]),
    "mpml_resample_batch": (C.c_int, [C.POINTER(C.c_void_p), C.POINTER(mpml_particles), C.c_int]),
    "mpml_counts": (C.c_int, [C.c_void_p, _I64]),
    "mpml_get_keys": (C.c_int, [C.c_void_p, C.c_int, _I64]),
    "mpml_get_field": (C.c_int, [C.c_void_p, C.c_int, _D]),
    "mpml_set_node_velocity": (C.c_int, [C.c_void_p, _D]),
    "mpml_stretch": (C.c_int, [C.c_void_p]),
    "mpml_eval": (C.c_int, [C.c_void_p, _D, _D, _D]),
    "mpml_linearize": (C.c_int, [C.c_void_p, _D]),
    "mpml_hvp": (C.c_int, [C.c_void_p, _D, _D]),
    "mpml_set_profiling": (C.c_int, [C.c_void_p, C.c_int]),
    "mpml_hvp_timing": (C.c_int, [C.c_void_p, _I64, _D, _D]),
    "mpml_hvp_bench": (C.c_int, [C.c_void_p, C.c_int, _D]),
    "mpml_kernel_launches": (C.c_int64, [C.c_void_p]),
    "mpml_pcg_timing": (C.c_int, [C.c_void_p, _I64, _I64, _D]),
    "mpml_nn_weight_count": (C.c_int, []),
    "mpml_nn_set_weights": (C.c_int, [C.c_void_p, C.POINTER(C.c_float)]),
    "mpml_nn_get_weights": (C.c_int, [C.c_void_p, C.POINTER(C.c_float)]),
    "mpml_nn_get_grad": (C.c_int, [C.c_void_p, C.POINTER(C.c_float)]),
    "mpml_nn_apply": (C.c_int, [C.c_void_p, _D, _D]),
    "mpml_nn_loss_grad": (C.c_int, [C.c_void_p, _D, _D, _D]),
    "mpml_nn_adam_step": (C.c_int, [C.c_void_p, C.c_float]),
    "mpml_nn_train": (C.c_int, [C.c_void_p, C.POINTER(mpml_train_opts), C.POINTER(mpml_train_stats)]),
    "mpml_sort_particles_noalloc": (C.c_int, [C.POINTER(C.c_int), C.c_double, C.c_int, C.c_void_p, C.c_int64,
                                              C.c_void_p, C.c_void_p, C.c_void_p]),
    "mpml_autotune_hvp": (C.c_int, [C.c_void_p, C.c_int, C.POINTER(C.c_int), C.POINTER(C.c_float)]),
    "mpml_set_hvp_tile": (C.c_int, [C.c_void_p, C.c_int]),
    "mpml_get_hvp_tile": (C.c_int, [C.c_void_p, C.POINTER(C.c_int), C.POINTER(C.c_char_p)]),
    "mpml_tile_cache_save": (C.c_int, [C.c_char_p]),
    "mpml_tile_cache_load": (C.c_int, [C.c_char_p]),
    "mpml_tile_cache_clear": (None, []),
    "mpml_set_pcg_config": (C.c_int, [C.c_void_p, C.POINTER(mpml_pcg_config)]),
    "mpml_get_pcg_config": (C.c_int, [C.c_void_p, C.POINTER(mpml_pcg_config), C.POINTER(C.c_int),
                                      C.POINTER(C.c_int)]),
    "mpml_autotune_pcg": (C.c_int, [C.c_void_p, C.c_int, C.c_int, C.POINTER(C.c_int), C.POINTER(C.c_float)]),
    "mpml_lame_parameters": (C.c_int, [C.c_double, C.c_double, _D, _D]),
}


def library_path() -> str:
    return _build.LIB


def load(build_if_stale: bool = False):
    """Load libmpml.so; raises OSError when it is missing (no fallback path exists)."""
    global _lib
    if _lib is None:
        if build_if_stale and _build.stale():
            _build.build()
        if not os.path.exists(_build.LIB):
            raise OSError(f"libmpml.so not built ({_build.LIB}); run __graft_entry__.build()")
        L = C.CDLL(_build.LIB)
        for name, (res, args) in EXPORTS.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


class MPMLError(RuntimeError):
    def __init__(self, code, where):
        self.code = code
        msg = load().mpml_status_str(code).decode()
        super().__init__(f"{where}: {msg} ({code})")


def _check(code, where):
    if code < 0:
        raise MPMLError(code, where)
    return code


# ---------------------------------------------------------------------------
# C names
# ---------------------------------------------------------------------------
def mpml_create(desc: mpml_scene_desc, mats, stream=None):
    arr = (mpml_material * len(mats))(*mats)
    h = C.c_void_p()
    _check(load().mpml_create(C.byref(desc), arr, len(mats), stream, C.byref(h)), "mpml_create")
    return h


def mpml_destroy(ctx):
    return load().mpml_destroy(ctx)


def mpml_set_time(ctx, t):
    return _check(load().mpml_set_time(ctx, float(t)), "mpml_set_time")


def mpml_sync(ctx):
    return _check(load().mpml_sync(ctx), "mpml_sync")


def mpml_resample(ctx, p: mpml_particles):
    return _check(load().mpml_resample(ctx, C.byref(p)), "mpml_resample")


def mpml_newton_step(ctx, opts: mpml_solver_opts | None = None, stats: mpml_solve_stats | None = None):
    stats = stats if stats is not None else mpml_solve_stats()
    rc = load().mpml_newton_step(ctx, C.byref(opts) if opts is not None else None, C.byref(stats))
    _check(rc, "mpml_newton_step")
    return rc, stats


def mpml_resample_batch(ctxs, parts):
    """Algorithm 2 for several contexts (device particles) with one host wait."""
    n = len(ctxs)
    arr = (C.c_void_p * n)(*[c.value if isinstance(c, C.c_void_p) else c for c in ctxs])
    ps = (mpml_particles * n)(*parts)
    return _check(load().mpml_resample_batch(arr, ps, n), "mpml_resample_batch")


def mpml_newton_step_batch(ctxs, opts: mpml_solver_opts | None = None):
    """Lockstep Newton solves of several contexts; returns (status, [mpml_solve_stats])."""
    n = len(ctxs)
    arr = (C.c_void_p * n)(*[c.value if isinstance(c, C.c_void_p) else c for c in ctxs])
    stats = (mpml_solve_stats * n)()
    rc = load().mpml_newton_step_batch(arr, n, C.byref(opts) if opts is not None else None, stats)
    _check(rc, "mpml_newton_step_batch")
    return rc, list(stats)


def mpml_explicit_step(ctx):
    return _check(load().mpml_explicit_step(ctx), "mpml_explicit_step")


def mpml_g2p(ctx, p: mpml_particles):
    return _check(load().mpml_g2p(ctx, C.byref(p)), "mpml_g2p")


def mpml_counts(ctx):
    out = (C.c_int64 * 4)()
    _check(load().mpml_counts(ctx, out), "mpml_counts")
    return dict(particles=out[0], cells=out[1], nodes=out[2], bricks=out[3])


def mpml_get_keys(ctx, what):
    n = mpml_counts(ctx)[{KEYS_PARTICLES: "particles", KEYS_CELLS: "cells", KEYS_NODES: "nodes"}[what]]
    out = np.zeros(n, dtype=np.int64)
    _check(load().mpml_get_keys(ctx, what, out.ctypes.data_as(_I64)), "mpml_get_keys")
    return out


_FIELD_WIDTH = {F_CELL_MASS: 1, F_CELL_VEL: 3, F_CELL_VGRAD: 9, F_CELL_VOL: -1, F_CELL_TAU: -9,
                F_CELL_STRETCH: -9, F_CELL_VEL_NEW: 3, F_CELL_VGRAD_NEW: 9, F_NODE_MASS: 1, F_NODE_VEL: 3,
                F_NODE_VHAT: 3, F_NODE_FIXED: 1, F_NODE_VNEW: 3}


def mpml_get_field(ctx, field, n_mats=1):
    counts = mpml_counts(ctx)
    n = counts["cells"] if field < 10 else counts["nodes"]
    w = _FIELD_WIDTH[field]
    width = w if w > 0 else n_mats * (-w)
    out = np.zeros(n * width)
    _check(load().mpml_get_field(ctx, field, out.ctypes.data_as(_D)), "mpml_get_field")
    if w == 1:
        return out
    if w == 3:
        return out.reshape(n, 3)
    if w == 9:
        return out.reshape(n, 3, 3)
    if w == -1:
        return out.reshape(n, n_mats)
    return out.reshape(n, n_mats, 3, 3)


def mpml_set_node_velocity(ctx, v):
    v = np.ascontiguousarray(v, dtype=np.float64)
    return _check(load().mpml_set_node_velocity(ctx, v.ctypes.data_as(_D)), "mpml_set_node_velocity")


def mpml_stretch(ctx):
    return _check(load().mpml_stretch(ctx), "mpml_stretch")


def mpml_eval(ctx, v, grad=True):
    v = np.ascontiguousarray(v, dtype=np.float64)
    phi = C.c_double()
    g = np.zeros_like(v) if grad else None
    _check(load().mpml_eval(ctx, v.ctypes.data_as(_D), C.byref(phi), g.ctypes.data_as(_D) if grad else None),
           "mpml_eval")
    return phi.value, g


def mpml_linearize(ctx, v):
    v = np.ascontiguousarray(v, dtype=np.float64)
    return _check(load().mpml_linearize(ctx, v.ctypes.data_as(_D)), "mpml_linearize")


def mpml_hvp(ctx, p):
    p = np.ascontiguousarray(p, dtype=np.float64)
    y = np.zeros_like(p)
    _check(load().mpml_hvp(ctx, p.ctypes.data_as(_D), y.ctypes.data_as(_D)), "mpml_hvp")
    return y


def mpml_set_profiling(ctx, enable):
    return _check(load().mpml_set_profiling(ctx, int(enable)), "mpml_set_profiling")


def mpml_hvp_timing(ctx):
    n, ms, b = C.c_int64(), C.c_double(), C.c_double()
    _check(load().mpml_hvp_timing(ctx, C.byref(n), C.byref(ms), C.byref(b)), "mpml_hvp_timing")
    return n.value, ms.value, b.value


def mpml_hvp_bench(ctx, iters):
    ms = C.c_double()
    _check(load().mpml_hvp_bench(ctx, int(iters), C.byref(ms)), "mpml_hvp_bench")
    return ms.value


def mpml_pcg_timing(ctx):
    n, it, ms = C.c_int64(), C.c_int64(), C.c_double()
    _check(load().mpml_pcg_timing(ctx, C.byref(n), C.byref(it), C.byref(ms)), "mpml_pcg_timing")
    return n.value, it.value, ms.value


def mpml_kernel_launches(ctx):
    return int(load().mpml_kernel_launches(ctx))


HVP_TILES = 3  # MPML_HVP_TILES


def mpml_autotune_hvp(ctx, reps=3):
    """(chosen tile, [mean ms of each tile]) on the current linearisation."""
    tile, ms = C.c_int(), (C.c_float * HVP_TILES)()
    _check(load().mpml_autotune_hvp(ctx, int(reps), C.byref(tile), ms), "mpml_autotune_hvp")
    return tile.value, [float(v) for v in ms]


def mpml_set_hvp_tile(ctx, tile):
    _check(load().mpml_set_hvp_tile(ctx, int(tile)), "mpml_set_hvp_tile")


def mpml_get_hvp_tile(ctx):
    tile, desc = C.c_int(), C.c_char_p()
    _check(load().mpml_get_hvp_tile(ctx, C.byref(tile), C.byref(desc)), "mpml_get_hvp_tile")
    return tile.value, (desc.value or b"").decode()


def mpml_set_pcg_config(ctx, tangent_staging=PCG_AUTO, ctas_per_sm=0, barrier_spins=0):
    cfg = mpml_pcg_config()
    cfg.tangent_staging, cfg.ctas_per_sm, cfg.barrier_spins = int(tangent_staging), int(ctas_per_sm), int(barrier_spins)
    return _check(load().mpml_set_pcg_config(ctx, C.byref(cfg)), "mpml_set_pcg_config")


def mpml_get_pcg_config(ctx):
    """(config dict, staging of the last persistent launch, its CTAs per SM)."""
    cfg, st, cp = mpml_pcg_config(), C.c_int(), C.c_int()
    _check(load().mpml_get_pcg_config(ctx, C.byref(cfg), C.byref(st), C.byref(cp)), "mpml_get_pcg_config")
    return (dict(tangent_staging=cfg.tangent_staging, ctas_per_sm=cfg.ctas_per_sm, barrier_spins=cfg.barrier_spins),
            st.value, cp.value)


def mpml_autotune_pcg(ctx, iters=20, reps=2):
    """(chosen shape, [ms of each of the PCG_SHAPES shapes, -1 where it does not fit])."""
    shape, ms = C.c_int(), (C.c_float * PCG_SHAPES)()
    _check(load().mpml_autotune_pcg(ctx, int(iters), int(reps), C.byref(shape), ms), "mpml_autotune_pcg")
    return shape.value, [float(v) for v in ms]


def mpml_tile_cache_save(path):
    _check(load().mpml_tile_cache_save(os.fsencode(path)), "mpml_tile_cache_save")


def mpml_tile_cache_load(path):
    _check(load().mpml_tile_cache_load(os.fsencode(path)), "mpml_tile_cache_load")


def mpml_tile_cache_clear():
    load().mpml_tile_cache_clear()


# ---------------------------------------------------------------------------
# marshalling helpers (no arithmetic)
# ---------------------------------------------------------------------------
def scene_desc(n, dx, dt, gravity=(0.0, -9.8, 0.0), precision=FP32, wall_layers=1, plate=None, inv_dx=None):
    d = mpml_scene_desc()
    n = (n, n, n) if np.isscalar(n) else tuple(n)
    for a in range(3):
        d.n[a] = int(n[a])
        d.gravity[a] = float(gravity[a])
    d.dx, d.dt = float(dx), float(dt)
    d.inv_dx = float(inv_dx if inv_dx is not None else 1.0 / dx)
    d.precision = int(precision)
    d.wall_layers = int(wall_layers)
    if plate is not None:
        d.has_plate = 1
        for a in range(3):
            d.plate_lo[a], d.plate_hi[a], d.plate_vel[a] = plate[0][a], plate[1][a], plate[2][a]
    return d


def material(model, mu, lam, plastic=ELASTIC, yield_stress=0.0, friction_angle=0.0):
    m = mpml_material()
    m.model, m.mu, m.lambda_ = int(model), float(mu), float(lam)
    m.plastic, m.yield_stress, m.friction_angle = int(plastic), float(yield_stress), float(friction_angle)
    return m


def solver_opts(cg_rtol=1e-6, cg_max=10000, newton_rtol=1e-6, newton_atol=0.0, newton_max=50, ls_c1=1e-4,
                ls_max=30, precond=PRECOND_JACOBI, check_every=16, use_graph=2, plastic_fixed_point=0,
                cg_forcing=0.0):
    o = mpml_solver_opts()
    o.cg_rtol, o.cg_max, o.newton_rtol, o.newton_atol, o.newton_max = cg_rtol, cg_max, newton_rtol, newton_atol, newton_max
    o.ls_c1, o.ls_max, o.precond, o.check_every, o.use_graph = ls_c1, ls_max, precond, check_every, use_graph
    o.plastic_fixed_point = int(plastic_fixed_point)
    o.cg_forcing = float(cg_forcing)
    return o


def particles_from_tensors(x, v, F, G, mass, volume, mat, perm=None):
    """Build an mpml_particles view over torch tensors (CUDA or pinned/CPU) or numpy arrays."""
    def ptr(t):
        if t is None:
            return None
        if hasattr(t, "data_ptr"):
            return C.c_void_p(t.data_ptr())
        return C.c_void_p(t.ctypes.data)

    on_dev = hasattr(x, "is_cuda") and x.is_cuda
    p = mpml_particles()
    p.n = int(x.shape[0])
    p.mem = MEM_DEVICE if on_dev else MEM_HOST
    p.x, p.v, p.F, p.G = ptr(x), ptr(v), ptr(F), ptr(G)
    p.mass, p.volume, p.mat, p.perm = ptr(mass), ptr(volume), ptr(mat), ptr(perm)
    return p


def mpml_lame_parameters(E, nu):
    """(mu, lambda) from Young's modulus and Poisson's ratio (computed by the library)."""
    mu, lam = C.c_double(), C.c_double()
    _check(load().mpml_lame_parameters(float(E), float(nu), C.byref(mu), C.byref(lam)), "mpml_lame_parameters")
    return mu.value, lam.value


lame_parameters = mpml_lame_parameters


# ---------------------------------------------------------------------------
# learned preconditioner
# ---------------------------------------------------------------------------
NN_SHAPES = ((27, 16, 3), (27, 16, 16), (27, 3, 16))


def nn_pack(Ws):
    """Concatenate per-layer (27, Cout, Cin) arrays into the C layout (float32)."""
    return np.ascontiguousarray(np.concatenate([np.asarray(W, np.float32).ravel() for W in Ws]))


def nn_unpack(flat):
    out, off = [], 0
    for sh in NN_SHAPES:
        n = int(np.prod(sh))
        out.append(np.asarray(flat[off:off + n], np.float64).reshape(sh))
        off += n
    return out


def mpml_nn_weight_count():
    return int(load().mpml_nn_weight_count())


def mpml_nn_set_weights(ctx, Ws):
    w = nn_pack(Ws)
    return _check(load().mpml_nn_set_weights(ctx, w.ctypes.data_as(C.POINTER(C.c_float))), "mpml_nn_set_weights")


def mpml_nn_get_weights(ctx):
    w = np.zeros(mpml_nn_weight_count(), np.float32)
    _check(load().mpml_nn_get_weights(ctx, w.ctypes.data_as(C.POINTER(C.c_float))), "mpml_nn_get_weights")
    return nn_unpack(w)


def mpml_nn_get_grad(ctx):
    w = np.zeros(mpml_nn_weight_count(), np.float32)
    _check(load().mpml_nn_get_grad(ctx, w.ctypes.data_as(C.POINTER(C.c_float))), "mpml_nn_get_grad")
    return nn_unpack(w)


def mpml_nn_apply(ctx, r):
    r = np.ascontiguousarray(r, dtype=np.float64)
    z = np.zeros_like(r)
    _check(load().mpml_nn_apply(ctx, r.ctypes.data_as(_D), z.ctypes.data_as(_D)), "mpml_nn_apply")
    return z


def mpml_nn_loss_grad(ctx, r, e):
    r = np.ascontiguousarray(r, dtype=np.float64)
    e = np.ascontiguousarray(e, dtype=np.float64)
    loss = C.c_double()
    _check(load().mpml_nn_loss_grad(ctx, r.ctypes.data_as(_D), e.ctypes.data_as(_D), C.byref(loss)),
           "mpml_nn_loss_grad")
    return loss.value, mpml_nn_get_grad(ctx)


def mpml_nn_adam_step(ctx, lr):
    return _check(load().mpml_nn_adam_step(ctx, float(lr)), "mpml_nn_adam_step")


def train_opts(samples=32, rtol=1e-8, cg_max=20000, epochs=20, batch=4, lr=1e-3):
    o = mpml_train_opts()
    o.samples, o.rtol, o.cg_max, o.epochs, o.batch, o.lr = samples, rtol, cg_max, epochs, batch, lr
    return o


def mpml_nn_train(ctx, opts=None):
    st = mpml_train_stats()
    _check(load().mpml_nn_train(ctx, C.byref(opts if opts is not None else train_opts()), C.byref(st)),
           "mpml_nn_train")
    return st


def nn_init_weights(seed=0, gain=1.0):
    """Seeded He-style initialisation (numpy PCG64), per-layer (27, Cout, Cin)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    Ws = []
    for (t, cout, cin) in NN_SHAPES:
        Ws.append(gain * np.sqrt(2.0 / (27 * cin)) * rng.standard_normal((t, cout, cin)))
    return Ws


def mpml_sort_particles_noalloc(n, inv_dx, precision, x, perm, keys=None, stream=None):
    """Allocation-free sort of the particles at x (a CUDA tensor, n_particles x 3, float32 for FP32 or
    float64 for FP64) into perm (int32 CUDA tensor) and optionally keys (int64 CUDA tensor).
    stream: a torch.cuda.Stream or a raw cudaStream_t (None = legacy default stream).
    Returns the status code (raises on errors)."""
    nn = (C.c_int * 3)(*[int(a) for a in n])
    np_ = int(x.shape[0]) if x is not None else 0
    s = getattr(stream, "cuda_stream", stream)
    rc = load().mpml_sort_particles_noalloc(nn, float(inv_dx), int(precision),
                                            x.data_ptr() if x is not None else None, np_,
                                            perm.data_ptr() if perm is not None else None,
                                            keys.data_ptr() if keys is not None else None, s)
    return _check(rc, "mpml_sort_particles_noalloc")
