"""Seeded synthetic scenes shaped like the paper's workloads.

This module only *generates inputs*: particle positions, velocities,
deformation gradients, masses, volumes, material ids and the scene
parameters.  It holds none of the method's arithmetic, so both the CUDA
path and the FP64 oracle can be fed from it without sharing any step of the
computation.

Seeding recipe (used by every scene): each voxel inside the shape receives
``ppc`` particles, stratified 2x2x2 per voxel with ``ppc // 8`` uniform
jittered samples per stratum (numpy PCG64 with the scene's seed), i.e.
``x = (voxel + (stratum + u) / 2) * dx`` with ``u ~ U[0,1)^3``.
``V_p = dx^3 / ppc``, ``m_p = rho * V_p``, ``F = I``, ``G = 0`` unless a scene
says otherwise.  Gravity is ``(0, -9.8, 0)``, the domain is the unit cube
(or ``n*dx`` per axis) with its origin at 0.
"""
from __future__ import annotations

import dataclasses
from typing import List, Optional, Tuple

import numpy as np

FIXED_COROTATED, NEO_HOOKEAN, HENCKY, WATER = 0, 1, 2, 3
ELASTIC, VON_MISES, DRUCKER_PRAGER = 0, 1, 2


@dataclasses.dataclass
class Material:
    model: int
    E: float
    nu: float
    rho: float = 1000.0
    plastic: int = ELASTIC
    yield_stress: float = 0.0
    friction_angle: float = 0.0  # radians


@dataclasses.dataclass
class Scene:
    name: str
    n: Tuple[int, int, int]
    dx: float
    inv_dx: float
    dt: float
    gravity: Tuple[float, float, float]
    materials: List[Material]
    wall_layers: int = 1
    plate: Optional[tuple] = None  # (lo3, hi3, vel3) moving Dirichlet box
    # particle arrays (float64; callers cast)
    x: np.ndarray = None
    v: np.ndarray = None
    F: np.ndarray = None
    G: np.ndarray = None
    mp: np.ndarray = None
    Vp: np.ndarray = None
    mat: np.ndarray = None

    @property
    def num_particles(self):
        return 0 if self.x is None else int(self.x.shape[0])

    def particles(self, dtype=np.float64):
        return dict(x=self.x.astype(dtype), v=self.v.astype(dtype), F=self.F.astype(dtype),
                    G=self.G.astype(dtype), mp=self.mp.astype(dtype), Vp=self.Vp.astype(dtype),
                    mat=self.mat.astype(np.int32))


def seed_voxels(voxels: np.ndarray, dx: float, ppc: int, rng: np.random.Generator) -> np.ndarray:
    """Stratified-jittered particle positions for integer voxel coordinates (N,3)."""
    assert ppc % 8 == 0, "ppc must be a multiple of 8 (2x2x2 strata)"
    per = ppc // 8
    strata = np.array([[a & 1, (a >> 1) & 1, (a >> 2) & 1] for a in range(8)], dtype=np.float64)
    nv = voxels.shape[0]
    base = np.repeat(voxels.astype(np.float64), 8 * per, axis=0)
    st = np.tile(np.repeat(strata, per, axis=0), (nv, 1))
    u = rng.random((nv * 8 * per, 3))
    return (base + (st + u) / 2.0) * dx


def _finish(sc: Scene, x, v, mat, ppc, F0=None):
    n = x.shape[0]
    sc.x = x
    sc.v = v
    sc.F = np.tile(np.eye(3), (n, 1, 1)) if F0 is None else np.tile(np.asarray(F0, float), (n, 1, 1))
    sc.G = np.zeros((n, 3, 3))
    Vp = sc.dx ** 3 / ppc
    sc.Vp = np.full(n, Vp)
    rho = np.array([m.rho for m in sc.materials])
    sc.mp = rho[mat] * Vp
    sc.mat = mat.astype(np.int32)
    return sc


def _grid_voxels(lo, hi):
    g = np.mgrid[lo[0]:hi[0], lo[1]:hi[1], lo[2]:hi[2]].reshape(3, -1).T
    return g.astype(np.int64)


def elastic_cube(variant: str = "fall", seed: int = 1, ppc: int = 8) -> Scene:
    """Fixed-corotated cube of 8^3 voxels at dx = 1/32 (E=1e5, nu=0.3, rho=1000), dt = 1e-3.

    variant 'fall': voxels [12,20)x[16,24)x[12,20) in free fall;
    'rest': voxels y in [1,9) touching the sticky floor;
    'stretched': as 'fall' with F0 = diag(1.05, 0.97, 1.0).
    """
    n = 32
    sc = Scene("elastic_cube_" + variant, (n, n, n), 1.0 / n, float(n), 1e-3, (0.0, -9.8, 0.0),
               [Material(FIXED_COROTATED, 1e5, 0.3)])
    rng = np.random.Generator(np.random.PCG64(seed))
    if variant == "rest":
        vox = _grid_voxels((12, 1, 12), (20, 9, 20))
    else:
        vox = _grid_voxels((12, 16, 12), (20, 24, 20))
    x = seed_voxels(vox, sc.dx, ppc, rng)
    F0 = np.diag([1.05, 0.97, 1.0]) if variant == "stretched" else None
    return _finish(sc, x, np.zeros_like(x), np.zeros(len(x), np.int64), ppc, F0)


def _sphere_voxels(n, center, radius, dx):
    g = _grid_voxels((0, 0, 0), (n, n, n))
    c = (g + 0.5) * dx
    return g[np.sum((c - np.asarray(center)) ** 2, axis=1) <= radius ** 2]


def two_spheres(n: int = 64, seed: int = 2, ppc: int = 8, gap: Optional[float] = None,
                dt: float = 2e-3) -> Scene:
    """Two Neo-Hookean spheres (E=1e6, nu=0.4, r=0.15) approaching at 2 m/s, no gravity.

    Default centres (0.3,0.5,0.5) and (0.7,0.5,0.5).  ``gap`` (metres) places the
    spheres that far apart along x instead, e.g. ``gap=dx`` to start at contact.
    """
    dx = 1.0 / n
    sc = Scene(f"two_spheres_{n}", (n, n, n), dx, float(n), dt, (0.0, 0.0, 0.0),
               [Material(NEO_HOOKEAN, 1e6, 0.4)])
    rng = np.random.Generator(np.random.PCG64(seed))
    r = 0.15
    if gap is None:
        c0, c1 = (0.3, 0.5, 0.5), (0.7, 0.5, 0.5)
    else:
        h = r + 0.5 * gap
        c0, c1 = (0.5 - h, 0.5, 0.5), (0.5 + h, 0.5, 0.5)
    v0 = _sphere_voxels(n, c0, r, dx)
    v1 = _sphere_voxels(n, c1, r, dx)
    x0 = seed_voxels(v0, dx, ppc, rng)
    x1 = seed_voxels(v1, dx, ppc, rng)
    x = np.concatenate([x0, x1])
    v = np.zeros_like(x)
    v[: len(x0), 0] = 1.0
    v[len(x0):, 0] = -1.0
    return _finish(sc, x, v, np.zeros(len(x), np.int64), ppc)


def pressed_block(n: int = 128, seed: int = 3, ppc: int = 8) -> Scene:
    """Stiff fixed-corotated block 0.5x0.3x0.5 (E=1e8, nu=0.33) on the floor under a plate.

    The block is x,z-centred with voxel rows y in [1, 1 + round(0.3 n)); a Dirichlet
    plate covering the block's top face moves down at 0.1 m/s.  dt = 1e-3.
    """
    dx = 1.0 / n
    sc = Scene(f"pressed_block_{n}", (n, n, n), dx, float(n), 1e-3, (0.0, -9.8, 0.0),
               [Material(FIXED_COROTATED, 1e8, 0.33)])
    wx = int(round(0.5 * n))
    wy = int(round(0.3 * n))
    x0 = (n - wx) // 2
    vox = _grid_voxels((x0, 1, x0), (x0 + wx, 1 + wy, x0 + wx))
    rng = np.random.Generator(np.random.PCG64(seed))
    x = seed_voxels(vox, dx, ppc, rng)
    top = (1 + wy) * dx
    lo = (x0 * dx, top, x0 * dx)
    hi = ((x0 + wx) * dx, top + 2 * dx, (x0 + wx) * dx)
    sc.plate = (lo, hi, (0.0, -0.1, 0.0))
    return _finish(sc, x, np.zeros_like(x), np.zeros(len(x), np.int64), ppc)


def slab_on_sand(n: int = 256, seed: int = 5, ppc: int = 8, dt: float = 2e-3, impact: bool = False) -> Scene:
    """A von Mises slab dropped onto a Drucker-Prager sand box (Hencky elasticity).
    Slab 0.6 x 0.1 x 0.6 at x, z in [0.35, 0.95], y in [0.5, 0.6] (E = 5e5, nu = 0.3,
    yield stress 2e3, rho = 1000); sand box 0.55 x 0.35 x 0.55 at x, z in [0.05, 0.6],
    y in [1/256, 0.35 + 1/256] (E = 1e6, nu = 0.3, friction angle 30 degrees, rho = 2000).
    Box edges are snapped to the voxel grid of size 1/n.

    ``impact=True`` starts at the moment of impact instead: the slab's lowest voxel row is
    one empty row above the sand's top row (so the trilinear stencils of both share a row of
    cells: mixed cells from the first step) and the slab moves down at the speed of a free
    fall from its original height, sqrt(2 g dh); the sand is at rest, F = I."""
    dx = 1.0 / n
    sc = Scene(f"slab_on_sand_{n}", (n, n, n), dx, float(n), dt, (0.0, -9.8, 0.0),
               [Material(HENCKY, 5e5, 0.3, 1000.0, VON_MISES, 2e3, 0.0),
                Material(HENCKY, 1e6, 0.3, 2000.0, DRUCKER_PRAGER, 0.0, float(np.radians(30.0)))])
    rng = np.random.Generator(np.random.PCG64(seed))

    def box(lo, hi):
        a = [int(round(v * n)) for v in lo]
        b = [int(round(v * n)) for v in hi]
        return _grid_voxels(a, b)

    y0 = 1.0 / 256
    slab = box((0.35, 0.5, 0.35), (0.95, 0.6, 0.95))
    sand = box((0.05, max(y0, 1.0 / n), 0.05), (0.6, 0.35 + y0, 0.6))
    v_slab = 0.0
    if impact:
        drop = int(slab[:, 1].min() - (sand[:, 1].max() + 2))  # voxel rows the slab falls
        slab = slab - np.array([0, drop, 0])
        v_slab = -float(np.sqrt(2.0 * 9.8 * drop * dx))
    xs = seed_voxels(slab, dx, ppc, rng)
    xb = seed_voxels(sand, dx, ppc, rng)
    x = np.concatenate([xs, xb])
    mat = np.concatenate([np.zeros(len(xs), np.int64), np.ones(len(xb), np.int64)])
    v = np.zeros_like(x)
    v[:len(xs), 1] = v_slab
    if impact:
        sc.name += "_impact"
    return _finish(sc, x, v, mat, ppc)


def batch_scene(index: int, n: int = 64, ppc: int = 8, dt: float = 1e-3,
                extent: Optional[int] = None, row: int = 2) -> Scene:
    """Scene ``index`` of the many-scene batch: its own n^3 unit domain, one fixed-corotated
    shape dropped onto the floor at 1 m/s.  Seeded with 4 + index: extent e ~ U{8..48} voxels
    (or ``extent``), shape box (e^3) / sphere (diameter e) / torus (R = 0.3 e, r = 0.15 e),
    E log-uniform in [1e4, 1e7] Pa, nu uniform in [0.2, 0.45]; the shape is centred in x, z
    with its lowest voxel in row ``row``: row 2 reaches the sticky floor after a short fall,
    row 1 touches it from the first step (the cells of that row reach node layer 0)."""
    rng = np.random.Generator(np.random.PCG64(4 + index))
    e = int(rng.integers(8, 49)) if extent is None else int(extent)
    shape = int(rng.integers(0, 3))
    E = float(10 ** rng.uniform(4.0, 7.0))
    nu = float(rng.uniform(0.2, 0.45))
    dx = 1.0 / n
    sc = Scene(f"batch_{index}_{['box', 'sphere', 'torus'][shape]}{e}", (n, n, n), dx, float(n), dt,
               (0.0, -9.8, 0.0), [Material(FIXED_COROTATED, E, nu)])
    lo = np.array([(n - e) // 2, row, (n - e) // 2])
    g = _grid_voxels(lo, lo + e)
    c = (g + 0.5 - lo - e / 2.0)  # voxel centres relative to the shape centre, in voxels
    if shape == 1:
        keep = np.sum(c * c, axis=1) <= (e / 2.0) ** 2
    elif shape == 2:
        R, r = 0.3 * e, 0.15 * e
        rho = np.sqrt(c[:, 0] ** 2 + c[:, 2] ** 2)
        keep = (rho - R) ** 2 + c[:, 1] ** 2 <= r * r
    else:
        keep = np.ones(len(g), bool)
    vox = g[keep]
    x = seed_voxels(vox, dx, ppc, rng)
    v = np.zeros_like(x)
    v[:, 1] = -1.0
    return _finish(sc, x, v, np.zeros(len(x), np.int64), ppc)


def dam_break(n: int = 64, seed: int = 8, ppc: int = 8, dt: float = 1e-3, with_cube: bool = True) -> Scene:
    """Water column collapsing in the unit box (Sec. "Water"): voxels x in [0.05, 0.4),
    y in [1/n, 0.55), z in [0.05, 0.95) of water (E = 1e5, nu = 0.45: bulk modulus
    3.3e5 Pa, rho = 1000), gravity, sticky walls; with ``with_cube`` a fixed-corotated
    cube (E = 1e5, nu = 0.3, rho = 500) of 0.15 m rests on the floor in the flow's path,
    so mixed water / solid cells arise when the front reaches it."""
    mats = [Material(WATER, 1e5, 0.45)]
    if with_cube:
        mats.append(Material(FIXED_COROTATED, 1e5, 0.3, rho=500.0))
    sc = Scene("dam_break", (n, n, n), 1.0 / n, float(n), dt, (0.0, -9.8, 0.0), mats)
    rng = np.random.Generator(np.random.PCG64(seed))
    lo = np.array([0.05, 1.0 / n, 0.05])
    hi = np.array([0.4, 0.55, 0.95])
    vw = _grid_voxels(tuple(np.ceil(lo * n - 1e-9).astype(int)), tuple(np.floor(hi * n + 1e-9).astype(int)))
    xw = seed_voxels(vw, sc.dx, ppc, rng)
    xs, ms = [xw], [np.zeros(len(xw), np.int64)]
    if with_cube:
        c0 = np.array([0.6, 1.0 / n, 0.425])
        vc = _grid_voxels(tuple(np.round(c0 * n).astype(int)), tuple(np.round((c0 + 0.15) * n).astype(int)))
        xc = seed_voxels(vc, sc.dx, ppc, rng)
        xs.append(xc)
        ms.append(np.ones(len(xc), np.int64))
    x = np.concatenate(xs)
    return _finish(sc, x, np.zeros_like(x), np.concatenate(ms), ppc)


def colliding_cubes(n: int = 64, seed: int = 6, ppc: int = 8, speed: float = 1.0) -> Scene:
    """Two 0.1 m elastic cubes (E=5e3, nu=0.3, rho=1e3) moving at +-speed along x, no gravity
    (the linear-momentum experiment of Sec. 6.6; its speed is not given, 1 m/s here)."""
    dx = 1.0 / n
    sc = Scene(f"colliding_cubes_{n}", (n, n, n), dx, float(n), 1e-3, (0.0, 0.0, 0.0),
               [Material(FIXED_COROTATED, 5e3, 0.3)])
    w = int(round(0.1 * n))
    y0 = (n - w) // 2
    a = _grid_voxels((n // 2 - w - 1, y0, y0), (n // 2 - 1, y0 + w, y0 + w))
    b = _grid_voxels((n // 2 + 1, y0, y0), (n // 2 + 1 + w, y0 + w, y0 + w))
    rng = np.random.Generator(np.random.PCG64(seed))
    xa, xb = seed_voxels(a, dx, ppc, rng), seed_voxels(b, dx, ppc, rng)
    x = np.concatenate([xa, xb])
    v = np.zeros_like(x)
    v[: len(xa), 0] = speed
    v[len(xa):, 0] = -speed
    return _finish(sc, x, v, np.zeros(len(x), np.int64), ppc)


def rotating_rod(n: int = 64, seed: int = 7, ppc: int = 8, omega: float = 4.0) -> Scene:
    """Rod along z (radius 0.05 m, length 0.4 m) spinning at omega_z, no gravity
    (the angular-momentum experiment of Sec. 6.6; material as the elastic cube)."""
    dx = 1.0 / n
    sc = Scene(f"rotating_rod_{n}", (n, n, n), dx, float(n), 1e-3, (0.0, 0.0, 0.0),
               [Material(FIXED_COROTATED, 1e5, 0.3)])
    g = _grid_voxels((0, 0, 0), (n, n, n))
    c = (g + 0.5) * dx
    keep = ((c[:, 0] - 0.5) ** 2 + (c[:, 1] - 0.5) ** 2 <= 0.05 ** 2) & (np.abs(c[:, 2] - 0.5) <= 0.2)
    rng = np.random.Generator(np.random.PCG64(seed))
    x = seed_voxels(g[keep], dx, ppc, rng)
    v = np.zeros_like(x)
    v[:, 0] = -omega * (x[:, 1] - 0.5)
    v[:, 1] = omega * (x[:, 0] - 0.5)
    sc = _finish(sc, x, v, np.zeros(len(x), np.int64), ppc)
    # affine velocity field of a rigid rotation: G = [[0,-w,0],[w,0,0],[0,0,0]]
    sc.G[:, 0, 1] = -omega
    sc.G[:, 1, 0] = omega
    return sc


def random_state(sc: Scene, seed: int, v_scale=0.1, G_scale=1.0, F_scale=0.02) -> Scene:
    """Perturb a scene's particle v, G and F with seeded noise (parity tests)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    n = sc.num_particles
    sc.v = sc.v + v_scale * rng.standard_normal((n, 3))
    sc.G = sc.G + G_scale * rng.standard_normal((n, 3, 3))
    sc.F = sc.F + F_scale * rng.standard_normal((n, 3, 3))
    return sc
