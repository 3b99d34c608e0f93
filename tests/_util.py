"""Test helpers: build oracle scenes from the seeded generator, brute-force references."""
import numpy as np

import oracle
from paper_2602_07853_gb300 import scenes


def oracle_scene(sc: scenes.Scene, time=0.0):
    return oracle.make_scene(sc.n, sc.dx, sc.dt, sc.gravity,
                             [(m.model, m.E, m.nu, m.plastic, m.yield_stress, m.friction_angle)
                              for m in sc.materials],
                             wall_layers=sc.wall_layers, plate=sc.plate, inv_dx=sc.inv_dx, time=time)


def make_oracle(sc: scenes.Scene, time=0.0):
    return oracle.Oracle(oracle_scene(sc, time))


def brick_key_np(ijk, n):
    """Brick-major key of integer coordinates (numpy restatement, for brute-force checks)."""
    n = (n, n, n) if np.isscalar(n) else tuple(n)
    ijk = np.asarray(ijk, dtype=np.int64)
    nbx, nby = (n[0] >> 3) + 1, (n[1] >> 3) + 1
    i, j, k = ijk[:, 0], ijk[:, 1], ijk[:, 2]
    b = ((k >> 3) * nby + (j >> 3)) * nbx + (i >> 3)
    return b * 512 + (k & 7) * 64 + (j & 7) * 8 + (i & 7)


def brute_force_sets(x, inv_dx, n):
    """Base cells, stable order, active cells and DOF nodes by brute force in numpy."""
    s = x.astype(np.float64) * inv_dx - 0.5
    b = np.floor(s).astype(np.int64)
    f = s - b
    keys = brick_key_np(b, n)
    perm = np.argsort(keys, kind="stable")
    cells = set()
    for p in range(len(x)):
        for o in range(8):
            oa = np.array([o & 1, (o >> 1) & 1, (o >> 2) & 1])
            w = np.prod(np.where(oa == 1, f[p], 1 - f[p]))
            if w > 0:
                cells.add(tuple(b[p] + oa))
    cells = np.array(sorted(cells), dtype=np.int64).reshape(-1, 3)
    ckeys = np.sort(brick_key_np(cells, n))
    nodes = set()
    for c in cells:
        for o in range(8):
            nodes.add((c[0] + (o & 1), c[1] + ((o >> 1) & 1), c[2] + ((o >> 2) & 1)))
    nodes = np.array(sorted(nodes), dtype=np.int64).reshape(-1, 3)
    nkeys = np.sort(brick_key_np(nodes, n))
    return keys[perm], perm, ckeys, nkeys
