"""mpml_sort_particles_noalloc (static device scratch, no allocation) against
the particle order and keys of mpml_resample, bit-exact.

Collected last on purpose: it must pass both alone in a fresh process (the
first call performs the per-device scratch look-up) and after every other
test has used the library.
"""
import numpy as np
import pytest
import torch

import paper_2602_07853_gb300.mpml as m
from paper_2602_07853_gb300 import scenes
from tests._gpu import GpuSim

pytestmark = pytest.mark.gpu


@pytest.fixture(autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.set_device(0)


def resample_order(sc, prec):
    """Particle positions on the device and the order / keys mpml_resample gives them."""
    g = GpuSim(sc, prec)
    g.set_particles()
    g.resample()
    m.mpml_sync(g.ctx)
    perm = g.t["perm"].cpu().numpy().copy()
    keys = g.keys(m.KEYS_PARTICLES)
    x = g.t["x"].clone()
    g.close()
    return x, perm, keys


def noalloc_order(sc, prec, x):
    return noalloc_order_grid(sc.n, sc.inv_dx, prec, x)


def noalloc_order_grid(grid, inv_dx, prec, x):
    n = x.shape[0]
    perm = torch.full((n,), -1, dtype=torch.int32, device="cuda")
    keys = torch.full((n,), -1, dtype=torch.int64, device="cuda")
    stream = torch.cuda.current_stream()
    rc = m.mpml_sort_particles_noalloc(grid, inv_dx, prec, x, perm, keys, stream)
    assert rc == m.OK
    return perm.cpu().numpy(), keys.cpu().numpy()


def test_noalloc_sort_matches_resample_on_consecutive_calls():
    # larger grid first, so that stale counters of the first call would corrupt the second
    cases = [(scenes.two_spheres(64, gap=1.0 / 64), m.FP64), (scenes.elastic_cube("fall"), m.FP32),
             (scenes.two_spheres(64, gap=1.0 / 64), m.FP32)]
    for sc, prec in cases:
        x, perm_ref, keys_ref = resample_order(sc, prec)
        assert len(perm_ref) > 0
        perm, keys = noalloc_order(sc, prec, x)
        assert np.array_equal(perm, perm_ref)
        assert np.array_equal(keys, keys_ref)


def test_noalloc_sort_errors_then_recovers():
    sc = scenes.elastic_cube("fall")
    x, perm_ref, keys_ref = resample_order(sc, m.FP32)
    n = x.shape[0]
    perm = torch.zeros(n, dtype=torch.int32, device="cuda")
    # particle 5 outside the grid: reported, nothing written out of bounds
    bad = x.clone()
    bad[5, 1] = -1.0
    with pytest.raises(m.MPMLError) as e:
        m.mpml_sort_particles_noalloc(sc.n, sc.inv_dx, m.FP32, bad, perm, None, torch.cuda.current_stream())
    assert e.value.code == m.ERR_OUT_OF_DOMAIN
    bad[5, 1] = float("nan")
    with pytest.raises(m.MPMLError) as e:
        m.mpml_sort_particles_noalloc(sc.n, sc.inv_dx, m.FP32, bad, perm, None, torch.cuda.current_stream())
    assert e.value.code == m.ERR_NONFINITE
    # grid above the scratch capacity: rejected on the host
    with pytest.raises(m.MPMLError) as e:
        m.mpml_sort_particles_noalloc((128, 128, 128), sc.inv_dx, m.FP32, x, perm, None, torch.cuda.current_stream())
    assert e.value.code == m.ERR_TOO_LARGE
    # the status word is cleared by the next call
    perm2, keys2 = noalloc_order(sc, m.FP32, x)
    assert np.array_equal(perm2, perm_ref)
    assert np.array_equal(keys2, keys_ref)


def host_order(x, n, inv_dx):
    """Brute-force order on the host: brick-major key of floor(x/dx - 1/2) (FP64, no fused
    multiply-add), stable in the input index."""
    s = x.astype(np.float64) * inv_dx - 0.5
    b = np.floor(s).astype(np.int64)
    NB = [(a >> 3) + 1 for a in n]
    brick = ((b[:, 2] >> 3) * NB[1] + (b[:, 1] >> 3)) * NB[0] + (b[:, 0] >> 3)
    key = brick * 512 + (b[:, 2] & 7) * 64 + (b[:, 1] & 7) * 8 + (b[:, 0] & 7)
    perm = np.argsort(key, kind="stable")
    return perm.astype(np.int32), key[perm]


def test_noalloc_sort_at_the_capacity_edge():
    """A 127^3 grid has NB = 16 bricks per axis, exactly MPML_NOALLOC_MAX_SLOTS = 2^21 dense slots,
    so the scan runs with as many block sums as one scan block holds.  Particles fill the last
    brick and the far faces; order and keys against a host stable argsort and mpml_resample."""
    n = (127, 127, 127)
    assert 16 ** 3 * 512 == m.NOALLOC_MAX_SLOTS
    inv_dx = 127.0
    rng = np.random.default_rng(21)
    far = rng.uniform(120.5, 126.5 - 1e-3, (4000, 3)) / inv_dx            # the last brick
    face = rng.uniform(1.0, 126.0, (6000, 3)) / inv_dx
    face[np.arange(6000), rng.integers(0, 3, 6000)] = (126.5 - 1e-3) / inv_dx  # on a far face
    x = np.concatenate([far, face, rng.uniform(1.0, 126.0, (2000, 3)) / inv_dx]).astype(np.float32)
    xt = torch.from_numpy(x).cuda()
    perm, keys = noalloc_order_grid(n, inv_dx, m.FP32, xt)
    perm_h, keys_h = host_order(x, n, inv_dx)
    assert np.array_equal(perm, perm_h)
    assert np.array_equal(keys, keys_h)
    assert keys.max() >= m.NOALLOC_MAX_SLOTS - 512  # the last brick is used
    sc = scenes.Scene("edge", n, 1.0 / 127, inv_dx, 1e-3, (0.0, -9.8, 0.0),
                      [scenes.Material(scenes.FIXED_COROTATED, 1e5, 0.3)])
    sc = scenes._finish(sc, x.astype(np.float64), np.zeros_like(x, dtype=np.float64),
                        np.zeros(len(x), np.int64), 8)
    _, perm_ref, keys_ref = resample_order(sc, m.FP32)
    assert np.array_equal(perm, perm_ref)
    assert np.array_equal(keys, keys_ref)


def test_noalloc_sort_crowded_centres():
    """Centres holding many particles (compressed material): 40 and 3000 particles share one
    centre each (the block-wide rank sort) and 5000 another (the single-thread fallback); the
    within-centre order is the input order."""
    n = (32, 32, 32)
    inv_dx = 32.0
    rng = np.random.default_rng(22)
    parts = [rng.uniform(2.0, 30.0, (3000, 3))]
    for cnt, cell in ((40, 5), (3000, 9), (5000, 20)):
        parts.append(cell + 0.5 + rng.uniform(0.0, 0.99, (cnt, 3)))
    x = np.concatenate(parts) / inv_dx
    x = x[rng.permutation(len(x))].astype(np.float32)
    xt = torch.from_numpy(x).cuda()
    for _ in range(2):  # two calls in a row share the scratch array
        perm, keys = noalloc_order_grid(n, inv_dx, m.FP32, xt)
        perm_h, keys_h = host_order(x, n, inv_dx)
        assert np.array_equal(perm, perm_h)
        assert np.array_equal(keys, keys_h)
