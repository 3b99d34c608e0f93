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
    n = x.shape[0]
    perm = torch.full((n,), -1, dtype=torch.int32, device="cuda")
    keys = torch.full((n,), -1, dtype=torch.int64, device="cuda")
    stream = torch.cuda.current_stream()
    rc = m.mpml_sort_particles_noalloc(sc.n, sc.inv_dx, prec, x, perm, keys, stream)
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
