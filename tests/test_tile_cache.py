"""Host side of the HVP launch-shape autotuner (no GPU): the process-wide cache's
text round trip, rejection of malformed files, and argument checks of the tile
calls.  The timing itself and the per-shape parity live in test_gpu_autotune."""
import ctypes as C

import pytest

import paper_2602_07853_gb300.mpml as m

pytestmark = pytest.mark.filterwarnings("ignore")


@pytest.fixture(autouse=True)
def _clean_cache():
    m.mpml_tile_cache_clear()
    yield
    m.mpml_tile_cache_clear()


def entries(path):
    rows = []
    for line in open(path):
        f = line.split()
        rows.append((int(f[0]), int(f[1]), int(f[2]), float(f[3])))
    return sorted(rows)


def test_cache_round_trip(tmp_path):
    src = tmp_path / "tiles.txt"
    src.write_text("25 10 1 0.5\n\n45 12 0 1.25\n25 3 2 0.0125\n")
    m.mpml_tile_cache_load(src)
    out = tmp_path / "out.txt"
    m.mpml_tile_cache_save(out)
    assert entries(out) == [(25, 3, 2, 0.0125), (25, 10, 1, 0.5), (45, 12, 0, 1.25)]
    # loading merges: a later file overrides the same key and keeps the others
    upd = tmp_path / "upd.txt"
    upd.write_text("25 10 0 0.4\n")
    m.mpml_tile_cache_load(upd)
    m.mpml_tile_cache_save(out)
    assert entries(out) == [(25, 3, 2, 0.0125), (25, 10, 0, 0.4), (45, 12, 0, 1.25)]


def test_persistent_solver_shapes_round_trip(tmp_path):
    """Formats 125 / 145 hold the persistent solver's shapes (0 .. PCG_SHAPES - 1)."""
    src = tmp_path / "pcg.txt"
    src.write_text(f"125 11 {m.PCG_SHAPES - 1} 2.5\n145 12 4 3.75\n25 11 0 0.5\n")
    m.mpml_tile_cache_load(src)
    out = tmp_path / "out.txt"
    m.mpml_tile_cache_save(out)
    assert entries(out) == [(25, 11, 0, 0.5), (125, 11, m.PCG_SHAPES - 1, 2.5), (145, 12, 4, 3.75)]


@pytest.mark.parametrize("bad", ["25 10 3 0.5\n",       # tile out of range
                                 f"145 10 {m.PCG_SHAPES} 0.5\n",  # persistent shape out of range
                                 "33 10 1 0.5\n",       # unknown tangent format
                                 "25 10 1\n",           # missing field
                                 "25 -1 1 0.5\n",       # negative size class
                                 "45 4 1 -2\n",         # negative time
                                 "45 4 1 0.5 junk\n"])  # trailing text
def test_malformed_cache_is_rejected_whole(tmp_path, bad):
    good = tmp_path / "good.txt"
    good.write_text("45 7 1 0.25\n")
    m.mpml_tile_cache_load(good)
    f = tmp_path / "bad.txt"
    f.write_text("25 5 0 0.125\n" + bad)
    with pytest.raises(m.MPMLError) as e:
        m.mpml_tile_cache_load(f)
    assert e.value.code == m.ERR_ARG
    out = tmp_path / "out.txt"
    m.mpml_tile_cache_save(out)
    assert entries(out) == [(45, 7, 1, 0.25)]  # nothing of the bad file merged


def test_missing_file_and_null_context(tmp_path):
    with pytest.raises(m.MPMLError):
        m.mpml_tile_cache_load(tmp_path / "absent.txt")
    lib = m.load()
    tile = C.c_int()
    assert lib.mpml_autotune_hvp(None, 1, C.byref(tile), None) == m.ERR_ARG
    assert lib.mpml_set_hvp_tile(None, 0) == m.ERR_ARG
    assert lib.mpml_get_hvp_tile(None, C.byref(tile), None) == m.ERR_ARG
