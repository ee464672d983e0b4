"""Tile-width table of the autotuner: host-only record / lookup, shape
buckets, the JSON cache round trip and rejection of malformed files; on a GPU,
css_autotune_select times the three widths and records the fastest."""
import ctypes as C
import json

import pytest
import torch

from paper_1312_6838_gb300 import _lib as L


@pytest.fixture(scope="module")
def lib():
    from paper_1312_6838_gb300 import build
    build.build()
    return L.load()


def test_record_lookup_and_buckets(lib):
    dev = b"Test GPU A"
    assert lib.css_tile_lookup(dev, L.CSS_BF16, 4096, 65536) == 0
    assert lib.css_tile_record(dev, L.CSS_BF16, 4096, 65536, 4) == 0
    assert lib.css_tile_lookup(dev, L.CSS_BF16, 4096, 65536) == 4
    # same power-of-two bucket: 4096..8191 rows, 65536..131071 columns
    assert lib.css_tile_lookup(dev, L.CSS_BF16, 8191, 100000) == 4
    assert lib.css_tile_lookup(dev, L.CSS_BF16, 8192, 65536) == 0
    assert lib.css_tile_lookup(dev, L.CSS_F32, 4096, 65536) == 0
    assert lib.css_tile_lookup(b"Other GPU", L.CSS_BF16, 4096, 65536) == 0
    assert lib.css_tile_record(dev, L.CSS_BF16, 4096, 65536, 3) == L.CSS_ERR_INVALID_ARG
    assert lib.css_tile_record(b"", L.CSS_BF16, 4096, 65536, 2) == L.CSS_ERR_INVALID_ARG
    assert lib.css_tile_record(b'bad"name', L.CSS_BF16, 4096, 65536, 2) == L.CSS_ERR_INVALID_ARG
    assert lib.css_tile_record(dev, L.CSS_BF16, 0, 65536, 2) == L.CSS_ERR_INVALID_ARG


def test_cache_round_trip(lib, tmp_path):
    dev = b"Test GPU B"
    assert lib.css_tile_record(dev, L.CSS_F32, 1000, 3000, 2) == 0
    assert lib.css_tile_record(dev, L.CSS_F64, 500, 1000, 8) == 0
    path = tmp_path / "tiles.json"
    assert lib.css_tile_cache_save(str(path).encode()) == 0
    data = json.loads(path.read_text())
    assert data["Test GPU B|f32|m9|n11"] == 2
    assert data["Test GPU B|f64|m8|n9"] == 8
    # a file written by another process merges into the table
    other = tmp_path / "other.json"
    other.write_text(json.dumps({"Test GPU C|bf16|m12|n16": 8, "Test GPU C|f32|m6|n10": 4}))
    assert lib.css_tile_cache_load(str(other).encode()) == 0
    assert lib.css_tile_lookup(b"Test GPU C", L.CSS_BF16, 4096, 65536) == 8
    assert lib.css_tile_lookup(b"Test GPU C", L.CSS_F32, 64, 1024) == 4


@pytest.mark.parametrize("text", ['{"x": 3}', '{"x": }', '[1, 2]', '{"x": 4', ''])
def test_malformed_cache_rejected(lib, tmp_path, text):
    path = tmp_path / "bad.json"
    path.write_text(text)
    assert lib.css_tile_cache_load(str(path).encode()) == L.CSS_ERR_INVALID_ARG
    assert lib.css_tile_lookup(b"x", L.CSS_BF16, 1, 1) == 0
    assert lib.css_tile_cache_load(str(tmp_path / "missing.json").encode()) == L.CSS_ERR_INVALID_ARG


@pytest.mark.gpu
def test_autotune_records_the_fastest_width(lib):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1312_6838_gb300 import css
    import css_inputs as ci
    from tests.gpu_helpers import dev_matrix
    A, _ = dev_matrix(ci.lowrank_uv(512, 20000, 16, 0.01, 31), torch.bfloat16)
    best, times = css.autotune(A, 8)
    assert best in (2, 4, 8)
    assert all(t > 0 for t in times.values())
    assert times[best] == min(times.values())
    name = torch.cuda.get_device_name().encode()
    assert lib.css_tile_lookup(name, L.CSS_BF16, 512, 20000) == best
