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


def test_plan_knobs_record_lookup_and_cache(lib, tmp_path):
    """Split share and pivot cost live in the same table under their own key
    suffixes, with their own value ranges, and survive the JSON round trip."""
    dev = b"Test GPU D"
    assert lib.css_tune_lookup(dev, L.CSS_BF16, 4096, 65536, L.CSS_KNOB_SPLIT_SHARE) == -1
    assert lib.css_tune_record(dev, L.CSS_BF16, 4096, 65536, L.CSS_KNOB_SPLIT_SHARE, 4) == 0
    assert lib.css_tune_record(dev, L.CSS_BF16, 2048, 262144, L.CSS_KNOB_PIVOT_COST, 300) == 0
    assert lib.css_tune_record(dev, L.CSS_BF16, 2048, 262144, L.CSS_KNOB_PIVOT_COST, 0) == 0
    assert lib.css_tune_lookup(dev, L.CSS_BF16, 4096, 65536, L.CSS_KNOB_SPLIT_SHARE) == 4
    assert lib.css_tune_lookup(dev, L.CSS_BF16, 2048, 262144, L.CSS_KNOB_PIVOT_COST) == 0
    # the tile knob is the tile table
    assert lib.css_tune_record(dev, L.CSS_BF16, 4096, 65536, L.CSS_KNOB_TILE_COLS, 2) == 0
    assert lib.css_tile_lookup(dev, L.CSS_BF16, 4096, 65536) == 2
    # each knob's own range
    assert lib.css_tune_record(dev, L.CSS_BF16, 4096, 65536, L.CSS_KNOB_SPLIT_SHARE, 3) == L.CSS_ERR_INVALID_ARG
    assert lib.css_tune_record(dev, L.CSS_BF16, 4096, 65536, L.CSS_KNOB_PIVOT_COST, -1) == L.CSS_ERR_INVALID_ARG
    assert lib.css_tune_record(dev, L.CSS_BF16, 4096, 65536, L.CSS_KNOB_PIVOT_COST, 1000001) == L.CSS_ERR_INVALID_ARG
    assert lib.css_tune_record(dev, L.CSS_BF16, 4096, 65536, 7, 2) == L.CSS_ERR_INVALID_ARG
    path = tmp_path / "knobs.json"
    assert lib.css_tile_cache_save(str(path).encode()) == 0
    data = json.loads(path.read_text())
    assert data["Test GPU D|bf16|m12|n16|split"] == 4
    assert data["Test GPU D|bf16|m11|n18|pivot"] == 0
    other = tmp_path / "more.json"
    other.write_text(json.dumps({"Test GPU E|f32|m12|n16|pivot": 1500, "Test GPU E|f32|m12|n16|split": 8}))
    assert lib.css_tile_cache_load(str(other).encode()) == 0
    assert lib.css_tune_lookup(b"Test GPU E", L.CSS_F32, 4096, 65536, L.CSS_KNOB_PIVOT_COST) == 1500
    assert lib.css_tune_lookup(b"Test GPU E", L.CSS_F32, 4096, 65536, L.CSS_KNOB_SPLIT_SHARE) == 8


@pytest.mark.parametrize("text", ['{"x|split": 3}', '{"x|pivot": 12345678}', '{"x|split": 16}'])
def test_malformed_knob_values_rejected(lib, tmp_path, text):
    path = tmp_path / "bad_knob.json"
    path.write_text(text)
    assert lib.css_tile_cache_load(str(path).encode()) == L.CSS_ERR_INVALID_ARG


@pytest.mark.gpu
def test_split_share_keeps_the_selection(lib):
    """Every split share hands out the same work in other units: the same
    picks on a problem inside its numerical rank, and rejection of values
    outside 1, 2, 4, 8."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1312_6838_gb300 import css
    import css_inputs as ci
    from tests.gpu_helpers import dev_matrix
    A, _ = dev_matrix(ci.lowrank_uv(256, 30000, 32, 0.01, 33), torch.bfloat16)
    ref = css.select(A, 16, split_share=2).indices.cpu().tolist()
    for share in (1, 4, 8):
        assert css.select(A, 16, split_share=share).indices.cpu().tolist() == ref
    with pytest.raises(L.CssError):
        css.select(A, 16, split_share=3)


@pytest.mark.gpu
def test_autotune_records_split_share_and_pivot_cost(lib):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1312_6838_gb300 import css
    import css_inputs as ci
    from tests.gpu_helpers import dev_matrix
    name = torch.cuda.get_device_name().encode()
    A, _ = dev_matrix(ci.lowrank_uv(512, 20000, 16, 0.01, 34), torch.bfloat16)
    css.autotune(A, 8)
    assert lib.css_tune_lookup(name, L.CSS_BF16, 512, 20000, L.CSS_KNOB_SPLIT_SHARE) in (1, 2, 4)
    import numpy as np
    A_np = ci.lowrank_uv(256, 12000, 24, 0.05, 35)
    A2, _ = dev_matrix(A_np, torch.bfloat16)
    B = css.to_colmajor(torch.from_numpy(A_np @ ci.gaussian_omega(12000, 32, 36, dtype=np.float64)).float().cuda())
    offs = ci.lognormal_blocks(12000, 8, 1500, 0.8, 37).tolist()
    best, times = css.autotune_distributed(A2, B, offs, 20, 20)
    assert best in (300, 700, 1500, 3000)
    assert times[best] == min(times.values())
    assert lib.css_tune_lookup(name, L.CSS_BF16, 256, 12000, L.CSS_KNOB_PIVOT_COST) == best
    # the recorded cost is what the next call without a cost uses; results stay valid
    got = css.distributed(A2, B, offs, 20, 20)
    assert got.n_sel == 20
