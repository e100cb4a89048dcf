"""The autotuner's shape table and its JSON cache, on the CPU (no CUDA call):
values round-trip through the file, a file written for another device or
SM count is refused and loads nothing, a malformed file is refused, and
clearing the table restores the fixed rules (lookups return -1)."""
import os

import pytest

from paper_2402_12833_gb300 import mpcg as M


@pytest.fixture()
def lib():
    try:
        M.load()
    except OSError as e:   # pragma: no cover - the library is built by the suite's first tests
        pytest.skip(str(e))
    M.mg_autotune_clear()
    yield M
    M.mg_autotune_clear()


def test_cache_round_trip(lib, tmp_path):
    path = str(tmp_path / "tune.json")
    rows = [(M.MG_TUNE_STREAM_BLOCKS, M.MG_TUNE_ANY, 2146689, 1, 0, 912),
            (M.MG_TUNE_SPMM_BLOCKS, M.MG_TUNE_F32, 2146689, 1, 6, 456),
            (M.MG_TUNE_GRAM_CHUNKS, M.MG_TUNE_ANY, 2146689, 1, 0, 526),
            (M.MG_TUNE_JACOBI_NARROW, M.MG_TUNE_DW, 35937, 3, 0, 1)]
    for r in rows:
        M.mg_autotune_set(*r)
    M.mg_autotune_save(path, "NVIDIA GB300", 152)
    M.mg_autotune_clear()
    assert M.mg_autotune_lookup(*rows[0][:5]) == -1
    assert M.mg_autotune_load(path, "NVIDIA GB300", 152) == len(rows)
    for r in rows:
        assert M.mg_autotune_lookup(*r[:5]) == r[5], r
    # a different column count or arithmetic is a different key
    assert M.mg_autotune_lookup(M.MG_TUNE_SPMM_BLOCKS, M.MG_TUNE_F32, 2146689, 1, 7) == -1
    assert M.mg_autotune_lookup(M.MG_TUNE_SPMM_BLOCKS, M.MG_TUNE_F64, 2146689, 1, 6) == -1


def test_cache_for_another_device_is_refused(lib, tmp_path):
    path = str(tmp_path / "tune.json")
    M.mg_autotune_set(M.MG_TUNE_STREAM_BLOCKS, M.MG_TUNE_ANY, 1000, 1, 0, 304)
    M.mg_autotune_save(path, "NVIDIA GB300", 152)
    M.mg_autotune_clear()
    for dev, sms in (("NVIDIA B200", 148), ("NVIDIA GB300", 148)):
        with pytest.raises(M.MpcgError) as e:
            M.mg_autotune_load(path, dev, sms)
        assert e.value.status == M.MPCG_ERR_ARG and "another device" in M.mpcg_last_error()
        assert M.mg_autotune_lookup(M.MG_TUNE_STREAM_BLOCKS, M.MG_TUNE_ANY, 1000, 1, 0) == -1


def test_malformed_or_missing_cache_is_refused(lib, tmp_path):
    bad = tmp_path / "bad.json"
    bad.write_text('{"format": "mpcg-autotune-1", "device": "NVIDIA GB300", "sm_count": 152, "entries": [\n'
                   '  {"fn": "no_such_shape", "kind": 0, "npts": 10, "nb": 1, "C": 0, "value": 1}\n]}\n')
    with pytest.raises(M.MpcgError):
        M.mg_autotune_load(str(bad), "NVIDIA GB300", 152)
    with pytest.raises(M.MpcgError):
        M.mg_autotune_load(str(tmp_path / "missing.json"), "NVIDIA GB300", 152)
    assert not os.path.exists(tmp_path / "missing.json")
