"""The autotuner's plan cache, on the host (no GPU): keys, round trips, and the
rule that a missing, corrupt or foreign cache file only means the sweep runs
again and the file is rewritten."""
import json
import os

import pytest

from paper_2607_02749_gb300 import _lib
from paper_2607_02749_gb300 import workloads as wl


@pytest.fixture
def handles():
    ham = wl.z_hamiltonian(10, 20, seed=0)
    h = _lib.gvqe_hamiltonian_create(10, ham.strings, ham.coeffs)
    a = _lib.gvqe_ansatz_create(10, 2, _lib.GVQE_ENT_LINEAR)
    yield a, h
    _lib.gvqe_destroy(a)
    _lib.gvqe_destroy(h)


def test_key_names_every_dimension(handles):
    a, h = handles
    k32 = _lib.gvqe_tune_key(a, h, 4, _lib.GVQE_FP32)
    k64 = _lib.gvqe_tune_key(a, h, 4, _lib.GVQE_FP64)
    ke = _lib.gvqe_tune_key(a, h, 4, _lib.GVQE_FP32 | _lib.GVQE_TUNE_ENERGY)
    kb = _lib.gvqe_tune_key(a, h, 1, _lib.GVQE_FP32)
    assert len({k32, k64, ke, kb}) == 4
    for part in ("gpu=", "n=10", "reps=2", "ent=0", "gates=1", "prec=fp32", "grad=1", "diag=1", "batch=4"):
        assert part in k32
    assert "grad=0" in ke and "prec=fp64" in k64 and "batch=1" in kb


def test_key_tells_diagonal_from_xy_hamiltonians(handles):
    a, _ = handles
    ham = wl.pauli_hamiltonian(10, 30, seed=1)
    h = _lib.gvqe_hamiltonian_create(10, ham.strings, ham.coeffs)
    try:
        assert "diag=0" in _lib.gvqe_tune_key(a, h, 1, _lib.GVQE_FP32)
    finally:
        _lib.gvqe_destroy(h)


def test_round_trip_and_replace(tmp_path):
    p = str(tmp_path / "tune.json")
    assert _lib.gvqe_tune_cache_get(p, "k1") is None  # no file yet
    _lib.gvqe_tune_cache_put(p, "k1", 13, 1, 12.5, "tb=13/one run: 12.5 ms")
    _lib.gvqe_tune_cache_put(p, 'k "2"\\x', 11, 2, 3.25, "a\nb")
    assert _lib.gvqe_tune_cache_get(p, "k1") == (13, 1, 12.5)
    assert _lib.gvqe_tune_cache_get(p, 'k "2"\\x') == (11, 2, 3.25)
    # the file is plain JSON
    d = json.load(open(p))
    assert d["k1"]["tile_bits"] == 13 and d["k1"]["sweep"] == "tb=13/one run: 12.5 ms"
    assert d['k "2"\\x']["sweep"] == "a\nb"
    _lib.gvqe_tune_cache_put(p, "k1", 12, 0, 9.0, "")
    assert _lib.gvqe_tune_cache_get(p, "k1") == (12, 0, 9.0)
    assert _lib.gvqe_tune_cache_get(p, "stale-key") is None
    assert not any(f.startswith("tune.json.tmp") for f in os.listdir(tmp_path))


@pytest.mark.parametrize("text", ["", "{", "not json", '{"k1": {"tile_bits": 13}}', '{"k1": [1, 2]}',
                                  '{"k1": {"tile_bits": 13, "split": 1}} trailing', "\x00\x01\x02",
                                  '{"k1": {"tile_bits": 13, "split": 1, "sweep": "\\u0041"}}'])
def test_corrupt_file_reads_as_empty_and_is_rewritten(tmp_path, text):
    p = str(tmp_path / "tune.json")
    with open(p, "w") as f:
        f.write(text)
    assert _lib.gvqe_tune_cache_get(p, "k1") is None
    _lib.gvqe_tune_cache_put(p, "k2", 10, 1, 1.0, "x")
    assert _lib.gvqe_tune_cache_get(p, "k2") == (10, 1, 1.0)
    assert list(json.load(open(p))) == ["k2"]


def test_split_depths_round_trip(tmp_path):
    p = str(tmp_path / "tune.json")
    for y in (1, 4, 8):  # GVQE_OPT_SPLIT_PASSES = 2 + y: a split pass with y top qubits
        _lib.gvqe_tune_cache_put(p, f"k{y}", 13, 2 + y, 1.0, "")
        assert _lib.gvqe_tune_cache_get(p, f"k{y}") == (13, 2 + y, 1.0)


def test_put_rejects_bad_entries(tmp_path):
    p = str(tmp_path / "tune.json")
    for tb, sp in ((9, 0), (14, 0), (12, 33), (12, -1)):
        with pytest.raises(_lib.GvqeError) as e:
            _lib.gvqe_tune_cache_put(p, "k", tb, sp, 1.0, "")
        assert e.value.code == _lib.GVQE_EINVAL
    assert not os.path.exists(p)


def test_unwritable_cache_path_is_an_error(tmp_path):
    p = str(tmp_path / "no-such-dir" / "tune.json")
    with pytest.raises(_lib.GvqeError) as e:
        _lib.gvqe_tune_cache_put(p, "k", 12, 0, 1.0, "")
    assert e.value.code == _lib.GVQE_EINVAL
