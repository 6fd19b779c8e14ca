"""Host logic of the pyramid tile cache (no GPU): the key names everything
the best tiling depends on, the file round-trips, and an unreadable or
corrupt cache reads as empty instead of failing the run."""
import json

from paper_2602_06688_gb300 import PupilDesc, PwfsDesc, autotune


def test_key_names_the_geometry_and_batch():
    pu = PupilDesc(480, 39.0 / 480, 0.28)
    k = autotune._key("GB300", pu, PwfsDesc(2, 48, 96, 480, 4.0), 1)
    assert k.startswith(autotune._VERSION + "|GB300|")
    assert all(f in k for f in ("np480", "pad2", "mod48", "sub96", "b1"))
    others = [autotune._key("GB300", pu, PwfsDesc(2, 48, 96, 480, 4.0), 8),
              autotune._key("GB300", pu, PwfsDesc(2, 24, 96, 480, 4.0), 1),
              autotune._key("GB300", pu, PwfsDesc(2, 48, 48, 480, 4.0), 1),
              autotune._key("GB300", PupilDesc(400, 0.1, 0.28), PwfsDesc(4, 48, 96, 480, 4.0), 1),
              autotune._key("other", pu, PwfsDesc(2, 48, 96, 480, 4.0), 1)]
    assert len(set(others + [k])) == 6


def test_store_and_load_round_trip(tmp_path, monkeypatch):
    path = tmp_path / "sub" / "tiles.json"
    monkeypatch.setenv("SPECULA_TUNE_CACHE", str(path))
    assert autotune.cache_path() == str(path)
    assert autotune._load() == {}                      # no file yet
    d = {"v5|GB300|np480|pad2|mod48|sub96|b1": [48, 1, 2]}
    autotune._store(d)                                 # creates the directory
    assert json.loads(path.read_text()) == d
    assert autotune._load() == d


def test_corrupt_cache_reads_as_empty(tmp_path, monkeypatch):
    path = tmp_path / "tiles.json"
    path.write_text("{not json")
    monkeypatch.setenv("SPECULA_TUNE_CACHE", str(path))
    assert autotune._load() == {}
