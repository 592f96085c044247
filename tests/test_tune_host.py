"""Host logic of the autotuner: cache keys that tell grid families apart,
and the JSON cache's round trip and its tolerance of a damaged file.  No GPU
is used (timing and launches are the GPU tests' part)."""
import json

import pytest


def test_grid_keys_tell_families_apart(product):
    atlas, _ = product
    from paper_1908_07038_gb300 import tune
    from synthetic.regional import DOMAINS
    proj, kw = DOMAINS["lambert"]
    grids = [atlas.Grid(16), atlas.Grid(16, regular=True), atlas.Grid(24),
             atlas.Grid.regional(proj, 17, 11, **kw), atlas.Grid.regional(proj, 11, 17, **kw),
             atlas.Grid.regional(DOMAINS["mercator"][0], 17, 11, **DOMAINS["mercator"][1])]
    keys = [tune._grid_key(g) for g in grids]
    assert keys[:3] == ["O16", "F16", "O24"]
    assert keys[3] == "lambert_conformal17x11"
    assert len(set(keys)) == len(keys)


def test_cache_round_trip_and_damaged_file(tmp_path, monkeypatch, product):
    from paper_1908_07038_gb300 import tune
    path = tmp_path / "tune.json"
    monkeypatch.delenv("ATLASGB_TUNE_CACHE", raising=False)
    assert tune._load_cache() == {}
    tune._store_cache({"x": 1})  # no file named: nothing is written
    assert not path.exists()
    monkeypatch.setenv("ATLASGB_TUNE_CACHE", str(path))
    assert tune._load_cache() == {}
    entry = {"GB300|O16|dt0|L5|ld8|gradient": dict(vec=4, batch=6, threads=256, bps=0, tile=1, ms=0.01)}
    tune._store_cache(entry)
    assert json.loads(path.read_text()) == entry
    assert tune._load_cache() == entry
    assert not list(tmp_path.glob("*.tmp"))  # written through a temporary file, then renamed
    path.write_text("{not json")
    assert tune._load_cache() == {}


@pytest.mark.parametrize("dtype", [0, 1, 2])
def test_candidates_respect_the_kernels_limits(product, dtype):
    """Every candidate shape is one atlas_fvm_set_launch accepts: vector
    widths of at most 16 bytes, batches of 3 or 6, whole warps."""
    from paper_1908_07038_gb300 import tune
    c = tune.CANDIDATES[dtype]
    es = {0: 4, 1: 8, 2: 2}[dtype]
    assert all(v * es <= 16 and 16 % (v * es) == 0 for v in c["vec"])
    assert set(c["batch"]) <= {3, 6}
    assert all(t % 32 == 0 and 32 <= t <= 1024 for t in c["threads"])
    assert all(t >= 1 for t in c["tile"])
    # and the library's own validation takes every combination, for every operator
    import itertools
    atlas, _ = product
    fvm = atlas.build_fvm(8)
    for op in atlas.OPS:
        for vec, batch, threads, bps, tile in itertools.product(c["vec"], c["batch"], c["threads"], c["bps"],
                                                                c["tile"]):
            fvm.set_launch(op, vec, batch, threads, bps, tile, dtype=dtype)
