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


def test_tune_fvm_picks_and_installs_the_fastest_candidate(product, monkeypatch, tmp_path):
    """The tuner's bookkeeping on the host, with the timing faked: every
    candidate (per-node shapes, then node-group shapes) is timed once, the
    fastest is installed (set_group / set_launch), reported with the
    node-group kernel's actual launch shape, and cached; a second run takes
    it from the cache without timing anything."""
    import torch
    atlas, _ = product
    from paper_1908_07038_gb300 import tune
    real = atlas.build_fvm(8)

    class Fvm:
        grid, nnodes = real.grid, real.nnodes

        def __init__(self):
            self.calls = []

        def set_launch(self, *a, **k):
            self.calls.append(("launch", a, k))
            real.set_launch(*a, **k)

        def set_group(self, *a, **k):
            self.calls.append(("group", a, k))
            real.set_group(*a, **k)

        def tile_info(self, op, nlev, ld, dtype=0):
            return dict(blocks_per_sm=1, stages=3, smem=1 << 17, max_rows=100)

    fvm = Fvm()
    timings = iter([5.0 - 0.01 * k for k in range(1000)])  # every later candidate is faster
    monkeypatch.setattr(tune, "time_call", lambda fn, reps=5, warmup=3: next(timings))
    monkeypatch.setattr(tune, "_call", lambda *a, **k: None)
    monkeypatch.setattr(torch.cuda, "get_device_name", lambda *a: "fake-gpu")
    monkeypatch.setenv("ATLASGB_TUNE_CACHE", str(tmp_path / "tune.json"))
    fields = tuple(torch.zeros((real.nnodes, 140)) for _ in range(3))
    best = tune.tune_fvm(fvm, atlas.ATLAS_F32, 137, 140, ("gradient",), fields=fields, reps=1)
    b = best["gradient"]
    last = tune.TILE_CANDIDATES[-1]  # timed last, hence fastest
    assert b["kernel"] == "tile" and (b["groups"], b["tile_bps"], b["npw"], b["rows"]) == last
    assert (b["tile_blocks"], b["tile_stages"]) == (1, 3)
    n_node = 1
    for v in tune.CANDIDATES[atlas.ATLAS_F32].values():
        n_node *= len(v)
    assert len(b["sweep"]) == n_node + len(tune.tile_candidates("gradient"))
    assert len(tune.tile_candidates("gradient")) < len(tune.tile_candidates("laplacian"))
    assert fvm.calls[-1][0] == "group" and fvm.calls[-1][2].get("nodes_per_warp") == last[2]
    assert fvm.calls[-1][2].get("rows_per_tile") == last[3]
    # cached: the second run times nothing
    monkeypatch.setattr(tune, "time_call", lambda *a, **k: pytest.fail("timed a cached shape"))
    again = tune.tune_fvm(fvm, atlas.ATLAS_F32, 137, 140, ("gradient",), fields=fields, reps=1)
    assert again["gradient"]["npw"] == last[2] and again["gradient"]["kernel"] == "tile"
