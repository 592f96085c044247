"""GPU remapping (atlas_remap_apply) against the oracle's remap (brute-force
location, Dot2 interpolation) on the same seeded source fields.

Tolerances: relative max-norm 1e-13 (FP64), 1e-5 (FP32), 2e-2 (BF16 storage).
The paper's example O32 -> F8 in full, ragged level counts and leading
dimensions, and O320 -> F160 and O1280 -> F640 x 137 levels on sampled
targets (the oracle searches every source triangle for each)."""
import numpy as np
import pytest

import synthetic

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    t = pytest.importorskip("torch")
    if not t.cuda.is_available():
        pytest.skip("no CUDA device")
    return t


def _relmax(a, b):
    den = np.max(np.abs(b))
    return np.max(np.abs(np.asarray(a, np.float64) - b)) / (den if den > 0 else 1.0)


def _setup(product, N, M):
    atlas = product[0]
    g = atlas.Grid(N)
    r = atlas.Remap(atlas.Mesh(g), atlas.Grid(M, regular=True))
    a = r.grid.arrays()
    return r, g.arrays(), np.stack([a["lon"], a["lat_node"]], 1)


@pytest.mark.parametrize("dt,nlev,ld_src,ld_dst", [(np.float64, 1, 1, 1), (np.float64, 5, 6, 8), (np.float32, 137, 140, 140),
                                                  (np.float32, 9, 9, 12), (np.float64, 137, 138, 138)])
def test_o32_to_f8(torch, product, omesh, dt, nlev, ld_src, ld_dst):
    r, g, tgt = _setup(product, 32, 8)
    f = synthetic.level_scalar(g["lon"], g["lat_node"], nlev, dt)
    src = torch.from_numpy(synthetic.padded(f, ld_src)).cuda()
    out = torch.full((r.ntgt, ld_dst), 7.0, dtype=src.dtype, device="cuda")
    r.apply(src, nlev, out=out)
    torch.cuda.synchronize()
    want = omesh(32).remap(tgt, f, nlev)
    tol = 1e-13 if dt == np.float64 else 1e-5
    assert _relmax(out[:, :nlev].double().cpu().numpy(), want) <= tol
    # levels past the last written vector keep their values
    vec = 16 // np.dtype(dt).itemsize
    end = -(-nlev // vec) * vec if ld_dst % vec == 0 and ld_src % vec == 0 else nlev
    if end < ld_dst:
        assert torch.all(out[:, end:] == 7.0)


def test_bf16_storage(torch, product, omesh):
    r, g, tgt = _setup(product, 32, 8)
    f = synthetic.level_scalar(g["lon"], g["lat_node"], 16, np.float32)
    src = torch.from_numpy(f).cuda().to(torch.bfloat16)
    out = r.apply(src)
    torch.cuda.synchronize()
    want = omesh(32).remap(tgt, src.float().cpu().numpy())
    assert _relmax(out.float().cpu().numpy(), want) <= 2e-2


@pytest.mark.parametrize("N,M,count,dt,ld", [(320, 160, 200, np.float32, 140), (320, 160, 200, np.float64, 138),
                                             (1280, 640, 30, np.float32, 140)])
def test_sampled_137_levels(torch, product, omesh, N, M, count, dt, ld):
    r, g, tgt = _setup(product, N, M)
    f = synthetic.level_scalar(g["lon"], g["lat_node"], 137, dt)
    src = torch.from_numpy(synthetic.padded(f, ld)).cuda()
    out = r.apply(src, 137)
    torch.cuda.synchronize()
    # targets of the first and last rows (every 64th) and random ones: the
    # oracle tests every source triangle per target (O1280: 13 M triangles)
    rng = np.random.default_rng(6)
    pl = 4 * M
    pick = np.unique(np.concatenate([np.arange(0, pl, 64), np.arange(r.ntgt - pl, r.ntgt, 64),
                                     rng.integers(0, r.ntgt, size=count)]))
    want = omesh(N).remap(tgt[pick], f, 137)
    got = out.index_select(0, torch.from_numpy(pick).cuda())[:, :137].double().cpu().numpy()
    del src, out
    torch.cuda.empty_cache()
    assert _relmax(got, want) <= (1e-13 if dt == np.float64 else 1e-5)
