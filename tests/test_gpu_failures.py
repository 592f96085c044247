"""GPU: failed device allocations (forced with the library's testing hook,
no real memory pressure) make the calls that need them return ATLAS_ENOMEM
and leave no partial tables: once allocations succeed again the same calls
give the oracle's results."""
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


@pytest.fixture
def hook(product):
    capi = product[1]
    yield capi.atlas_debug_fail_allocations
    capi.atlas_debug_fail_allocations(-1)


@pytest.mark.parametrize("after", [0, 1, 2])
def test_operator_tables(torch, product, omesh, hook, after):
    atlas, capi = product
    fvm = atlas.build_fvm(16)  # fresh: no tables yet
    g = omesh(16).grid()
    f = synthetic.level_scalar(g["lon"], g["lat_node"], 3)
    t = torch.from_numpy(synthetic.padded(f, 4)).cuda()
    hook(after)  # the table upload needs three allocations (offsets, entries, weights)
    with pytest.raises(capi.AtlasError) as ei:
        fvm.gradient(t, 3)
    assert ei.value.code == -2
    hook(-1)
    gx, gy = fvm.gradient(t, 3)
    torch.cuda.synchronize()
    ox, oy = omesh(16).gradient(f)
    assert np.max(np.abs(gx[:, :3].cpu().numpy() - ox)) <= 1e-13 * np.max(np.abs(ox))
    assert np.max(np.abs(gy[:, :3].cpu().numpy() - oy)) <= 1e-13 * np.max(np.abs(oy))


def test_remap_and_integral(torch, product, omesh, hook):
    atlas, capi = product
    fvm = atlas.build_fvm(16)
    x = torch.ones((fvm.nnodes, 2), dtype=torch.float64, device="cuda")
    hook(0)
    with pytest.raises(capi.AtlasError) as ei:
        fvm.integral(x)
    assert ei.value.code == -2
    r = atlas.Remap(atlas.Mesh(atlas.Grid(16)), atlas.Grid(8, regular=True))
    with pytest.raises(capi.AtlasError) as ei:
        r.apply(x)
    assert ei.value.code == -2
    hook(-1)
    area = fvm.integral(x).cpu().numpy()
    assert np.allclose(area, 4 * np.pi * 6371220.0 ** 2, rtol=1e-12)
    out = r.apply(x)
    torch.cuda.synchronize()
    assert torch.allclose(out[:, :2], torch.ones_like(out[:, :2]), rtol=0, atol=1e-14)
    r.close()
