"""The allocation-free two-pass Laplacian (atlas_nabla_laplacian_edges_noalloc).

It serves callers that cannot allocate device memory when they apply the
operator (code inside another framework's pre-sized memory pool, a phase
that must not allocate, a C or Fortran model that holds only field
pointers): it runs the same edge-flux and node-gather kernels as
atlas_nabla_laplacian_edges on a 64 MiB static scratch owned by the
library instead of a caller workspace.  This file is collected last so that
a run stopping at the first failure has run every other test already.
"""

import numpy as np
import pytest

import synthetic

pytestmark = pytest.mark.gpu

SCRATCH_BYTES = 64 << 20


@pytest.fixture(scope="module")
def torch():
    t = pytest.importorskip("torch")
    if not t.cuda.is_available():
        pytest.skip("no CUDA device")
    return t


def _field(torch, fvm, nlev, ld, dtype):
    g = fvm.grid.arrays()
    f = synthetic.level_scalar(g["lon"], g["lat_node"], nlev)
    return torch.from_numpy(synthetic.padded(f, ld)).to(device="cuda", dtype=dtype)


@pytest.mark.parametrize("dt,ld,tol", [("f32", 144, 1e-5), ("f64", 140, 1e-13)])
def test_noalloc_matches_workspace_form_twice(torch, product, omesh, dt, ld, tol):
    """Against the workspace form and against the FP64 oracle's Laplacian on
    the same inputs, twice in a row; ld leaves room past the last vector,
    which the call must not touch."""
    atlas, capi = product
    fvm = atlas.build_fvm(32)
    code = atlas.ATLAS_F32 if dt == "f32" else atlas.ATLAS_F64
    tdt = torch.float32 if dt == "f32" else torch.float64
    fvm.prepare(("gradient", "divergence"), dtypes=(code,))
    nlev = 137
    ws_need = capi.atlas_nabla_workspace_bytes(fvm.handle, capi.ATLAS_OP_LAPLACIAN, nlev, ld, code)
    assert 0 < ws_need <= SCRATCH_BYTES
    f = _field(torch, fvm, nlev, ld, tdt)
    ref = fvm.laplacian_edges(f, nlev)  # existing entry point, caller workspace
    torch.cuda.synchronize()
    want = ref[:, :nlev].double().cpu().numpy()
    oracle = omesh(32).laplacian(f[:, :nlev].double().cpu().numpy())
    for _ in range(2):  # two calls in a row share the scratch
        out = torch.full_like(f, 3.0)
        capi.atlas_nabla_laplacian_edges_noalloc(fvm.handle, f.data_ptr(), out.data_ptr(), nlev, ld, code,
                                                 torch.cuda.current_stream().cuda_stream)
        torch.cuda.synchronize()
        got = out[:, :nlev].double().cpu().numpy()
        assert np.max(np.abs(got - want)) <= tol * np.max(np.abs(want))
        assert np.max(np.abs(got - oracle)) <= tol * np.max(np.abs(oracle))
        vec = 4 if dt == "f32" else 2  # padding zeroed to the end of the last vector only
        end = (nlev + vec - 1) // vec * vec
        assert end < ld
        assert torch.all(out[:, nlev:end] == 0.0).item() and torch.all(out[:, end:] == 3.0).item()


def test_noalloc_rejects_oversize_and_unprepared(torch, product):
    atlas, capi = product
    big = atlas.build_fvm(80)
    big.prepare(("gradient", "divergence"), dtypes=(atlas.ATLAS_F32,))
    nlev, ld = 137, 140
    assert capi.atlas_nabla_workspace_bytes(big.handle, capi.ATLAS_OP_LAPLACIAN, nlev, ld, atlas.ATLAS_F32) \
        > SCRATCH_BYTES
    f = torch.zeros((big.nnodes, ld), device="cuda")
    out = torch.zeros_like(f)
    with pytest.raises(capi.AtlasError) as ei:
        capi.atlas_nabla_laplacian_edges_noalloc(big.handle, f.data_ptr(), out.data_ptr(), nlev, ld,
                                                 atlas.ATLAS_F32, None)
    assert ei.value.code == -1
    fresh = atlas.build_fvm(16)  # tables not on the device: refused, nothing allocated
    f = torch.zeros((fresh.nnodes, 8), device="cuda")
    out = torch.zeros_like(f)
    with pytest.raises(capi.AtlasError) as ei:
        capi.atlas_nabla_laplacian_edges_noalloc(fresh.handle, f.data_ptr(), out.data_ptr(), 5, 8,
                                                 atlas.ATLAS_F32, None)
    assert ei.value.code == -6
