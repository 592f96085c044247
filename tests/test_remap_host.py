"""Remapping, host side (no GPU): the F<N> grid and the located triangles and
weights of atlas_remap_create against the oracle's brute-force search."""
import numpy as np
import pytest


@pytest.fixture(scope="module")
def atlas(product):
    return product[0]


def _wmap(nodes, w):
    return [dict(zip(a, b)) for a, b in zip(nodes.tolist(), w.tolist())]


def test_regular_gaussian_grid(atlas):
    for N in (1, 8, 40):
        F = atlas.Grid(N, regular=True)
        a = F.arrays()
        assert F.nnodes == 8 * N * N and F.nlat == 2 * N
        assert np.all(a["pl"] == 4 * N)
        x, _ = np.polynomial.legendre.leggauss(2 * N)
        assert np.max(np.abs(a["lat"] - np.arcsin(x)[::-1])) <= 1e-14
        assert np.array_equal(a["lat"], atlas.Grid(N).arrays()["lat"])  # same latitudes as O<N>
        j = np.tile(np.arange(4 * N), 2 * N)
        assert np.max(np.abs(a["lon"] - 2 * np.pi * j / (4 * N))) <= 1e-15


def test_f_grid_meshes(atlas):
    """F<N> grids are meshed like O<N> (counts: T = 2V - 8N, E = 3V - 4N)."""
    m = atlas.Mesh(atlas.Grid(8, regular=True))
    assert (m.ntri, m.nedges) == (2 * 512 - 64, 3 * 512 - 32)


@pytest.mark.parametrize("N,M", [(16, 8), (32, 8), (64, 16), (48, 24)])
def test_weights_equal_the_oracle_search(atlas, omesh, N, M):
    g = atlas.Grid(N)
    m = atlas.Mesh(g)
    F = atlas.Grid(M, regular=True)
    r = atlas.Remap(m, F)
    nodes, w = r.tables()
    a = F.arrays()
    on, ow = omesh(N).remap_weights(np.stack([a["lon"], a["lat_node"]], 1))
    A, B = _wmap(nodes, w), _wmap(on, ow)
    for t in range(len(A)):
        keys = set(A[t]) | set(B[t])
        # the same triangle, or on a shared edge the one with the same
        # non-zero weights (the third weight is then 0 up to rounding)
        assert max(abs(A[t].get(k, 0.0) - B[t].get(k, 0.0)) for k in keys) <= 1e-14, t
    r.close()


def test_polar_cap_targets_are_refused(atlas, product):
    m = atlas.Mesh(atlas.Grid(8))
    with pytest.raises(product[1].AtlasError) as ei:
        atlas.Remap(m, atlas.Grid(32, regular=True))  # F32's first row is nearer the pole than O8's
    assert "polar" in str(ei.value)


def test_remap_keeps_its_mesh(atlas):
    g = atlas.Grid(8)
    m = atlas.Mesh(g)
    r = atlas.Remap(m, atlas.Grid(4, regular=True))
    m.close()  # refused while the remap holds it
    nodes, w = r.tables()
    assert nodes.shape == (128, 3) and np.allclose(w.sum(1), 1)
    r.close()
