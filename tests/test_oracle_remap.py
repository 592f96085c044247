"""Pins of the oracle's remapping (linear element-based interpolation in 3D on
the sphere, the method of the paper's O32 -> F8 example, Sec. 4.3).

What the mathematics fixes: the three weights of a target are the
barycentric coordinates of the point where the ray along the target
direction crosses the located triangle, so (a) they sum to 1 and are >= 0,
(b) the weighted sum of the vertex vectors is that crossing point, parallel
to the target direction, (c) a target on a source node takes that node's
value, (d) the interpolation error of a smooth field falls at second order
with the source resolution.  Target grids: F<N> (2N Gaussian latitudes from
numpy's Gauss-Legendre nodes, 4N longitudes from 0), an independent source
of the points."""
import numpy as np
import pytest


def f_grid(N):
    x, _ = np.polynomial.legendre.leggauss(2 * N)
    lat = np.arcsin(x)[::-1]  # north to south
    lon = 2 * np.pi * np.arange(4 * N) / (4 * N)
    return np.array([(a, b) for b in lat for a in lon])


def unit(ll):
    return np.stack([np.cos(ll[:, 1]) * np.cos(ll[:, 0]), np.cos(ll[:, 1]) * np.sin(ll[:, 0]), np.sin(ll[:, 1])], 1)


def smooth(ll):
    lon, lat = ll[:, 0], ll[:, 1]
    return np.cos(lat) ** 2 * np.cos(2 * lon) + 0.5 * np.sin(lat) + 0.3 * np.cos(lat) * np.sin(lon)


@pytest.mark.parametrize("N,M", [(16, 8), (32, 8), (32, 16)])
def test_weights_are_barycentric_coordinates_of_the_ray_crossing(omesh, N, M):
    m = omesh(N)
    tgt = f_grid(M)
    nodes, w = m.remap_weights(tgt)
    assert np.all(w >= -1e-12)
    assert np.max(np.abs(w.sum(1) - 1)) <= 4e-16
    g = m.grid()
    src = np.stack([g["lon"], g["lat_node"]], 1)
    q = np.einsum("tk,tkc->tc", w, unit(src)[nodes])
    p = unit(tgt)
    assert np.max(np.linalg.norm(np.cross(q, p), axis=1)) <= 1e-14
    assert np.all(np.einsum("tc,tc->t", q, p) > 0.99)
    # each located triangle is a triangle of the mesh
    tri = {tuple(sorted(t)) for t in m.mesh()["tri"].tolist()}
    assert all(tuple(sorted(n)) in tri for n in nodes.tolist())


def test_targets_on_source_nodes_take_the_node_values(omesh):
    m = omesh(16)
    g = m.grid()
    src = np.stack([g["lon"], g["lat_node"]], 1)
    f = np.random.default_rng(1).standard_normal((m.nnodes, 2))
    out = m.remap(src, f)
    assert np.max(np.abs(out - f)) <= 1e-13 * np.max(np.abs(f))


def test_remap_converges_at_second_order(omesh):
    """O16, O32, O64 -> F8 (the paper's target grid): the max error of a
    smooth field falls by about 4 per refinement."""
    tgt = f_grid(8)
    errs = []
    for N in (16, 32, 64):
        m = omesh(N)
        g = m.grid()
        f = smooth(np.stack([g["lon"], g["lat_node"]], 1))[:, None]
        errs.append(np.max(np.abs(m.remap(tgt, f)[:, 0] - smooth(tgt))))
    s = [np.log2(errs[i] / errs[i + 1]) for i in range(2)]
    assert np.mean(s) >= 1.9 and min(s) >= 1.7, (errs, s)  # measured 1.80, 2.22


def test_o32_to_f8_example(omesh):
    """The paper's example: an analytic field on O32 remapped to F8 (512
    points), every point located, error below 1e-2 of the field's range."""
    m = omesh(32)
    tgt = f_grid(8)
    g = m.grid()
    f = smooth(np.stack([g["lon"], g["lat_node"]], 1))[:, None]
    out = m.remap(tgt, f)[:, 0]
    assert out.shape == (512,)
    assert np.max(np.abs(out - smooth(tgt))) <= 1e-2 * np.ptp(smooth(tgt))


def test_polar_cap_targets_are_not_located(omesh):
    m = omesh(8)
    with pytest.raises(ValueError):
        m.remap_weights(np.array([[0.3, np.radians(89.9)]]))
