"""Pins of the oracle's median-dual geometry (volumes, normals, closure) and of
the exactness of its operators on fields that are linear in (lon, lat).

Reading (the paper names the operators only, Sec. 2.3): each node owns the
median-dual cell built from triangle centroids and side midpoints in the
(lon, lat) plane, first and last rows extended to the poles; its volume is
the exact integral of R^2 cos(lat) dlon dlat over the cell.
"""
import numpy as np
import pytest

R = 6371220.0

_GL_X, _GL_W = np.polynomial.legendre.leggauss(12)
_GL_X = 0.5 * (_GL_X + 1.0)
_GL_W = 0.5 * _GL_W


def _int_cos_triangle(A, B, C):
    """Integral of cos(lat) over the triangle ABC of the (lon, lat) plane
    (Duffy-collapsed 12x12 Gauss-Legendre; arrays of triangles)."""
    A, B, C = (np.asarray(p, dtype=np.float64) for p in (A, B, C))
    det = np.abs((B[..., 0] - A[..., 0]) * (C[..., 1] - B[..., 1]) - (B[..., 1] - A[..., 1]) * (C[..., 0] - B[..., 0]))
    tot = np.zeros(A.shape[:-1])
    for u, wu in zip(_GL_X, _GL_W):
        for v, wv in zip(_GL_X, _GL_W):
            y = A[..., 1] + u * (B[..., 1] - A[..., 1]) + u * v * (C[..., 1] - B[..., 1])
            tot += wu * wv * u * np.cos(y)
    return tot * det


def _plain_area_triangle(A, B, C):
    return 0.5 * np.abs((B[..., 0] - A[..., 0]) * (C[..., 1] - A[..., 1]) - (C[..., 0] - A[..., 0]) * (B[..., 1] - A[..., 1]))


def _dual_by_quadrature(m):
    """Cell volumes and plain (lon, lat) areas from the triangles: each triangle
    gives each vertex the quadrilateral (vertex, side midpoint, centroid, side
    midpoint); polar cells add the rectangle up to the pole."""
    d = m.mesh()
    g = m.grid()
    pl, lat = g["pl"], g["lat"]
    tr, tj, tv = d["tri_r"], d["tri_j"], d["tri"]
    P = np.stack([2 * np.pi * tj / pl[tr], lat[tr]], axis=-1)  # [T,3,2]
    c = P.mean(axis=1)
    vol = np.zeros(m.nnodes)
    area = np.zeros(m.nnodes)
    for k in range(3):
        p = P[:, k]
        m1 = 0.5 * (p + P[:, (k + 1) % 3])
        m2 = 0.5 * (p + P[:, (k + 2) % 3])
        q = _int_cos_triangle(p, m1, c) + _int_cos_triangle(p, c, m2)
        a = _plain_area_triangle(p, m1, c) + _plain_area_triangle(p, c, m2)
        np.add.at(vol, tv[:, k], q)
        np.add.at(area, tv[:, k], a)
    off = np.concatenate([[0], np.cumsum(pl)])
    for r, top in ((0, np.pi / 2), (m.nlat - 1, -np.pi / 2)):
        dl = 2 * np.pi / pl[r]
        sl = slice(off[r], off[r + 1])
        vol[sl] += dl * abs(np.sin(top) - np.sin(lat[r]))
        area[sl] += dl * abs(top - lat[r])
    return R * R * vol, area


@pytest.mark.parametrize("N", [1, 2, 4, 8])
def test_volumes_match_quadrature(omesh, N):
    m = omesh(N)
    V = m.dual()["V"]
    Vq, _ = _dual_by_quadrature(m)
    assert np.max(np.abs(V - Vq) / Vq) <= 1e-13


@pytest.mark.parametrize("N", [2, 16, 64])
def test_sum_of_volumes(omesh, N):
    m = omesh(N)
    V = m.dual()["V"]
    assert np.all(V > 0)
    s = np.sum(np.sort(V))
    assert abs(s / (4 * np.pi * R * R) - 1.0) <= 1e-12


@pytest.mark.parametrize("N", [2, 16, 64])
def test_closure_every_cell(omesh, N):
    m = omesh(N)
    res, absum = m.closure()
    assert np.max(np.abs(res).max(axis=1) / absum) <= 1e-15


@pytest.mark.parametrize("N", [2, 16])
def test_normals_point_from_a_to_b(omesh, N):
    m = omesh(N)
    d = m.mesh()
    g = m.grid()
    S = m.dual()["S"]
    lon, lat = g["lon"], g["lat_node"]
    reg = ~d["is_pole"].astype(bool)
    a, b = d["e2n"][reg, 0], d["e2n"][reg, 1]
    dl = np.angle(np.exp(1j * (lon[b] - lon[a])))  # unwrapped longitude difference
    dp = lat[b] - lat[a]
    assert np.all(S[reg, 0] * dl + S[reg, 1] * dp > 0)
    pole = d["is_pole"].astype(bool)
    north = d["e2n"][pole, 0] < m.nnodes // 2
    C = 2 * np.pi * R / 20
    assert np.allclose(S[pole, 1], np.where(north, C, -C), rtol=1e-15, atol=0)
    assert np.all(S[pole, 0] == 0)


def test_volume_symmetries(omesh):
    """Quarter-turn invariance; N/S mirror symmetry away from the equator band."""
    N = 8
    m = omesh(N)
    V = m.dual()["V"]
    pl = m.grid()["pl"]
    off = np.concatenate([[0], np.cumsum(pl)])
    for r in range(2 * N):
        row = V[off[r]:off[r + 1]]
        q = pl[r] // 4
        assert np.allclose(row, np.roll(row, q), rtol=4e-16, atol=0)
    for r in range(N - 1):
        a = V[off[r]:off[r + 1]]
        b = V[off[2 * N - 1 - r]:off[2 * N - r]]
        assert np.allclose(a, b, rtol=4e-16, atol=0)


def _seam_free(m, lon):
    """Nodes whose every edge neighbour lies within half a turn in longitude
    (so that lon is a single-valued linear function on the cell)."""
    d = m.mesh()
    ptr, n2e, e2n = d["n2e_ptr"], d["n2e"], d["e2n"]
    ok = np.ones(m.nnodes, bool)
    for i in range(m.nnodes):
        for e in n2e[ptr[i]:ptr[i + 1]]:
            j = e2n[e, 0] + e2n[e, 1] - i
            if abs(lon[j] - lon[i]) >= np.pi - 1e-9:
                ok[i] = False
    return ok


@pytest.mark.parametrize("N", [2, 8, 16])
def test_gradient_exact_for_linear_fields(omesh, N):
    """The median-dual Green-Gauss sum is exact for fields linear in (lon, lat):
    sum_e n_ie (f_j - f_i)/2 = R A_i grad_(lon,lat) f with A_i the plain cell
    area.  Hence f = lat gives g_lon = 0 and g_lat V_i/(R cos_i) = A_i on every
    non-polar cell; f = lon gives g_lon V_i/R = A_i and g_lat = 0 on cells away
    from the longitude seam."""
    m = omesh(N)
    g = m.grid()
    du = m.dual()
    V, cos = du["V"], du["coslat"]
    _, A = _dual_by_quadrature(m)
    lon, lat = g["lon"], g["lat_node"]
    pl = g["pl"]
    nonpolar = np.ones(m.nnodes, bool)
    nonpolar[:pl[0]] = False
    nonpolar[m.nnodes - pl[-1]:] = False

    gx, gy = m.gradient(lat)
    scale = 1.0 / (R * np.min(A / (V / R**2)))
    assert np.max(np.abs(gx)) <= 1e-13 * scale
    got = gy[:, 0] * V / (R * cos)
    assert np.max(np.abs(got[nonpolar] - A[nonpolar]) / A[nonpolar]) <= 1e-12

    ok = _seam_free(m, lon)
    gx, gy = m.gradient(lon)
    got = gx[:, 0] * V / R
    assert np.max(np.abs(got[ok] - A[ok]) / A[ok]) <= 1e-12
    assert np.max(np.abs(gy[ok, 0])) <= 1e-13 * scale


@pytest.mark.parametrize("N", [2, 8, 16])
def test_divergence_exact_for_linear_fluxes(omesh, N):
    """F = (u, v cos lat) linear in (lon, lat): u = lon gives V div / R = A on
    seam-free cells; v cos = pi/2 - lat gives V div / R = -A on every cell but
    the southern polar row (whose pole segment would carry flux pi)."""
    m = omesh(N)
    g = m.grid()
    du = m.dual()
    V, cos = du["V"], du["coslat"]
    _, A = _dual_by_quadrature(m)
    lon, lat = g["lon"], g["lat_node"]
    pl = g["pl"]
    ok = _seam_free(m, lon)
    d = m.divergence(lon, np.zeros_like(lon))[:, 0]
    got = d * V / R
    assert np.max(np.abs(got[ok] - A[ok]) / A[ok]) <= 1e-12
    v = (np.pi / 2 - lat) / cos
    d = m.divergence(np.zeros_like(lon), v)[:, 0]
    got = d * V / R
    keep = np.ones(m.nnodes, bool)
    keep[m.nnodes - pl[-1]:] = False
    assert np.max(np.abs(got[keep] + A[keep]) / A[keep]) <= 1e-12


@pytest.mark.parametrize("N", [4, 16])
def test_averaged_form_agrees_within_closure_residual(omesh, N):
    """The textbook averaged form sum n (f_a+f_b)/2 / V differs from the
    closure-exact form only by f_i (sum_e n_ie) / V_i."""
    m = omesh(N)
    g = m.grid()
    rng = np.random.default_rng(5)
    f = np.cos(g["lat_node"]) * np.cos(g["lon"]) + rng.standard_normal(m.nnodes)
    ga_x, ga_y = m.gradient_averaged(f)
    gd_x, gd_y = m.gradient(f)
    du = m.dual()
    V, cos = du["V"], du["coslat"]
    res, absum = m.closure()
    bound = np.abs(f) * absum / V * 2e-15 + 1e-15 * (np.abs(gd_x[:, 0]) + np.abs(gd_y[:, 0]))
    assert np.all(np.abs(ga_x[:, 0] - gd_x[:, 0]) <= bound + np.abs(f * res[:, 0] / V))
    assert np.all(np.abs(ga_y[:, 0] - gd_y[:, 0]) <= bound + np.abs(cos * f * res[:, 1] / V))
