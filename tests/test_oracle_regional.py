"""Pins of the regional-grid oracle (``oracle/regional_oracle.c``) against
geometry and closed forms, not against its own formulas:

* projections: the rotated lon-lat inverse against great-circle distances
  to the rotated poles and origin; Mercator and Lambert conformality (equal,
  orthogonal steps on the sphere) and scale factors against chord lengths;
  known points (the Lambert origin, the Mercator equator);
* the plane median dual: exact cell areas of the structured triangulation
  (interior dx dy, sides a half, corners a third or a sixth), closure of
  every cell, boundary included;
* exactness: fields linear in the plane have the exact gradient, divergence
  and curl (through the scale factors) at every node, boundary included;
* the discrete Gauss theorem: sum_i V_i div_i = 0 for fields vanishing on
  the boundary;
* second-order convergence in the interior for smooth fields on the sphere
  (gradient against the analytic tangent gradient, Laplacian of a degree-2
  harmonic, curl of a solid-body rotation), first order at the boundary.
"""
import numpy as np
import pytest

from oracle import oracle
from synthetic.regional import DOMAINS

R = oracle.R_EARTH
CASES = DOMAINS


def _mesh(name, nx=17, ny=11, **over):
    proj, kw = CASES[name]
    kw = dict(kw, **over)
    return oracle.RegionalMesh(proj, nx, ny, **kw)


def _unit(lon, lat):
    return np.stack([np.cos(lat) * np.cos(lon), np.cos(lat) * np.sin(lon), np.sin(lat)], 1)


def _angle(p, q):
    return np.arctan2(np.linalg.norm(np.cross(p, q), axis=-1), (p * q).sum(-1))


def test_counts_and_triangles():
    m = _mesh("lambert", 7, 5)
    g = m.geometry()
    assert (m.nnodes, m.ntri) == (35, 2 * 6 * 4)
    tri = g["tri"]
    x, y = g["x"], g["y"]
    a = (x[tri[:, 1]] - x[tri[:, 0]]) * (y[tri[:, 2]] - y[tri[:, 0]]) - \
        (x[tri[:, 2]] - x[tri[:, 0]]) * (y[tri[:, 1]] - y[tri[:, 0]])
    assert np.all(a > 0)  # counter-clockwise
    edges = {tuple(sorted((int(t[k]), int(t[(k + 1) % 3])))) for t in tri for k in range(3)}
    assert len(edges) == 3 * 35 - 2 * 7 - 2 * 5 + 1


def test_rotated_lonlat_against_great_circle_distances():
    sp = (10.0, -40.0)
    m = _mesh("rotated", 9, 7)
    g = m.geometry()
    P = _unit(g["lon"], g["lat"])
    north = _unit(np.radians([sp[0] + 180.0]), np.radians([-sp[1]]))[0]   # antipode of the south pole
    origin = _unit(np.radians([sp[0]]), np.radians([sp[1] + 90.0]))[0]    # rotated (0, 0)
    x, y = g["x"], g["y"]  # rotated lon, lat in radians
    assert np.max(np.abs(_angle(P, north[None]) - (np.pi / 2 - y))) <= 1e-13
    assert np.max(np.abs(_angle(P, origin[None]) - np.arccos(np.cos(x) * np.cos(y)))) <= 1e-12
    # the third distance fixes the side: rotated (90, 0) = north x origin
    e2 = np.cross(north, origin)
    assert np.max(np.abs(_angle(P, e2[None]) - np.arccos(np.cos(y) * np.sin(x)))) <= 1e-12
    # no rotation: the plain lon-lat grid
    plain = _mesh("rotated", 9, 7, south_pole=(0.0, -90.0)).geometry()
    assert np.max(np.abs(plain["lon"] - plain["x"])) <= 1e-15
    assert np.max(np.abs(plain["lat"] - plain["y"])) <= 1e-15
    assert np.max(np.abs(plain["hx"] - np.cos(plain["y"]))) == 0.0


@pytest.mark.parametrize("name", ["rotated", "mercator", "lambert", "lambert_south", "polar"])
def test_scale_factors_and_orthogonality_from_chords(name):
    """Tiny steps: the true distance of a plane step dx is h dx (unit
    sphere), equal in both directions for a conformal projection, and the
    x and y steps are orthogonal on the sphere."""
    proj, kw = CASES[name]
    kw = dict(kw)
    if proj == "rotated_lonlat":
        step, unit = 1e-4, np.radians(1.0)
    else:
        step, unit = 1.0, 1.0 / R
    cx, cy = 0.5 * (kw["xmin"] + kw["xmax"]), 0.5 * (kw["ymin"] + kw["ymax"])
    for ox, oy in [(0.0, 0.0), (0.3, -0.2), (-0.4, 0.35)]:
        x0 = cx + ox * (kw["xmax"] - kw["xmin"])
        y0 = cy + oy * (kw["ymax"] - kw["ymin"])
        kw.update(xmin=x0 - step, xmax=x0 + step, ymin=y0 - step, ymax=y0 + step)
        g = oracle.RegionalMesh(proj, 3, 3, **kw).geometry()
        P = _unit(g["lon"], g["lat"])
        c = 4  # centre of the 3 x 3 block; x to the right, y upwards (row 0 is the top)
        dxv, dyv = P[5] - P[3], P[1] - P[7]
        hx = np.linalg.norm(dxv) / (2 * step * unit)
        hy = np.linalg.norm(dyv) / (2 * step * unit)
        assert abs(hx - g["hx"][c]) <= 1e-6 * g["hx"][c], (name, hx, g["hx"][c])
        assert abs(hy - g["hy"][c]) <= 1e-6 * g["hy"][c], (name, hy, g["hy"][c])
        assert abs(np.dot(dxv, dyv)) <= 1e-6 * np.linalg.norm(dxv) * np.linalg.norm(dyv)
        # right-handed: x then y turns counter-clockwise seen from outside
        assert np.dot(np.cross(dxv, dyv), P[c]) > 0


def test_known_points():
    g = _mesh("mercator", 5, 5, ymin=-1.0e5, ymax=1.0e5).geometry()
    eq = np.abs(g["y"]) < 1e-300
    assert eq.sum() == 5 and np.all(np.abs(g["lat"][eq]) <= 1e-16) and np.allclose(g["hx"][eq], 1.0, rtol=0, atol=1e-15)
    assert np.max(np.abs(g["lon"] - (np.radians(20.0) + g["x"]))) <= 1e-15
    g = _mesh("lambert", 5, 5, xmin=-1e5, xmax=1e5, ymin=-1e5, ymax=1e5).geometry()
    c = 12  # the plane origin is (lon0, lat0), where the cone touches: scale 1
    assert abs(g["lon"][c] - np.radians(5.0)) <= 1e-15 and abs(g["lat"][c] - np.radians(50.0)) <= 1e-15
    assert abs(g["hx"][c] - 1.0) <= 1e-15
    for pole in (90.0, -90.0):
        g = _mesh("polar", 5, 5, xmin=-1e5, xmax=1e5, ymin=-1e5, ymax=1e5, lat0=pole).geometry()
        c = 12  # the plane origin is the pole, where the plane touches: scale 1
        assert abs(g["lat"][c] - np.radians(pole)) <= 1e-15 and abs(g["hx"][c] - 1.0) <= 1e-15
        # the central meridian leaves the north pole along -y (the south pole along +y)
        below = 22 if pole > 0 else 2
        assert abs(g["lon"][below] - np.radians(-45.0)) <= 1e-15
        # a point of the plane at distance rho lies at colatitude 2 atan(rho / 2R)
        rho = np.hypot(g["x"], g["y"])
        assert np.max(np.abs((np.pi / 2 - np.abs(g["lat"])) - 2 * np.arctan(rho / 2))) <= 1e-15


@pytest.mark.parametrize("name", ["rotated", "lambert"])
def test_cell_areas_and_closure(name):
    nx, ny = 9, 6
    m = _mesh(name, nx, ny)
    g = m.geometry()
    dx = (g["x"][1] - g["x"][0]) * R
    dy = (g["y"][0] - g["y"][nx]) * R
    r, j = np.divmod(np.arange(nx * ny), nx)
    expect = np.full(nx * ny, dx * dy)
    side = (r == 0) | (r == ny - 1) | (j == 0) | (j == nx - 1)
    expect[side] = 0.5 * dx * dy
    # corners: top-left and bottom-right touch two triangles, the others one
    expect[0] = expect[nx * ny - 1] = dx * dy / 3.0
    expect[nx - 1] = expect[(ny - 1) * nx] = dx * dy / 6.0
    assert np.max(np.abs(g["area"] - expect) / expect) <= 1e-12
    assert abs(g["area"].sum() - (nx - 1) * (ny - 1) * dx * dy) <= 1e-12 * g["area"].sum()
    res, ab = m.closure()
    assert np.max(np.abs(res).max(1) / ab) <= 1e-15


@pytest.mark.parametrize("name", list(CASES))
def test_linear_fields_are_exact_everywhere(name):
    m = _mesh(name)
    g = m.geometry()
    x, y, hx, hy = g["x"], g["y"], g["hx"], g["hy"]
    a, b, c, d = 0.7, -1.3, 0.45, 2.1
    # (the constant 3 costs rounding of order eps |f| sum|n| / V in the
    # averaged form, about 1e-13 of the gradient here)
    gx, gy = m.gradient((a * x + b * y + 3.0)[:, None])
    ex, ey = a / (R * hx), b / (R * hy)
    assert np.max(np.abs(gx[:, 0] - ex)) <= 1e-12 * np.max(np.abs(ex))
    assert np.max(np.abs(gy[:, 0] - ey)) <= 1e-12 * np.max(np.abs(ey))
    # divergence: h_y u and h_x v linear in the plane
    u = (a * x + b * y) / hy
    v = (c * x + d * y) / hx
    div = m.divergence(u[:, None], v[:, None])[:, 0]
    edv = (a + d) / (R * hx * hy)
    assert np.max(np.abs(div - edv)) <= 1e-12 * np.max(np.abs(edv))
    # curl: h_y v and h_x u linear in the plane
    u = (a * x + b * y) / hx
    v = (c * x + d * y) / hy
    cur = m.curl(u[:, None], v[:, None])[:, 0]
    ecu = (c - b) / (R * hx * hy)
    assert np.max(np.abs(cur - ecu)) <= 1e-12 * np.max(np.abs(ecu))


def test_discrete_gauss_theorem():
    nx, ny = 15, 12
    m = _mesh("lambert", nx, ny)
    g = m.geometry()
    rng = np.random.default_rng(4)
    r, j = np.divmod(np.arange(nx * ny), nx)
    inner = (r > 0) & (r < ny - 1) & (j > 0) & (j < nx - 1)
    u = np.where(inner, rng.standard_normal(nx * ny), 0.0)[:, None]
    v = np.where(inner, rng.standard_normal(nx * ny), 0.0)[:, None]
    Vol = g["area"] * g["hx"] * g["hy"]
    div = m.divergence(u, v)[:, 0]
    assert abs(np.sum(Vol * div)) <= 1e-13 * np.sum(np.abs(Vol * div))
    cur = m.curl(u, v)[:, 0]
    assert abs(np.sum(Vol * cur)) <= 1e-13 * np.sum(np.abs(Vol * cur))


def test_adjoints_are_transposes():
    """<G f, y> = <f, G^T y> and <D w, z> = <w, D^T z> (plain sums)."""
    m = _mesh("mercator", 11, 9)
    rng = np.random.default_rng(7)
    V = m.nnodes
    f, y0, y1, u, v, z = (rng.standard_normal((V, 2)) for _ in range(6))
    gx, gy = m.gradient(f)
    lhs = np.sum(gx * y0) + np.sum(gy * y1)
    rhs = np.sum(f * m.gradient_adjoint(y0, y1))
    assert abs(lhs - rhs) <= 1e-13 * abs(lhs)
    d = m.divergence(u, v)
    xu, xv = m.divergence_adjoint(z)
    assert abs(np.sum(d * z) - (np.sum(u * xu) + np.sum(v * xv))) <= 1e-13 * abs(np.sum(d * z))


def _frames(proj, n, kw, dom):
    """Oracle mesh plus the unit vectors of the grid's x and y directions on
    the sphere, from meshes shifted by a tiny plane step."""
    xmin, xmax, ymin, ymax = dom
    m = oracle.RegionalMesh(proj, n, n, xmin, xmax, ymin, ymax, **kw)
    d = (xmax - xmin) * 1e-6

    def pos(sx, sy):
        gg = oracle.RegionalMesh(proj, n, n, xmin + sx, xmax + sx, ymin + sy, ymax + sy, **kw).geometry()
        return _unit(gg["lon"], gg["lat"])
    ex = pos(d, 0) - pos(-d, 0)
    ey = pos(0, d) - pos(0, -d)
    return m, ex / np.linalg.norm(ex, axis=1)[:, None], ey / np.linalg.norm(ey, axis=1)[:, None]


def _inner(n, k):
    r, j = np.divmod(np.arange(n * n), n)
    return (r >= k) & (r < n - k) & (j >= k) & (j < n - k)


def test_convergence_on_the_sphere():
    """f = z x (a degree-2 harmonic: Laplacian -6 f / R^2) and the solid-body
    rotation w = k x p (divergence 0, vorticity 2 k.p / R) on a 3000 km
    Lambert domain: interior errors fall at second order, boundary-node
    gradient errors at first order."""
    kw = dict(lat0=50.0, lon0=10.0)
    dom = (-1.5e6, 1.5e6, -1.5e6, 1.5e6)
    kax = np.array([0.3, -0.5, 0.8])
    kax /= np.linalg.norm(kax)
    errs = []
    for n in (16, 32, 64):
        m, ex, ey = _frames("lambert_conformal", n, kw, dom)
        g = m.geometry()
        P = _unit(g["lon"], g["lat"])
        f = P[:, 2] * P[:, 0]
        g3 = np.stack([P[:, 2], 0 * P[:, 0], P[:, 0]], 1)
        gt = (g3 - (g3 * P).sum(1)[:, None] * P) / R
        gx, gy = m.gradient(f[:, None])
        eg = np.maximum(np.abs(gx[:, 0] - (gt * ex).sum(1)), np.abs(gy[:, 0] - (gt * ey).sum(1))) * R
        lap = m.laplacian(f[:, None])[:, 0]
        el = np.abs(lap + 6.0 / R**2 * f) * R**2
        w = np.cross(kax, P)
        u, v = (w * ex).sum(1), (w * ey).sum(1)
        ed = np.abs(m.divergence(u[:, None], v[:, None])[:, 0]) * R
        ec = np.abs(m.curl(u[:, None], v[:, None])[:, 0] - 2.0 * (P @ kax) / R) * R
        I1, I2 = _inner(n, 1), _inner(n, 2)
        errs.append((eg[I1].max(), el[I2].max(), ec[I1].max(), eg[~I1].max(), ed[I1].max()))
    e = np.array(errs)
    slopes = np.log2(e[:-1] / e[1:])
    assert np.all(slopes[:, 0] >= 1.9) and np.all(slopes[:, 1] >= 1.9) and np.all(slopes[:, 2] >= 1.9), slopes
    assert np.all(slopes[:, 3] >= 0.95), slopes  # boundary nodes: first order
    assert np.all(e[:, 4] <= 1e-6)  # the rotation's divergence vanishes (to the frames' accuracy)


def test_closure_exact_and_averaged_forms_agree():
    """The oracle's closure-exact gradient and the averaged form differ only
    by f_i times the rounding residual of the cell's closure (plus the
    rounding of each sum)."""
    m = _mesh("lambert_south", 21, 15)
    g = m.geometry()
    rng = np.random.default_rng(8)
    f = (2.0 + np.cos(g["lat"]) * np.sin(2 * g["lon"]))[:, None] + 1e-3 * rng.standard_normal((m.nnodes, 1))
    gx, gy = m.gradient(f)
    ax, ay = m.gradient_averaged(f)
    res, ab = m.closure()
    eps = np.finfo(float).eps
    for c, (d, h) in enumerate(((gx - ax, g["hx"]), (gy - ay, g["hy"]))):
        bound = (np.abs(f[:, 0]) * (np.abs(res[:, c]) + 8 * eps * ab) + 8 * eps * ab * np.abs(f).max()) / (g["area"] * h)
        assert np.all(np.abs(d[:, 0]) <= bound)


@pytest.mark.parametrize("name", ["mercator", "lambert", "lambert_south", "polar"])
def test_plane_linear_fields_are_harmonic_on_conformal_grids(name):
    """On a conformal projection (h_x = h_y = h) a field linear in the plane
    is harmonic: the exact gradient (a, b)/(R h) makes h_y g_x and h_x g_y
    constant, whose flux divergence is 0.  The discrete Laplacian vanishes at
    every node, boundary included, to rounding of the gradient's size over
    a cell."""
    m = _mesh(name, 19, 14)
    g = m.geometry()
    x, y = g["x"], g["y"]
    f = (0.8 * x - 1.7 * y + 2.0)[:, None]
    lap = m.laplacian(f)[:, 0]
    gx, _ = m.gradient(f)
    scale = np.max(np.abs(gx)) / np.min(np.sqrt(g["area"]))  # |grad| / cell size
    assert np.max(np.abs(lap)) <= 1e-12 * scale  # about 1e-14 measured; a non-conformal grid gives 3e-3


def test_lambert_golden_fixture_unchanged():
    """The regional oracle still writes the frozen 4 x 3 Lambert fixture
    (tests/golden/lambert_4x3.txt, written by tests/golden/make_golden.py)."""
    import os
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "lambert_4x3.txt")
    rows = [l.split() for l in open(path) if not l.startswith("#")]
    want = np.array([[float.fromhex(v) for v in r] for r in rows])
    g = _mesh("lambert", 4, 3).geometry()
    got = np.stack([g[k] for k in ("lon", "lat", "hx", "hy", "area")], 1)
    assert want.shape == (12, 5) and np.array_equal(got, want)
