"""Regional grids on the host (no GPU): the library's grid, mesh and plane
dual against the oracle (coordinates and scale factors to rounding,
connectivity bit-exact), the library's FP64 operator tables applied in
numpy against the oracle's operators (1e-13), and the refusals."""
import numpy as np
import pytest

from synthetic.regional import DOMAINS


@pytest.fixture(scope="module")
def atlas(product):
    return product[0]


def _pair(atlas, oracle_mod, name, nx, ny):
    proj, kw = DOMAINS[name]
    return atlas.build_fvm_regional(proj, nx, ny, **kw), oracle_mod.RegionalMesh(proj, nx, ny, **kw)


@pytest.mark.parametrize("name", list(DOMAINS))
def test_grid_mesh_and_dual_match_the_oracle(atlas, oracle_mod, name):
    nx, ny = 13, 9
    fvm, om = _pair(atlas, oracle_mod, name, nx, ny)
    g, og = fvm.grid.arrays(), om.geometry()
    assert fvm.nnodes == om.nnodes == nx * ny and fvm.grid.nlat == ny and np.all(g["pl"] == nx)
    for a, b in ((g["lon"], og["lon"]), (g["lat_node"], og["lat"]), (g["xy"][:, 0], og["x"]), (g["xy"][:, 1], og["y"]),
                 (g["scale"][:, 0], og["hx"]), (g["scale"][:, 1], og["hy"])):
        assert np.max(np.abs(a - b)) <= 4e-15 * max(1.0, np.max(np.abs(b)))
    m = fvm.mesh.arrays()
    assert fvm.mesh.ntri == om.ntri
    assert sorted(map(tuple, np.sort(m["tri"], 1).tolist())) == sorted(map(tuple, np.sort(og["tri"], 1).tolist()))
    edges = sorted({tuple(sorted((int(t[k]), int(t[(k + 1) % 3])))) for t in og["tri"] for k in range(3)})
    assert np.array_equal(m["e2n"], np.array(edges, dtype=np.int32))
    assert not m["is_pole"].any()
    d = fvm.arrays()
    assert np.max(np.abs(d["area"] - og["area"]) / og["area"]) <= 1e-14
    assert np.max(np.abs(d["V"] - og["area"] * og["hx"] * og["hy"]) / d["V"]) <= 1e-14
    # boundary normals only on the boundary edges, all pointing out of the rectangle
    nb = d["Sb"]
    on = np.abs(nb).sum(1) > 0
    assert on.sum() == 2 * (nx - 1) + 2 * (ny - 1)


def _apply(t, xs):
    """Difference-form table out_c(i) = sum_q W (x_m(nbr) - x_m(i)) + B x_m(i), in numpy."""
    V = len(t["ptr"]) - 1
    rows = np.repeat(np.arange(V), np.diff(t["ptr"]))
    nbr, w, b = t["nbr"], t["w"], t["b"]
    outs = [np.zeros_like(xs[0]) for _ in range(t["nout"])]
    if t["nin"] == 1:
        d = xs[0][nbr] - xs[0][rows]
        for c in range(t["nout"]):
            np.add.at(outs[c], rows, w[:, c][:, None] * d)
            outs[c] += b[:, c][:, None] * xs[0]
    else:
        for m in range(2):
            np.add.at(outs[0], rows, w[:, m][:, None] * (xs[m][nbr] - xs[m][rows]))
            outs[0] += b[:, m][:, None] * xs[m]
    return outs


def _rel(a, b):
    return np.max(np.abs(a - b)) / np.max(np.abs(b))


@pytest.mark.parametrize("name", list(DOMAINS))
def test_tables_equal_the_oracle_operators(atlas, oracle_mod, name):
    fvm, om = _pair(atlas, oracle_mod, name, 17, 11)
    V = fvm.nnodes
    rng = np.random.default_rng(11)
    x, y = rng.standard_normal((V, 3)), rng.standard_normal((V, 3))
    gx, gy = _apply(fvm.stencil_table("gradient"), [x])
    ox, oy = om.gradient(x)
    assert max(_rel(gx, ox), _rel(gy, oy)) <= 1e-13
    assert _rel(_apply(fvm.stencil_table("divergence"), [x, y])[0], om.divergence(x, y)) <= 1e-13
    assert _rel(_apply(fvm.stencil_table("curl"), [x, y])[0], om.curl(x, y)) <= 1e-13
    t = fvm.stencil_table("laplacian")
    rows = np.repeat(np.arange(V), np.diff(t["ptr"]))
    lap = np.zeros_like(x)
    np.add.at(lap, rows, t["w"][:, 0][:, None] * (x[t["nbr"]] - x[rows]))
    assert _rel(lap, om.laplacian(x)) <= 1e-13
    assert _rel(_apply(fvm.stencil_table("gradient_adjoint"), [x, y])[0], om.gradient_adjoint(x, y)) <= 1e-13
    au, av = _apply(fvm.stencil_table("divergence_adjoint"), [x])
    ou, ov = om.divergence_adjoint(x)
    assert max(_rel(au, ou), _rel(av, ov)) <= 1e-13
    vt, gt = fvm.stencil_table("vector_gradient"), fvm.stencil_table("gradient")
    assert np.array_equal(vt["w"], gt["w"]) and np.array_equal(vt["nbr"], gt["nbr"])


def test_refusals(atlas, product):
    capi = product[1]
    bad = [
        ("lambert_conformal", 1, 5, dict(xmin=-1e5, xmax=1e5, ymin=-1e5, ymax=1e5)),
        ("lambert_conformal", 5, 5, dict(xmin=1e5, xmax=-1e5, ymin=-1e5, ymax=1e5)),
        ("rotated_lonlat", 5, 5, dict(xmin=-5, xmax=5, ymin=80, ymax=90)),
        ("rotated_lonlat", 5, 5, dict(xmin=-180, xmax=180, ymin=0, ymax=10)),
        ("lambert_conformal", 5, 5, dict(xmin=-1e5, xmax=1e5, ymin=-1e5, ymax=1e5, lat0=0.0)),
        ("lambert_conformal", 5, 5, dict(xmin=-1e6, xmax=1e6, ymin=0.0, ymax=8e6, lat0=50.0)),  # holds the pole
        ("mercator", 5, 5, dict(xmin=-1e5, xmax=1e5, ymin=0.0, ymax=6e7)),
        ("mercator", 5, 5, dict(xmin=-1e5, xmax=1e5, ymin=-1e5, ymax=1e5, radius=-1.0)),
        ("polar_stereographic", 5, 5, dict(xmin=-1e5, xmax=1e5, ymin=-1e5, ymax=1e5, lat0=60.0)),  # not a pole
    ]
    for proj, nx, ny, kw in bad:
        with pytest.raises(capi.AtlasError) as ei:
            atlas.Grid.regional(proj, nx, ny, **kw)
        assert ei.value.code == -1, (proj, kw)
    import ctypes
    h = ctypes.c_void_p()
    prm = (ctypes.c_double * 8)(-1, 1, -1, 1, 0, 0, 0, 0)
    with pytest.raises(capi.AtlasError):
        capi.atlas_grid_regional(7, 5, 5, ctypes.cast(prm, ctypes.c_void_p), ctypes.byref(h))
    g = atlas.Grid(4)
    with pytest.raises(capi.AtlasError):
        capi.atlas_grid_regional_info(g.handle, None, None, None, None, None)


def test_remap_refuses_a_regional_source_and_takes_a_regional_target(atlas, oracle_mod, product, omesh):
    proj, kw = DOMAINS["lambert"]
    rg = atlas.Grid.regional(proj, 9, 7, **kw)
    with pytest.raises(product[1].AtlasError) as ei:
        atlas.Remap(atlas.Mesh(rg), atlas.Grid(4, regular=True))
    assert "global" in str(ei.value)
    r = atlas.Remap(atlas.Mesh(atlas.Grid(32)), rg)
    nodes, w = r.tables()
    a = rg.arrays()
    on, ow = omesh(32).remap_weights(np.stack([a["lon"], a["lat_node"]], 1))
    for t in range(len(nodes)):
        A, B = dict(zip(nodes[t].tolist(), w[t].tolist())), dict(zip(on[t].tolist(), ow[t].tolist()))
        assert max(abs(A.get(k, 0.0) - B.get(k, 0.0)) for k in set(A) | set(B)) <= 1e-14
    r.close()


def test_edge_variant_refuses_regional_before_any_pointer_use(atlas, product):
    capi = product[1]
    proj, kw = DOMAINS["mercator"]
    fvm = atlas.build_fvm_regional(proj, 9, 7, **kw)
    fake = [0x10000 * (k + 1) for k in range(4)]  # never dereferenced: the call is refused first
    for fn, args in [(capi.atlas_nabla_gradient_edges, fake[:3]), (capi.atlas_nabla_laplacian_edges, fake[:2])]:
        with pytest.raises(capi.AtlasError) as ei:
            fn(fvm.handle, *args, fake[3], 1 << 20, 4, 4, capi.ATLAS_F32, None)
        assert ei.value.code == -1 and "global" in str(ei.value)


@pytest.mark.parametrize("name", ["mercator", "lambert", "lambert_south"])
def test_laplacian_table_is_zero_on_plane_linear_fields(atlas, name):
    """The library's composed two-ring Laplacian table (FP64, applied in
    numpy) annihilates fields linear in a conformal projection's plane at
    every node, boundary included (they are harmonic there)."""
    proj, kw = DOMAINS[name]
    fvm = atlas.build_fvm_regional(proj, 19, 14, **kw)
    g = fvm.grid.arrays()
    x, y = g["xy"][:, 0], g["xy"][:, 1]
    f = 0.8 * x - 1.7 * y + 2.0
    t = fvm.stencil_table("laplacian")
    V = fvm.nnodes
    rows = np.repeat(np.arange(V), np.diff(t["ptr"]))
    lap = np.zeros(V)
    np.add.at(lap, rows, t["w"][:, 0] * (f[t["nbr"]] - f[rows]))
    gx = _apply(fvm.stencil_table("gradient"), [f[:, None]])[0][:, 0]
    scale = np.max(np.abs(gx)) / np.min(np.sqrt(fvm.arrays()["area"]))
    assert np.max(np.abs(lap)) <= 1e-12 * scale
