"""The product's host geometry (C++, edge-based construction) against the
oracle (C, triangle loop): connectivity and CSR bit-exact, FP64 geometry
bit-exact, and the operator stencil tables evaluated on the CPU agreeing
with the oracle's operators.  No GPU is used.
"""
import numpy as np
import pytest

R = 6371220.0


@pytest.mark.parametrize("N", [1, 2, 5, 16, 32, 80])
def test_geometry_bitwise_equal_to_oracle(pfvm, omesh, N):
    f = pfvm(N)
    om = omesh(N)
    g, og = f.grid.arrays(), om.grid()
    assert np.array_equal(g["pl"], og["pl"])
    assert np.array_equal(g["lat"], og["lat"])
    assert np.array_equal(g["lon"], og["lon"]) and np.array_equal(g["lat_node"], og["lat_node"])
    m, omm = f.mesh.arrays(), om.mesh()
    for k in ("e2n", "is_pole", "n2e_ptr", "n2e", "n2e_sign", "tri"):
        assert np.array_equal(m[k], omm[k]), k
    d, od = f.arrays(), om.dual()
    for k in ("S", "V", "coslat", "pole_nphi"):
        assert np.array_equal(d[k], od[k]), k


def _apply(tab, xs):
    """Evaluate a stencil table on the CPU (test-side numpy, FP64):
    out_c(i) = sum_q sum_m W_cm(q) (x_m(nbr q) - x_m(i)) + sum_m B_cm(i) x_m(i)."""
    ptr, nbr, w, b = tab["ptr"], tab["nbr"], tab["w"], tab["b"]
    V = ptr.shape[0] - 1
    rows = np.repeat(np.arange(V), np.diff(ptr))
    L = xs[0].shape[1]
    outs = []
    if tab["nin"] == 1:
        d = xs[0][nbr] - xs[0][rows]
        for c in range(tab["nout"]):
            o = np.zeros((V, L))
            np.add.at(o, rows, w[:, c:c + 1] * d)
            o += b[:, c:c + 1] * xs[0]
            outs.append(o)
    else:
        o = np.zeros((V, L))
        for mm in range(2):
            np.add.at(o, rows, w[:, mm:mm + 1] * (xs[mm][nbr] - xs[mm][rows]))
            o += b[:, mm:mm + 1] * xs[mm]
        outs.append(o)
    return outs


def _relmax(a, b):
    return np.max(np.abs(a - b)) / np.max(np.abs(b))


@pytest.mark.parametrize("N", [2, 8, 16])
def test_stencil_tables_reproduce_oracle(pfvm, omesh, N):
    f = pfvm(N)
    om = omesh(N)
    rng = np.random.default_rng(N)
    L = 3
    x, y = rng.standard_normal((2, f.nnodes, L))
    g = om.grid()
    smooth = np.cos(g["lat_node"])[:, None] * np.cos(g["lon"])[:, None] * (1 + 0.1 * np.arange(L))
    for inp in (x, smooth + 1e-3 * y):
        gx, gy = _apply(f.stencil_table("gradient"), [inp])
        ox, oy = om.gradient(inp)
        assert _relmax(gx, ox) <= 1e-13 and _relmax(gy, oy) <= 1e-13
        (d,) = _apply(f.stencil_table("divergence"), [inp, y])
        assert _relmax(d, om.divergence(inp, y)) <= 1e-13
        (lap,) = _apply(f.stencil_table("laplacian"), [inp])
        assert _relmax(lap, om.laplacian(inp)) <= 1e-12
        (ga,) = _apply(f.stencil_table("gradient_adjoint"), [inp, y])
        assert _relmax(ga, om.gradient_adjoint(inp, y)) <= 1e-13
        du, dv = _apply(f.stencil_table("divergence_adjoint"), [inp])
        ou, ov = om.divergence_adjoint(inp)
        assert _relmax(du, ou) <= 1e-13 and _relmax(dv, ov) <= 1e-13
        (z,) = _apply(f.stencil_table("curl"), [inp, y])
        assert _relmax(z, om.curl(inp, y)) <= 1e-13
        vg = _apply(f.stencil_table("vector_gradient"), [inp]) + _apply(f.stencil_table("vector_gradient"), [y])
        for a, b in zip(vg, om.vector_gradient(inp, y)):
            assert _relmax(a, b) <= 1e-13


def test_vector_table_shapes(pfvm):
    """Curl: two inputs, one output, B term, no pole entries; vector
    gradient: one input (a component), two outputs, B term only on the
    polar rows, the same neighbours as the gradient."""
    f = pfvm(8)
    c, d = f.stencil_table("curl"), f.stencil_table("divergence")
    assert (c["nin"], c["nout"]) == (2, 1)
    assert np.array_equal(c["ptr"], d["ptr"]) and np.array_equal(c["nbr"], d["nbr"])
    assert np.array_equal(c["w"][:, 0], -d["w"][:, 1]) and np.array_equal(c["w"][:, 1], d["w"][:, 0])
    vg, g = f.stencil_table("vector_gradient"), f.stencil_table("gradient")
    assert (vg["nin"], vg["nout"]) == (1, 2)
    assert np.array_equal(vg["ptr"], g["ptr"]) and np.array_equal(vg["nbr"], g["nbr"])
    flipped = np.any(vg["w"] != g["w"], axis=1)
    pl0 = int(f.grid.arrays()["pl"][0])
    rows = np.repeat(np.arange(f.nnodes), np.diff(g["ptr"]))
    assert np.all(np.isin(rows[flipped], np.r_[0:pl0, f.nnodes - pl0:f.nnodes]))
    assert np.count_nonzero(flipped) == 2 * pl0  # one pole entry per polar node
    assert np.array_equal(vg["w"][flipped], -g["w"][flipped])
    assert np.count_nonzero(np.any(vg["b"] != 0, axis=1)) == 2 * pl0


def test_laplacian_table_rows_sum_to_zero_structure(pfvm):
    """The fused Laplacian stores only off-diagonal entries of L = D G; the
    two-ring has ~18 neighbours per interior node."""
    f = pfvm(16)
    t = f.stencil_table("laplacian")
    deg = np.diff(t["ptr"])
    assert 12 <= np.median(deg) <= 24
    assert t["nin"] == 1 and t["nout"] == 1
