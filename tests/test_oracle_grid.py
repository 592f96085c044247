"""Pins of the oracle's grid and mesh (latitudes, octahedral rows, zipper
triangulation, pole edges, CSR) against mathematics and brute force.

The paper names the grids only ("O32", "F8", Sec. 4.3, Fig. 4); the row rule,
zipper and pole edges are the readings stated in ``oracle/atlas_oracle.c``.
"""
from fractions import Fraction

import numpy as np
import pytest

R = 6371220.0


@pytest.mark.parametrize("n", [2, 4, 32, 64, 128, 640])
def test_latitudes_match_legendre_roots(oracle_mod, n):
    theta = oracle_mod.gauss_colatitudes(n)
    x, _ = np.polynomial.legendre.leggauss(n)
    # leggauss returns ascending x; colatitudes ascend from the north pole
    assert np.max(np.abs(np.cos(theta) - x[::-1])) <= 1e-14
    # exact mirror symmetry and strict ordering
    h = n // 2
    assert np.array_equal(theta[::-1][:h], np.pi - theta[:h])
    assert np.all(np.diff(theta) > 0)


def test_latitudes_near_pole_are_roots(oracle_mod):
    # P_n(cos t) changes sign across every returned root: evaluate the
    # Legendre series with numpy at t(1 -/+ 1e-9); near the pole this checks
    # the colatitude to ~1e-9 relative, where x-space comparisons cannot.
    n = 2560
    theta = oracle_mod.gauss_colatitudes(n)[:8]
    c = np.zeros(n + 1); c[-1] = 1.0
    lo = np.polynomial.legendre.legval(np.cos(theta * (1 - 1e-9)), c)
    hi = np.polynomial.legendre.legval(np.cos(theta * (1 + 1e-9)), c)
    assert np.all(np.sign(lo) != np.sign(hi))


@pytest.mark.parametrize("N", [1, 2, 3, 4, 8, 16, 32])
def test_counts(omesh, N):
    m = omesh(N)
    V = 4 * N * N + 36 * N
    assert m.nnodes == V
    assert m.ntri == 2 * V - 40
    assert m.nedges == 3 * V - 20
    g = m.grid()
    pl = g["pl"]
    for r in range(2 * N):
        i = r + 1 if r < N else 2 * N - r
        assert pl[r] == 4 * i + 16
    d = m.mesh()
    assert d["n2e_ptr"][-1] == 2 * m.nedges
    # Euler characteristic of the sphere minus two polar holes
    assert m.nnodes - (m.nedges - 20) + m.ntri == 0


def _zipper_bruteforce(n1, n2):
    """Triangles of one band from a merged sort of the 'next longitude' events
    (Fractions; ties: the row with fewer points first, equal rows: north)."""
    events = [(Fraction(a, n1), 0) for a in range(1, n1 + 1)] + [(Fraction(b, n2), 1) for b in range(1, n2 + 1)]
    north_first = 0 if n1 <= n2 else 1

    def key(ev):
        lam, row = ev
        return (lam, 0 if row == north_first else 1)

    events.sort(key=key)
    ia = ib = 0
    tris = []
    for _, row in events:
        if row == 0:
            tris.append(((0, ia), (0, ia + 1), (1, ib)))
            ia += 1
        else:
            tris.append(((0, ia), (1, ib), (1, ib + 1)))
            ib += 1
    return tris


@pytest.mark.parametrize("N", [2, 3])
def test_zipper_bruteforce(omesh, N):
    m = omesh(N)
    d = m.mesh()
    g = m.grid()
    pl = g["pl"]
    got = {}
    for t in range(m.ntri):
        r = int(d["tri_r"][t].min())
        tri = tuple((int(d["tri_r"][t, k]) - r, int(d["tri_j"][t, k])) for k in range(3))
        got.setdefault(r, []).append(tri)
    ties = 0
    for r in range(2 * N - 1):
        want = _zipper_bruteforce(int(pl[r]), int(pl[r + 1]))
        assert got[r] == want
        n1, n2 = int(pl[r]), int(pl[r + 1])
        ties += sum(1 for a in range(1, n1 + 1) if Fraction(a, n1) * n2 == int(Fraction(a, n1) * n2))
    # 4 tie events per non-equatorial band, n per equatorial band (incl. the closing one)
    assert ties == 4 * (2 * N - 2) + (4 * N + 16)


def test_o2_triangles_tile_each_band(omesh):
    """Every band is tiled: the plain (lon, lat) areas of its triangles add up
    to the strip area, every triangle is non-degenerate and all have the same
    orientation within their type, and each side is shared correctly."""
    m = omesh(2)
    d = m.mesh()
    g = m.grid()
    pl, lat = g["pl"], g["lat"]
    areas = {}
    for t in range(m.ntri):
        r = d["tri_r"][t]
        lam = 2 * np.pi * d["tri_j"][t] / pl[r]
        phi = lat[r]
        a = 0.5 * ((lam[1] - lam[0]) * (phi[2] - phi[0]) - (lam[2] - lam[0]) * (phi[1] - phi[0]))
        assert abs(a) > 1e-6
        areas.setdefault(int(r.min()), []).append(abs(a))
    for r, al in areas.items():
        strip = 2 * np.pi * (lat[r] - lat[r + 1])
        assert abs(sum(al) - strip) <= 1e-13 * strip
    # side incidence: every regular side in 2 triangles, except ring sides of
    # the first and last row (1 triangle)
    cnt = {}
    for t in range(m.ntri):
        v = d["tri"][t]
        for k in range(3):
            a, b = sorted((int(v[k]), int(v[(k + 1) % 3])))
            cnt[(a, b)] = cnt.get((a, b), 0) + 1
    off = np.concatenate([[0], np.cumsum(pl)])
    rows = np.searchsorted(off, np.arange(m.nnodes), side="right") - 1
    for (a, b), c in cnt.items():
        polar_ring = rows[a] == rows[b] and rows[a] in (0, 2 * m.N - 1)
        assert c == (1 if polar_ring else 2)
    # edges = sides + 20 pole edges
    e2n = d["e2n"]
    regular = {tuple(map(int, e)) for e, p in zip(e2n, d["is_pole"]) if not p}
    assert regular == set(cnt)


@pytest.mark.parametrize("N", [2, 5, 16])
def test_edges_csr_and_pole_edges(omesh, N):
    m = omesh(N)
    d = m.mesh()
    g = m.grid()
    pl = g["pl"]
    e2n, is_pole = d["e2n"], d["is_pole"]
    assert np.all(e2n[:, 0] < e2n[:, 1])
    key = e2n[:, 0].astype(np.int64) * (1 << 32) + e2n[:, 1]
    assert np.all(np.diff(key) > 0)
    pole = e2n[is_pole.astype(bool)]
    last = m.nnodes - pl[-1]
    want = [(j, j + 10) for j in range(10)] + [(last + j, last + j + 10) for j in range(10)]
    assert sorted(map(tuple, pole.tolist())) == want
    ptr, n2e, sg = d["n2e_ptr"], d["n2e"], d["n2e_sign"]
    for i in range(m.nnodes):
        es = n2e[ptr[i]:ptr[i + 1]]
        assert np.all(np.diff(es) > 0)
        for e, s in zip(es, sg[ptr[i]:ptr[i + 1]]):
            assert e2n[e, 0 if s == 1 else 1] == i


@pytest.mark.parametrize("N", [3, 8])
def test_mesh_symmetries(omesh, N):
    """Quarter-turn invariance of the integer zipper and N/S mirror symmetry
    away from the equator band."""
    m = omesh(N)
    d = m.mesh()
    pl = m.grid()["pl"]
    tri = {}
    for t in range(m.ntri):
        r = d["tri_r"][t]
        j = d["tri_j"][t] % pl[r]
        tri[t] = frozenset(zip(r.tolist(), j.tolist()))
    S = set(tri.values())
    rot = {frozenset((r, (j + pl[r] // 4) % pl[r]) for r, j in s) for s in S}
    assert rot == S
    nl = 2 * N
    mirror = {frozenset((nl - 1 - r, j) for r, j in s) for s in S}
    band = lambda s: min(r for r, _ in s)
    keep = lambda s: band(s) != N - 1
    assert {s for s in mirror if keep(s)} == {s for s in S if keep(s)}


def test_o2_golden_fixture_unchanged(omesh):
    """The oracle still writes the frozen O2 fixtures (tests/golden)."""
    import os
    here = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
    m = omesh(2)
    d = m.mesh()
    du = m.dual()
    lines = [l for l in open(os.path.join(here, "o2_connectivity.txt")) if not l.startswith("#")]
    assert tuple(map(int, lines[0].split())) == (m.nnodes, m.ntri, m.nedges)
    e = np.array([list(map(int, l.split())) for l in lines[1:1 + m.nedges]])
    assert np.array_equal(e[:, :2], d["e2n"]) and np.array_equal(e[:, 2], d["is_pole"])
    assert np.array_equal(np.array(lines[1 + m.nedges].split(), dtype=np.int64), d["n2e_ptr"])
    vals = [l.split() for l in open(os.path.join(here, "o2_dual.txt")) if not l.startswith("#")]
    V = np.array([float.fromhex(v[0]) for v in vals[:m.nnodes]])
    S = np.array([[float.fromhex(a), float.fromhex(b)] for a, b in vals[m.nnodes:]])
    assert np.array_equal(V, du["V"]) and np.array_equal(S, du["S"])
