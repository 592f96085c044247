"""Geometry cache (host only): an fvm saved with ``atlas_fvm_save`` and read
back with ``atlas_fvm_load`` has bit-identical grid, mesh, dual and operator
tables, passes the consistency check, and works with the rest of the API;
damaged files (a flipped byte, a cut end, a foreign file, a missing path)
are refused with the reason."""
import numpy as np
import pytest

from synthetic.regional import DOMAINS


@pytest.fixture(scope="module")
def atlas(product):
    return product[0]


def _same_dicts(a, b):
    assert a.keys() == b.keys()
    for k in a:
        assert np.array_equal(a[k], b[k]), k


@pytest.mark.parametrize("which", ["O16", "F8", "lambert", "rotated"])
def test_round_trip_is_bit_exact(atlas, tmp_path, which):
    if which == "O16":
        fvm = atlas.build_fvm(16)
    elif which == "F8":
        fvm = atlas.build_fvm(8, regular=True)
    else:
        proj, kw = DOMAINS[which]
        fvm = atlas.build_fvm_regional(proj, 13, 9, **kw)
    path = tmp_path / "geom.bin"
    fvm.save(path)
    got = atlas.load_fvm(path)
    assert (got.nnodes, got.mesh.nedges, got.mesh.ntri, got.R) == (fvm.nnodes, fvm.mesh.nedges, fvm.mesh.ntri, fvm.R)
    assert (got.grid.projection, got.grid.N, got.grid.regular) == (fvm.grid.projection, fvm.grid.N, fvm.grid.regular)
    _same_dicts(got.grid.arrays(), fvm.grid.arrays())
    _same_dicts(got.mesh.arrays(), fvm.mesh.arrays())
    _same_dicts(got.arrays(), fvm.arrays())
    for op in ("gradient", "divergence", "laplacian", "gradient_adjoint", "curl"):
        a, b = got.stencil_table(op), fvm.stencil_table(op)
        for k in ("ptr", "nbr", "w", "b"):
            assert np.array_equal(a[k], b[k]), (op, k)
    assert got.check() == fvm.check()


def test_damaged_files_are_refused(atlas, product, tmp_path):
    capi = product[1]
    fvm = atlas.build_fvm(8)
    path = tmp_path / "geom.bin"
    fvm.save(path)
    raw = bytearray(path.read_bytes())
    cases = {"checksum": None, "truncated": None, "not a geometry file": None, "cannot open": None}
    flipped = bytearray(raw)
    flipped[len(raw) // 2] ^= 0x10
    (tmp_path / "flip.bin").write_bytes(bytes(flipped))
    (tmp_path / "cut.bin").write_bytes(bytes(raw[:len(raw) - 100]))
    (tmp_path / "foreign.bin").write_bytes(b"#!/bin/sh\n" + bytes(200))
    for name, why in (("flip.bin", "checksum"), ("cut.bin", "truncated"), ("foreign.bin", "not a geometry file"),
                      ("missing.bin", "cannot open")):
        with pytest.raises(capi.AtlasError) as ei:
            atlas.load_fvm(tmp_path / name)
        assert ei.value.code == -1 and why in str(ei.value), (name, str(ei.value))
        cases[why] = True
    assert all(cases.values())


# ---------------------------------------------------------------- file pieces
_FNV_OFFSET, _FNV_PRIME, _M64 = 1469598103934665603, 1099511628211, (1 << 64) - 1
# vectors of a geometry file in write order, with their element types
_VECS = (("pl", "<i4"), ("off", "<i8"), ("colat", "<f8"), ("lat", "<f8"), ("lonlat", "<f8"), ("xy", "<f8"),
         ("h", "<f8"), ("e2n", "<i4"), ("is_pole", "u1"), ("n2e_ptr", "<i4"), ("n2e", "<i4"), ("n2e_sign", "<i1"),
         ("tri", "<i4"), ("side_off", "<f8"), ("side_lat", "<f8"), ("mid_lat", "<f8"), ("S", "<f8"), ("V", "<f8"),
         ("coslat", "<f8"), ("pole_nphi", "<f8"), ("A", "<f8"), ("Sb", "<f8"))


def _pieces(raw):
    """Split a geometry file into the pieces its writer hashed one by one:
    magic, version, reserved word, eight sizes, the radius, eight projection
    parameters, then per vector (length, element size, reserved, data);
    returns [(offset, length)] and the offsets of each vector's data."""
    out, data, o = [], {}, 0

    def take(n):
        nonlocal o
        out.append((o, n))
        o += n

    for n in (8, 4, 4) + (8,) * 8 + (8,) + (8,) * 8:
        take(n)
    for name, dt in _VECS:
        n = int(np.frombuffer(raw, "<u8", 1, o)[0])
        es = int(np.frombuffer(raw, "<u4", 1, o + 8)[0])
        assert es == np.dtype(dt).itemsize, (name, es)
        take(8), take(4), take(4)
        data[name] = (o, n, dt)
        if n:
            take(n * es)
    assert o == len(raw) - 8
    return out, data


def _fnv(raw, pieces):
    """The file's checksum: FNV-1a over each piece's 64-bit little-endian
    words, then its remaining bytes."""
    h = _FNV_OFFSET
    for o, n in pieces:
        k = 0
        while k + 8 <= n:
            h = ((h ^ int.from_bytes(raw[o + k:o + k + 8], "little")) * _FNV_PRIME) & _M64
            k += 8
        for c in raw[o + k:o + n]:
            h = ((h ^ c) * _FNV_PRIME) & _M64
    return h


def test_out_of_range_connectivity_is_refused_before_any_launch(atlas, product, tmp_path):
    """A geometry file whose checksum is right but whose edge table points
    past the last node (a corrupted table, not a damaged file) is refused by
    the host validation of atlas_fvm_load, with the reason; no table built
    from it ever reaches a kernel.  The same holds for a node->edge entry
    past the last edge."""
    capi = product[1]
    fvm = atlas.build_fvm(8)
    path = tmp_path / "geom.bin"
    fvm.save(path)
    raw = bytearray(path.read_bytes())
    pieces, data = _pieces(raw)
    assert _fnv(raw, pieces) == int.from_bytes(raw[-8:], "little")  # the checksum is understood
    V, E = fvm.nnodes, fvm.mesh.nedges
    for name, index, value, why in (("e2n", 2 * (E // 2) + 1, V + 5, "edge ends out of range"),
                                    ("n2e", 7, E + 3, "edge id out of range (node 1)")):
        bad = bytearray(raw)
        o, n, dt = data[name]
        es = np.dtype(dt).itemsize
        bad[o + index * es:o + (index + 1) * es] = int(value).to_bytes(es, "little", signed=True)
        bad[-8:] = _fnv(bad, pieces).to_bytes(8, "little")
        p = tmp_path / ("bad_%s.bin" % name)
        p.write_bytes(bytes(bad))
        with pytest.raises(capi.AtlasError) as ei:
            atlas.load_fvm(p)
        assert ei.value.code == -1 and "inconsistent" in str(ei.value) and why in str(ei.value), (name, str(ei.value))
    # the untouched bytes still load
    assert atlas.load_fvm(path).nnodes == V
