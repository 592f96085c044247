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
