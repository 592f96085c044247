"""The C ABI without a GPU: every symbol declared in include/atlas_gb.h is
exported, handles and arguments are validated on the host with the
documented error codes, and operator calls refuse to run without CUDA
(there is no CPU fallback)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "atlas_gb.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(atlas_[a-z0-9_]+)\s*\(", src)))


def test_every_declared_symbol_is_exported(product):
    _, capi = product
    names = _declared()
    assert len(names) >= 30
    for n in names:
        assert hasattr(capi.lib, n), n
        assert n in capi.EXPORTED, n


def test_error_codes_on_bad_arguments(product):
    atlas, capi = product
    E = capi.AtlasError
    out = ctypes.c_void_p()
    with pytest.raises(E) as ei:
        capi.atlas_grid_octahedral(0, ctypes.byref(out))
    assert ei.value.code == -1
    with pytest.raises(E) as ei:
        capi.atlas_grid_octahedral(8001, ctypes.byref(out))
    assert ei.value.code == -1
    with pytest.raises(E) as ei:
        capi.atlas_grid_octahedral(4, None)
    assert ei.value.code == -1
    fvm = atlas.build_fvm(4)
    h = fvm.handle
    fake = 1 << 20  # never dereferenced: validation fails first
    # bad dtype, ld < nlev, NULL field, misaligned field, overlapping fields
    for args, code in [((h, fake, fake + 4096, fake + 8192, 3, 4, 7, None), -5),
                       ((h, fake, fake + 4096, fake + 8192, 5, 4, 0, None), -1),
                       ((h, None, fake + 4096, fake + 8192, 3, 4, 0, None), -1),
                       ((h, fake + 2, fake + 4096, fake + 8192, 3, 4, 0, None), -4),
                       ((h, fake, fake, fake + 8192, 3, 4, 0, None), -1)]:
        with pytest.raises(E) as ei:
            capi.atlas_nabla_gradient(*args)
        assert ei.value.code == code, args
    assert capi.atlas_nabla_workspace_bytes(h, 0, 3, 4, 0) > 0
    assert capi.atlas_nabla_workspace_bytes(h, 3, 3, 4, 0) == 0
    with pytest.raises(E) as ei:
        capi.atlas_nabla_gradient_edges(h, fake, fake + 4096, fake + 8192, fake + 1 << 24, 16, 3, 4, 0, None)
    assert ei.value.code in (-1, -4)
    with pytest.raises(E) as ei:
        capi.atlas_fvm_set_launch(h, 0, -1, 3, 0, 0, 0, 0)
    assert ei.value.code == -1
    with pytest.raises(E) as ei:
        capi.atlas_fvm_set_launch(h, 0, -1, 0, 0, 0, 0, -1)
    assert ei.value.code == -1
    with pytest.raises(E) as ei:
        capi.atlas_fvm_set_launch(h, 0, 7, 0, 0, 0, 0, 1)
    assert ei.value.code == -5
    capi.atlas_fvm_set_launch(h, 0, -1, 0, 0, 0, 0, 16)
    capi.atlas_fvm_set_launch(h, 4, 1, 0, 3, 128, 0, 1)
    # node-group kernel settings: enable -1..2, blocks per SM 0..2, groups
    # per tile 0..15, nodes per warp 0, 2 or 4, rows per tile 0..3; a bad
    # one changes nothing
    for args in ((0, -1, 3, 0, 0, 0, 0), (0, -1, -2, 0, 0, 0, 0), (0, -1, 1, 3, 0, 0, 0), (0, -1, 1, 0, 16, 0, 0),
                 (0, -1, 1, 0, 0, 3, 0), (0, -1, 1, 0, 0, 1, 0), (8, -1, 1, 0, 0, 0, 0), (0, -1, 1, 0, 0, 0, 4),
                 (0, -1, 1, 0, 0, 0, -1)):
        with pytest.raises(E) as ei:
            capi.atlas_fvm_set_group(h, *args)
        assert ei.value.code == -1, args
    with pytest.raises(E) as ei:
        capi.atlas_fvm_set_group(h, 0, 5, 1, 0, 0, 0, 0)
    assert ei.value.code == -5
    for args in ((0, -1, 2, 2, 5, 2, 0), (4, 0, 0, 0, 0, 4, 2), (4, 2, -1, 1, 7, 0, 3)):
        capi.atlas_fvm_set_group(h, *args)
    # a destroyed handle is rejected, not dereferenced
    fvm.close()
    with pytest.raises(E) as ei:
        capi.atlas_nabla_gradient(h, fake, fake + 4096, fake + 8192, 3, 4, 0, None)
    assert ei.value.code == -6
    # a grid in use by a mesh is not destroyed
    g = atlas.Grid(2)
    m = atlas.Mesh(g)
    capi.atlas_grid_destroy(g.handle)
    capi.atlas_grid_info(g.handle, None, None, None, None, None)  # still alive
    m.close()
    g.close()


def test_no_cpu_fallback_without_cuda(product):
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a CUDA device is present")
    atlas, capi = product
    fvm = atlas.build_fvm(4)
    with pytest.raises(capi.AtlasError) as ei:
        capi.atlas_nabla_gradient(fvm.handle, 1 << 20, 1 << 21, 1 << 22, 3, 4, 0, None)
    assert ei.value.code == -3
    with pytest.raises(capi.AtlasError) as ei:
        capi.atlas_fvm_prepare(fvm.handle, 1, 1)
    assert ei.value.code == -3
    # the host-only inspection still works
    t = fvm.stencil_table("gradient")
    assert t["nbr"].shape[0] == 2 * fvm.mesh.nedges


def test_info_strings(product):
    _, capi = product
    assert capi.atlas_version().startswith(b"atlasgb")
    assert b"atlasgb" in capi.atlas_info()
    capi.atlas_init()
    capi.atlas_finalize()


def test_integral_argument_errors_without_a_gpu(product):
    """atlas_fvm_integral validates its arguments before touching the device."""
    atlas, capi = product
    fvm = atlas.build_fvm(4)
    need = capi.atlas_fvm_integral_workspace_bytes(fvm.handle, 7)
    assert need > 0 and need % 8 == 0
    fake = 0x100000
    bad = [
        (fake, -1, 10, 7, 8, capi.ATLAS_F32, fake, fake, need),          # negative node0
        (fake, 0, fvm.nnodes + 1, 7, 8, capi.ATLAS_F32, fake, fake, need),  # past the last node
        (fake, 0, 10, 7, 8, capi.ATLAS_F32, None, fake, need),           # out NULL
        (fake, 0, 10, 7, 8, capi.ATLAS_F32, fake + 4, fake, need),       # out misaligned
        (fake, 0, 10, 7, 8, capi.ATLAS_F32, fake, fake, need - 8),       # workspace too small
        (fake, 0, 10, 7, 6, capi.ATLAS_F32, fake, fake, need),           # ld < nlev
        (fake, 0, 10, 7, 8, 9, fake, fake, need),                        # unknown dtype
    ]
    for args in bad:
        with pytest.raises(capi.AtlasError) as ei:
            capi.atlas_fvm_integral(fvm.handle, *args, None)
        assert ei.value.code in (-1, -4, -5), args


def test_leading_dimension_above_int32_is_refused(product):
    """ld is bounded by 2^31 - 1, so that node * ld * element size cannot
    overflow; larger values are refused before any size is computed or the
    device is touched."""
    atlas, capi = product
    E = capi.AtlasError
    fvm = atlas.build_fvm(4)
    h = fvm.handle
    fake = 1 << 20
    for ld in (1 << 31, 1 << 40, (1 << 62) + 3):
        with pytest.raises(E) as ei:
            capi.atlas_nabla_gradient(h, fake, fake + 4096, fake + 8192, 3, ld, 0, None)
        assert ei.value.code == -1 and "2^31" in str(ei.value)
        with pytest.raises(E) as ei:
            capi.atlas_nabla_vector_gradient(h, fake, fake + 4096, fake + 8192, fake + 12288, fake + 16384,
                                             fake + 20480, 3, ld, 0, None)
        assert ei.value.code == -1
        assert capi.atlas_nabla_workspace_bytes(h, 0, 3, ld, 0) == 0
        with pytest.raises(E) as ei:
            capi.atlas_fvm_integral(h, fake, 0, 10, 7, ld, capi.ATLAS_F32, fake, fake, 1 << 20, None)
        assert ei.value.code == -1
    r = atlas.Remap(atlas.Mesh(atlas.Grid(4)), atlas.Grid(2, regular=True))
    for lds, ldd in ((1 << 31, 8), (8, 1 << 31)):
        with pytest.raises(E) as ei:
            capi.atlas_remap_apply(r.handle, fake, fake + (1 << 24), 3, lds, ldd, 0, None)
        assert ei.value.code == -1
    # the largest accepted ld passes validation and stops at the device check
    import torch
    if not torch.cuda.is_available():
        with pytest.raises(E) as ei:
            capi.atlas_nabla_gradient(h, fake, fake + (1 << 44), fake + (1 << 45), 3, (1 << 31) - 1, 0, None)
        assert ei.value.code == -3


def test_missing_library_fails_loudly(tmp_path):
    """A copy of the package without its built library cannot be imported:
    there is no other implementation to fall back on."""
    import shutil
    import subprocess
    import sys
    src = os.path.join(ROOT, "paper_1908_07038_gb300")
    dst = tmp_path / "paper_1908_07038_gb300"
    dst.mkdir()
    for name in os.listdir(src):
        if name.endswith(".py"):
            shutil.copy(os.path.join(src, name), dst / name)
    for mod in ("capi", "atlas", "batch", "partition", "hoststep", "tune"):
        r = subprocess.run([sys.executable, "-c", "import paper_1908_07038_gb300.%s" % mod], cwd=str(tmp_path),
                           capture_output=True, text=True, timeout=300,
                           env=dict(os.environ, PYTHONPATH=str(tmp_path)))
        assert r.returncode != 0, mod
        assert "ImportError" in r.stderr and "libatlasgb.so is not built" in r.stderr, (mod, r.stderr[-500:])


@pytest.mark.parametrize("compiler,std,src", [("gcc", "c89", "int main(void) { return 0; }\n"),
                                              ("gcc", "c99", "int main(void) { return 0; }\n"),
                                              ("g++", "c++11", "int main() { return 0; }\n"),
                                              ("g++", "c++17", "int main() { return 0; }\n")])
def test_header_compiles_alone(tmp_path, compiler, std, src):
    """include/atlas_gb.h is self-contained C: it compiles on its own, warning
    free under -pedantic, as C89, C99 and C++."""
    import shutil
    import subprocess
    if not shutil.which(compiler):
        pytest.skip(compiler + " missing")
    f = tmp_path / ("h.c" if compiler == "gcc" else "h.cpp")
    f.write_text('#include "atlas_gb.h"\n' + src)
    subprocess.check_call([compiler, "-std=" + std, "-Wall", "-Wextra", "-pedantic", "-Werror",
                           "-I", os.path.join(ROOT, "include"), "-c", str(f), "-o", str(tmp_path / "h.o")])
