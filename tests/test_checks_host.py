"""Host-side consistency checks and fault injection (no GPU): every built
fvm passes ``atlas_fvm_check``; corrupting the host geometry through its
exposed arrays (a face normal, a volume) is detected with the bad node named;
the allocation-failure hook validates its argument."""
import ctypes

import numpy as np
import pytest

from synthetic.regional import DOMAINS


@pytest.fixture(scope="module")
def atlas(product):
    return product[0]


def test_every_grid_family_passes(atlas):
    worst = [atlas.build_fvm(N).check() for N in (1, 2, 16, 80)]
    worst.append(atlas.build_fvm(8, regular=True).check())
    for proj, kw in DOMAINS.values():
        worst.append(atlas.build_fvm_regional(proj, 13, 9, **kw).check())
    assert max(worst) <= 1e-14


def _host_array(ptr, n):
    return np.ctypeslib.as_array(ctypes.cast(ptr, ctypes.POINTER(ctypes.c_double)), shape=(n,))


def test_corrupted_normal_and_volume_are_detected(atlas, product):
    capi = product[1]
    fvm = atlas.build_fvm(8)
    V, S = ctypes.c_void_p(), ctypes.c_void_p()
    capi.atlas_fvm_info(fvm.handle, ctypes.byref(V), ctypes.byref(S), None, None)
    s = _host_array(S, 2 * fvm.mesh.nedges)
    e = 123
    a, b = fvm.mesh.arrays()["e2n"][e]
    keep = s[2 * e]
    s[2 * e] = keep * 1.001 + 1.0  # one face normal off: both cells of the edge stop closing
    with pytest.raises(capi.AtlasError) as ei:
        fvm.check()
    assert ei.value.code == -1 and "does not close" in str(ei.value)
    assert "node %d" % a in str(ei.value) or "node %d" % b in str(ei.value)
    s[2 * e] = keep
    assert fvm.check() <= 1e-14
    v = _host_array(V, fvm.nnodes)
    v[5] = -v[5]
    with pytest.raises(capi.AtlasError) as ei:
        fvm.check()
    assert "volume" in str(ei.value) and "node 5" in str(ei.value)
    v[5] = -v[5]
    assert fvm.check() <= 1e-14


def test_allocation_hook_arguments(product):
    capi = product[1]
    with pytest.raises(capi.AtlasError):
        capi.atlas_debug_fail_allocations(-2)
    capi.atlas_debug_fail_allocations(-1)
