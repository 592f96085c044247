"""GPU parity of the curl and the vector gradient (through the C ABI) with the
FP64 oracle on the same seeded inputs.

Tolerances as for the scalar operators (relative max-norm per output
component): FP64 1e-13, FP32 1e-5, BF16 storage 2e-2, the oracle fed the
same rounded inputs.  Full comparisons on O16..O80 with ragged level counts;
O320 and O1280 x 137 on sampled nodes (every polar-row node and every row's
first and last node included)."""
import numpy as np
import pytest

import synthetic

pytestmark = pytest.mark.gpu

TOL = {np.float64: 1e-13, np.float32: 1e-5}


@pytest.fixture(scope="module")
def torch():
    t = pytest.importorskip("torch")
    if not t.cuda.is_available():
        pytest.skip("no CUDA device")
    return t


def _relmax(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    den = np.max(np.abs(b))
    return np.max(np.abs(a - b)) / (den if den > 0 else 1.0)


def _dev(torch, x, ld, dtype=None):
    t = torch.from_numpy(np.ascontiguousarray(synthetic.padded(np.asarray(x), ld)))
    if dtype is not None:
        t = t.to(dtype)
    return t.cuda()


def _run(torch, fvm, tu, tv, nlev):
    z = fvm.curl(tu, tv, nlev)
    vg = fvm.vector_gradient(tu, tv, nlev)
    torch.cuda.synchronize()
    return [z] + list(vg)


def _want(om, u, v, nlev, nodes=None):
    return [om.curl(u, v, nlev, nodes=nodes)] + list(om.vector_gradient(u, v, nlev, nodes=nodes))


@pytest.mark.parametrize("N,nlev,ld,dt", [(16, 1, 2, np.float64), (32, 5, 6, np.float64), (80, 137, 138, np.float64),
                                          (16, 3, 4, np.float32), (32, 7, 8, np.float32), (80, 137, 140, np.float32),
                                          (80, 9, 9, np.float32)])
def test_full_parity(torch, pfvm, omesh, N, nlev, ld, dt):
    fvm, om = pfvm(N), omesh(N)
    g = om.grid()
    u, v = synthetic.level_vector(g["lon"], g["lat_node"], nlev, dt)
    got = _run(torch, fvm, _dev(torch, u, ld), _dev(torch, v, ld), nlev)
    want = _want(om, u, v, nlev)
    worst = [_relmax(a[:, :nlev].double().cpu().numpy(), b) for a, b in zip(got, want)]
    assert max(worst) <= TOL[dt], worst


def test_bf16_storage(torch, pfvm, omesh):
    fvm, om = pfvm(32), omesh(32)
    g = om.grid()
    u, v = synthetic.level_vector(g["lon"], g["lat_node"], 8, np.float32)
    tu, tv = _dev(torch, u, 8, torch.bfloat16), _dev(torch, v, 8, torch.bfloat16)
    got = _run(torch, fvm, tu, tv, 8)
    ur, vr = (t.float().cpu().numpy() for t in (tu, tv))
    want = _want(om, ur, vr, 8)
    worst = [_relmax(a.float().cpu().numpy(), b) for a, b in zip(got, want)]
    assert max(worst) <= 2e-2, worst


def test_vector_gradient_is_the_scalar_gradient_off_the_polar_rows(torch, pfvm):
    """Same neighbours and weights off the polar rows (the B term adds exact
    zeros there): bitwise equal to atlas_nabla_gradient of each component.
    On the polar rows the meridional components differ (the pole face has a
    purely meridional normal, so the zonal ones do not)."""
    fvm = pfvm(32)
    rng = np.random.default_rng(4)
    u = torch.from_numpy(rng.standard_normal((fvm.nnodes, 12)).astype(np.float32)).cuda()
    v = torch.from_numpy(rng.standard_normal((fvm.nnodes, 12)).astype(np.float32)).cuda()
    ux, uy, vx, vy = fvm.vector_gradient(u, v)
    sx, sy = fvm.gradient(u)
    tx, ty = fvm.gradient(v)
    torch.cuda.synchronize()
    pl0 = int(fvm.grid.arrays()["pl"][0])
    inner = slice(pl0, fvm.nnodes - pl0)
    for a, b in ((ux, sx), (uy, sy), (vx, tx), (vy, ty)):
        assert torch.equal(a[inner], b[inner])
    for a, b in ((ux, sx), (vx, tx)):
        assert torch.equal(a, b)
    for a, b in ((uy, sy), (vy, ty)):
        assert not torch.equal(a[:pl0], b[:pl0]) and not torch.equal(a[-pl0:], b[-pl0:])


def test_overlapping_outputs_are_rejected(torch, pfvm):
    from paper_1908_07038_gb300.capi import AtlasError
    fvm = pfvm(16)
    u = torch.zeros((fvm.nnodes, 4), device="cuda")
    v = torch.zeros_like(u)
    a, b, c = (torch.zeros_like(u) for _ in range(3))
    with pytest.raises(AtlasError):
        fvm.vector_gradient(u, v, out=(a, b, c, a))
    with pytest.raises(AtlasError):
        fvm.vector_gradient(u, v, out=(a, b, c, v))
    with pytest.raises(AtlasError):
        fvm.curl(u, v, out=u)


@pytest.mark.parametrize("N,count,dt,ld", [(320, 20000, np.float32, 140), (320, 20000, np.float64, 138),
                                           (1280, 6000, np.float32, 140), (1280, 3000, np.float64, 138)])
def test_sampled_137_levels(torch, pfvm, omesh, N, count, dt, ld):
    fvm, om = pfvm(N), omesh(N)
    g = om.grid()
    off = np.concatenate([[0], np.cumsum(g["pl"])])
    nodes = synthetic.sample_nodes(om.nnodes, off, count)
    u, v = synthetic.level_vector(g["lon"], g["lat_node"], 137, dt)
    tu, tv = _dev(torch, u, ld), _dev(torch, v, ld)
    got = _run(torch, fvm, tu, tv, 137)
    idx = torch.from_numpy(nodes).cuda()
    want = _want(om, u, v, 137, nodes=nodes)
    worst = [_relmax(a.index_select(0, idx)[:, :137].double().cpu().numpy(), b) for a, b in zip(got, want)]
    del tu, tv, got
    torch.cuda.empty_cache()
    assert max(worst) <= TOL[dt], worst


# ------------------------------------------------------------ curl adjoint
@pytest.mark.parametrize("N,nlev,ld,dt", [(16, 3, 4, np.float64), (80, 137, 138, np.float64),
                                          (16, 5, 8, np.float32), (80, 137, 140, np.float32),
                                          (32, 9, 9, np.float32)])
def test_curl_adjoint_parity(torch, pfvm, omesh, N, nlev, ld, dt):
    """atlas_nabla_curl_adjoint against the oracle's transpose of the curl's
    matrix rows, on N(0,1) inputs."""
    fvm, om = pfvm(N), omesh(N)
    rng = np.random.default_rng(N + nlev)
    z = rng.standard_normal((om.nnodes, nlev)).astype(dt)
    gu, gv = fvm.curl_adjoint(_dev(torch, z, ld), nlev)
    torch.cuda.synchronize()
    wu, wv = om.curl_adjoint(z)
    worst = [_relmax(a[:, :nlev].double().cpu().numpy(), b) for a, b in ((gu, wu), (gv, wv))]
    assert max(worst) <= TOL[dt], worst


def test_curl_adjoint_bf16(torch, pfvm, omesh):
    fvm, om = pfvm(32), omesh(32)
    rng = np.random.default_rng(5)
    z = rng.standard_normal((om.nnodes, 8)).astype(np.float32)
    tz = _dev(torch, z, 8, torch.bfloat16)
    gu, gv = fvm.curl_adjoint(tz, 8)
    torch.cuda.synchronize()
    wu, wv = om.curl_adjoint(tz.float().cpu().numpy())
    worst = [_relmax(a.float().cpu().numpy(), b) for a, b in ((gu, wu), (gv, wv))]
    assert max(worst) <= 2e-2, worst


def test_curl_backward_is_the_curl_adjoint_kernel(torch, pfvm):
    """CurlFn.backward returns exactly what atlas_nabla_curl_adjoint gives
    (no arithmetic of the binding's own)."""
    from paper_1908_07038_gb300 import atlas
    fvm = pfvm(16)
    rng = np.random.default_rng(6)
    u, v, zb = (torch.from_numpy(rng.standard_normal((fvm.nnodes, 4))).cuda() for _ in range(3))
    u.requires_grad_(True)
    v.requires_grad_(True)
    z = atlas.curl_fn(u, v, fvm)
    (z * zb).sum().backward()
    au, av = fvm.curl_adjoint(zb)
    torch.cuda.synchronize()
    assert torch.equal(u.grad, au) and torch.equal(v.grad, av)
