"""GPU parity: the CUDA kernels (through the C ABI) against the FP64 oracle on
the same seeded inputs.

Tolerances (relative max-norm per output component, ||a - b||_inf /
||b||_inf): FP64 path 1e-13, FP32 path 1e-5 (both as required for this
path), BF16 storage 2e-2 (output rounding to 8 significant bits).  The FP32
and BF16 paths are compared with the oracle fed the same rounded inputs,
upcast exactly.  Sizes: full comparisons on O2..O80 with up to 137 levels and
ragged tails; O320 x 137 (the FP32/FP64 comparison workload) and O1280 x 137
(the benchmark workload) on sampled nodes that include every polar-row node
and every row's first and last node.
"""
import numpy as np
import pytest

import synthetic

pytestmark = pytest.mark.gpu

R = 6371220.0


@pytest.fixture(scope="module")
def torch():
    t = pytest.importorskip("torch")
    if not t.cuda.is_available():
        pytest.skip("no CUDA device")
    return t


def _relmax(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    den = np.max(np.abs(b))
    return np.max(np.abs(a - b)) / (den if den > 0 else 1.0)


def _dev(torch, x, ld=None, dtype=None):
    """numpy [V][nlev] -> CUDA tensor [V][ld] (zero padding)."""
    x = np.asarray(x)
    if ld is not None and ld != x.shape[1]:
        x = synthetic.padded(x, ld)
    t = torch.from_numpy(np.ascontiguousarray(x))
    if dtype is not None:
        t = t.to(dtype)
    return t.cuda()


def _host(t, nlev):
    return t[:, :nlev].double().cpu().numpy()


TOL = {"f64": 1e-13, "f32": 1e-5, "bf16": 2e-2}


def _all_ops(torch, fvm, f, u, v, nlev):
    gx, gy = fvm.gradient(f, nlev)
    d = fvm.divergence(u, v, nlev)
    lap = fvm.laplacian(f, nlev)
    ga = fvm.gradient_adjoint(u, v, nlev)
    da_u, da_v = fvm.divergence_adjoint(f, nlev)
    torch.cuda.synchronize()
    return dict(gx=gx, gy=gy, div=d, lap=lap, ga=ga, da_u=da_u, da_v=da_v)


def _oracle_all(om, f, u, v, nlev, nodes=None):
    gx, gy = om.gradient(f, nlev, nodes=nodes)
    d = om.divergence(u, v, nlev, nodes=nodes)
    lap = om.laplacian(f, nlev, nodes=nodes)
    ga = om.gradient_adjoint(u, v, nlev, nodes=nodes)
    da_u, da_v = om.divergence_adjoint(f, nlev, nodes=nodes)
    return dict(gx=gx, gy=gy, div=d, lap=lap, ga=ga, da_u=da_u, da_v=da_v)


# --------------------------------------------------------------------- cfg0
def test_cfg0_o32_fp64(torch, pfvm, omesh):
    """O32, one level, FP64: scalar through gradient and Laplacian, vector
    through divergence, plus the adjoints, within 1e-13 of the oracle."""
    fvm, om = pfvm(32), omesh(32)
    g = om.grid()
    f = synthetic.level_scalar(g["lon"], g["lat_node"], 1)
    u, v = synthetic.level_vector(g["lon"], g["lat_node"], 1)
    got = _all_ops(torch, fvm, _dev(torch, f), _dev(torch, u), _dev(torch, v), 1)
    want = _oracle_all(om, f, u, v, 1)
    for k in want:
        assert _relmax(_host(got[k], 1), want[k]) <= TOL["f64"], k


@pytest.mark.parametrize("N,nlev,ld", [(1, 1, 1), (2, 5, 5), (2, 5, 8), (8, 137, 137), (8, 137, 140),
                                       (16, 3, 4), (32, 9, 12)])
def test_fp32_ragged_levels_and_layouts(torch, pfvm, omesh, N, nlev, ld):
    """FP32 path for every op on ragged level counts and both aligned (vector)
    and unaligned (element-wise) leading dimensions."""
    fvm, om = pfvm(N), omesh(N)
    g = om.grid()
    f = synthetic.level_scalar(g["lon"], g["lat_node"], nlev, np.float32)
    u, v = synthetic.level_vector(g["lon"], g["lat_node"], nlev, np.float32, noise=True)
    got = _all_ops(torch, fvm, _dev(torch, f, ld), _dev(torch, u, ld), _dev(torch, v, ld), nlev)
    want = _oracle_all(om, f, u, v, nlev)
    for k in want:
        assert _relmax(_host(got[k], nlev), want[k]) <= TOL["f32"], (k, N, nlev, ld)
    # padding levels of the outputs: zero up to the end of the last vector
    # (when ld is a multiple of the 4-level vector), never written beyond
    if ld > nlev:
        out = torch.full((fvm.nnodes, ld), 7.0, device="cuda")
        gy = torch.full_like(out, 7.0)
        fvm.gradient(_dev(torch, f, ld), nlev, out=(out, gy))
        torch.cuda.synchronize()
        end = (nlev + 3) // 4 * 4 if ld % 4 == 0 else nlev
        for t in (out, gy):
            assert torch.all(t[:, nlev:end] == 0.0).item() and torch.all(t[:, end:] == 7.0).item()


def test_fp64_and_fp32_o80_137(torch, pfvm, omesh):
    """Full-field comparison on O80 x 137 (28480 nodes, several thousand
    blocks and a ragged level tail) in FP64 and FP32."""
    fvm, om = pfvm(80), omesh(80)
    g = om.grid()
    nlev = 137
    f = synthetic.level_scalar(g["lon"], g["lat_node"], nlev)
    u, v = synthetic.level_vector(g["lon"], g["lat_node"], nlev)
    got = _all_ops(torch, fvm, _dev(torch, f, 138), _dev(torch, u, 138), _dev(torch, v, 138), nlev)
    want = _oracle_all(om, f, u, v, nlev)
    for k in want:
        assert _relmax(_host(got[k], nlev), want[k]) <= TOL["f64"], k
    f32, u32, v32 = (x.astype(np.float32) for x in (f, u, v))
    got = _all_ops(torch, fvm, _dev(torch, f32, 140), _dev(torch, u32, 140), _dev(torch, v32, 140), nlev)
    want = _oracle_all(om, f32, u32, v32, nlev)
    for k in want:
        assert _relmax(_host(got[k], nlev), want[k]) <= TOL["f32"], k


def test_bf16_storage_o80(torch, pfvm, omesh):
    """BF16 storage, FP32 arithmetic: against the oracle on the bf16-rounded
    inputs; the error is the output rounding (2^-8 relative)."""
    fvm, om = pfvm(80), omesh(80)
    g = om.grid()
    nlev = 60
    f = synthetic.level_scalar(g["lon"], g["lat_node"], nlev)
    u, v = synthetic.level_vector(g["lon"], g["lat_node"], nlev)
    tf, tu, tv = (_dev(torch, x, 64, torch.bfloat16) for x in (f, u, v))
    fr, ur, vr = (t[:, :nlev].double().cpu().numpy() for t in (tf, tu, tv))
    got = _all_ops(torch, fvm, tf, tu, tv, nlev)
    want = _oracle_all(om, fr, ur, vr, nlev)
    for k in want:
        assert _relmax(_host(got[k], nlev), want[k]) <= TOL["bf16"], k


def test_edge_based_two_pass_forms(torch, pfvm, omesh):
    """Edge-flux + node-gather kernels (gradient, divergence, two-pass
    Laplacian) in FP64 and FP32 against the oracle."""
    fvm, om = pfvm(80), omesh(80)
    g = om.grid()
    nlev = 91
    f = synthetic.level_scalar(g["lon"], g["lat_node"], nlev)
    u, v = synthetic.level_vector(g["lon"], g["lat_node"], nlev)
    want_g = om.gradient(f)
    want_d = om.divergence(u, v)
    want_l = om.laplacian(f)
    for ld, tol, cast in ((92, TOL["f64"], np.float64), (92, TOL["f32"], np.float32)):
        fc, uc, vc = (x.astype(cast) for x in (f, u, v))
        if cast is np.float32:
            want_g = om.gradient(fc)
            want_d = om.divergence(uc, vc)
            want_l = om.laplacian(fc)
        tf, tu, tv = (_dev(torch, x, ld) for x in (fc, uc, vc))
        gx, gy = fvm.gradient_edges(tf, nlev)
        d = fvm.divergence_edges(tu, tv, nlev)
        lap = fvm.laplacian_edges(tf, nlev)
        torch.cuda.synchronize()
        assert _relmax(_host(gx, nlev), want_g[0]) <= tol
        assert _relmax(_host(gy, nlev), want_g[1]) <= tol
        assert _relmax(_host(d, nlev), want_d) <= tol
        assert _relmax(_host(lap, nlev), want_l) <= tol


def test_gradient_of_constant_is_exactly_zero_on_gpu(torch, pfvm):
    fvm = pfvm(32)
    for dt in (torch.float32, torch.float64, torch.bfloat16):
        f = torch.full((fvm.nnodes, 8), 2.5, dtype=dt, device="cuda")
        gx, gy = fvm.gradient(f)
        gxe, gye = fvm.gradient_edges(f) if dt != torch.bfloat16 else (gx, gy)
        torch.cuda.synchronize()
        for t in (gx, gy, gxe, gye):
            assert torch.count_nonzero(t).item() == 0


def test_deterministic_and_launch_shape_independent(torch, product):
    """No atomics: repeated runs and every levels-per-thread / block / tile
    shape give bitwise identical results."""
    atlas, _ = product
    fvm = atlas.build_fvm(32)
    rng = np.random.default_rng(11)
    f = _dev(torch, rng.standard_normal((fvm.nnodes, 40)).astype(np.float32))
    fb = f.to(torch.bfloat16)
    ref = [t.clone() for t in fvm.gradient(f)]
    lref = fvm.laplacian(f).clone()
    bref = [t.clone() for t in fvm.gradient(fb)]
    for vec, batch, threads, bps, tile in ((1, 3, 128, 2, 1), (2, 6, 512, 1, 4), (4, 3, 256, 0, 64),
                                           (4, 6, 64, 3, 4096), (4, 3, 96, 0, 7), (8, 3, 128, 0, 8)):
        fvm.set_launch("gradient", vec, batch, threads, bps, tile)
        fvm.set_launch("laplacian", vec, batch, threads, bps, tile)
        gx, gy = fvm.gradient(f)
        lap = fvm.laplacian(f)
        bx, by = fvm.gradient(fb)
        torch.cuda.synchronize()
        assert torch.equal(gx, ref[0]) and torch.equal(gy, ref[1]) and torch.equal(lap, lref)
        assert torch.equal(bx, bref[0]) and torch.equal(by, bref[1])


def test_empty_and_offset_views(torch, pfvm, omesh):
    fvm, om = pfvm(16), omesh(16)
    f = torch.zeros((fvm.nnodes, 4), device="cuda")
    fvm.gradient(f, 0)  # zero levels: a no-op
    torch.cuda.synchronize()
    # a field starting 1 element into its buffer: vector loads are not
    # aligned, the element-wise path must take over
    rng = np.random.default_rng(12)
    x = rng.standard_normal((fvm.nnodes, 9))
    buf = torch.zeros(fvm.nnodes * 9 + 1, dtype=torch.float64, device="cuda")
    view = buf[1:].view(fvm.nnodes, 9)
    view.copy_(torch.from_numpy(x))
    ox = torch.empty_like(view)
    oy = torch.empty_like(view)
    fvm.gradient(view, out=(ox, oy))
    torch.cuda.synchronize()
    wx, wy = om.gradient(x)
    assert _relmax(ox.cpu().numpy(), wx) <= TOL["f64"] and _relmax(oy.cpu().numpy(), wy) <= TOL["f64"]


# ------------------------------------------------------ large sampled cases
def _sampled_case(torch, pfvm, omesh, N, nlev, count, dtype_np, tol, ld):
    fvm, om = pfvm(N), omesh(N)
    g = om.grid()
    pl = g["pl"]
    off = np.concatenate([[0], np.cumsum(pl)])
    nodes = synthetic.sample_nodes(om.nnodes, off, count)
    f = synthetic.level_scalar(g["lon"], g["lat_node"], nlev, dtype_np)
    u, v = synthetic.level_vector(g["lon"], g["lat_node"], nlev, dtype_np)
    tf, tu, tv = (_dev(torch, x, ld) for x in (f, u, v))
    got = _all_ops(torch, fvm, tf, tu, tv, nlev)
    idx = torch.from_numpy(nodes).cuda()
    want = _oracle_all(om, f, u, v, nlev, nodes=nodes)
    worst = {}
    for k in want:
        a = got[k].index_select(0, idx)[:, :nlev].double().cpu().numpy()
        worst[k] = _relmax(a, want[k])
    del tf, tu, tv, got
    torch.cuda.empty_cache()
    return worst


def test_o320_137_fp32_and_fp64_sampled(torch, pfvm, omesh):
    w32 = _sampled_case(torch, pfvm, omesh, 320, 137, 20000, np.float32, TOL["f32"], 140)
    assert max(w32.values()) <= TOL["f32"], w32
    w64 = _sampled_case(torch, pfvm, omesh, 320, 137, 20000, np.float64, TOL["f64"], 138)
    assert max(w64.values()) <= TOL["f64"], w64


def test_o1280_137_fp32_sampled(torch, pfvm, omesh):
    """The benchmark workload (O1280 x 137, FP32, ld = 140, the launch shape
    the benchmark times) on sampled nodes."""
    w32 = _sampled_case(torch, pfvm, omesh, 1280, 137, 6000, np.float32, TOL["f32"], 140)
    assert max(w32.values()) <= TOL["f32"], w32


def test_o1280_137_fp64_sampled(torch, pfvm, omesh):
    w64 = _sampled_case(torch, pfvm, omesh, 1280, 137, 3000, np.float64, TOL["f64"], 138)
    assert max(w64.values()) <= TOL["f64"], w64


def test_o1280_64bit_element_offsets(torch, pfvm, omesh):
    """O1280 with ld = 328: nnodes * ld = 2.16e9 elements, past 2^31, so the
    per-node kernels take their 64-bit offset form (the tiles do not fit in
    shared memory at this ld, so every operator runs per node); 8 levels,
    sampled nodes against the oracle."""
    fvm, om = pfvm(1280), omesh(1280)
    g = om.grid()
    V, nlev, ld = om.nnodes, 8, 328
    assert V * ld >= 2 ** 31
    off = np.concatenate([[0], np.cumsum(g["pl"])])
    nodes = synthetic.sample_nodes(V, off, 4000)
    f = synthetic.level_scalar(g["lon"], g["lat_node"], nlev, np.float32)
    u, v = synthetic.level_vector(g["lon"], g["lat_node"], nlev, np.float32)
    assert fvm.tile_info("gradient", nlev, ld)["stages"] == 0  # per node at this ld
    big = []
    for x in (f, u, v):
        t = torch.zeros((V, ld), device="cuda")
        t[:, :nlev] = torch.from_numpy(x).cuda()
        big.append(t)
    tf, tu, tv = big
    idx = torch.from_numpy(nodes).cuda()
    pick = lambda t: t.index_select(0, idx)[:, :nlev].double().cpu().numpy()
    gx, gy = fvm.gradient(tf, nlev)
    wx, wy = om.gradient(f, nlev, nodes=nodes)
    assert _relmax(pick(gx), wx) <= TOL["f32"] and _relmax(pick(gy), wy) <= TOL["f32"]
    del gx, gy
    d = fvm.divergence(tu, tv, nlev)
    assert _relmax(pick(d), om.divergence(u, v, nlev, nodes=nodes)) <= TOL["f32"]
    del d
    lap = fvm.laplacian(tf, nlev)
    assert _relmax(pick(lap), om.laplacian(f, nlev, nodes=nodes)) <= TOL["f32"]
    del lap, tf, tu, tv, big
    torch.cuda.empty_cache()
