"""GPU parity on regional (limited-area) grids: every operator of a regional
fvm runs the same stencil kernels as the global grids, with the tables of
the projection's plane dual.  Against the regional oracle on the same seeded
inputs (FP64 1e-13, FP32 1e-5 relative max-norm per output component), at
small sizes in full and at the 1536 x 1440 x 90 Lambert configuration on
sampled nodes (corners and sides included); plus exact results (constants,
plane-linear fields), odd node counts, partitions, batches, autograd and the
refusal of the edge-based variant."""
import numpy as np
import pytest

import synthetic
from synthetic.regional import DOMAINS, LAM, LAM_NLEV, LAM_NX, LAM_NY

pytestmark = pytest.mark.gpu

R = 6371220.0


@pytest.fixture(scope="module")
def torch():
    t = pytest.importorskip("torch")
    if not t.cuda.is_available():
        pytest.skip("no CUDA device")
    return t


def _relmax(a, b):
    den = np.max(np.abs(b))
    return np.max(np.abs(np.asarray(a, np.float64) - b)) / (den if den > 0 else 1.0)


def _inputs(g, nlev, dt):
    f = synthetic.level_scalar(g["lon"], g["lat_node"], nlev, dt)
    u, v = synthetic.level_vector(g["lon"], g["lat_node"], nlev, dt, noise=True)
    return f, u, v


def _run_all(fvm, tf, tu, tv, nlev):
    got = {}
    got["gx"], got["gy"] = fvm.gradient(tf, nlev)
    got["div"] = fvm.divergence(tu, tv, nlev)
    got["lap"] = fvm.laplacian(tf, nlev)
    got["ga"] = fvm.gradient_adjoint(tu, tv, nlev)
    got["du"], got["dv"] = fvm.divergence_adjoint(tf, nlev)
    got["curl"] = fvm.curl(tu, tv, nlev)
    got["ux"], got["uy"], got["vx"], got["vy"] = fvm.vector_gradient(tu, tv, nlev)
    return got


def _oracle_all(om, f, u, v, nlev, nodes=None):
    want = {}
    want["gx"], want["gy"] = om.gradient(f, nlev, nodes)
    want["div"] = om.divergence(u, v, nlev, nodes)
    want["lap"] = om.laplacian(f, nlev, nodes)
    want["ga"] = om.gradient_adjoint(u, v, nlev, nodes)
    want["du"], want["dv"] = om.divergence_adjoint(f, nlev, nodes)
    want["curl"] = om.curl(u, v, nlev, nodes)
    want["ux"], want["uy"], want["vx"], want["vy"] = om.vector_gradient(u, v, nlev, nodes)
    return want


@pytest.mark.parametrize("name", list(DOMAINS))
@pytest.mark.parametrize("nx,ny,nlev,ld,dt", [(37, 29, 5, 6, np.float64), (61, 47, 9, 12, np.float32),
                                              (2, 2, 1, 2, np.float64), (5, 7, 3, 4, np.float32)])
def test_all_operators_against_the_oracle(torch, product, oracle_mod, name, nx, ny, nlev, ld, dt):
    atlas = product[0]
    proj, kw = DOMAINS[name]
    fvm = atlas.build_fvm_regional(proj, nx, ny, **kw)
    om = oracle_mod.RegionalMesh(proj, nx, ny, **kw)
    g = fvm.grid.arrays()
    if nx * ny < 64:
        # degenerate grids: the smooth recipe is almost linear across them and
        # its Laplacian is ~1e-4 of its terms, so take N(0, 1) fields there
        f, u, v = (synthetic.normal((nx * ny, nlev), 40 + k).astype(dt) for k in range(3))
    else:
        f, u, v = _inputs(g, nlev, dt)
    tf, tu, tv = (torch.from_numpy(synthetic.padded(x, ld)).cuda() for x in (f, u, v))
    got = _run_all(fvm, tf, tu, tv, nlev)
    torch.cuda.synchronize()
    want = _oracle_all(om, f, u, v, nlev)
    tol = 1e-13 if dt == np.float64 else 1e-5
    worst = {k: _relmax(got[k][:, :nlev].double().cpu().numpy(), want[k]) for k in want}
    assert max(worst.values()) <= tol, worst


@pytest.mark.parametrize("name", ["lambert", "rotated"])
def test_bfloat16_storage(torch, product, oracle_mod, name):
    """BF16 storage, FP32 arithmetic: against the oracle fed the same
    BF16-rounded inputs (2e-2 relative max-norm, as on the global grids)."""
    atlas = product[0]
    proj, kw = DOMAINS[name]
    nx, ny, nlev, ld = 61, 47, 9, 16
    fvm = atlas.build_fvm_regional(proj, nx, ny, **kw)
    om = oracle_mod.RegionalMesh(proj, nx, ny, **kw)
    g = fvm.grid.arrays()
    f, u, v = _inputs(g, nlev, np.float64)
    tf, tu, tv = (torch.from_numpy(synthetic.padded(x, ld)).cuda().to(torch.bfloat16) for x in (f, u, v))
    got = _run_all(fvm, tf, tu, tv, nlev)
    torch.cuda.synchronize()
    up = lambda t: t[:, :nlev].float().double().cpu().numpy()  # noqa: E731
    want = _oracle_all(om, up(tf), up(tu), up(tv), nlev)
    worst = {k: _relmax(up(got[k]), want[k]) for k in want}
    assert max(worst.values()) <= 2e-2, worst


def test_exact_results(torch, product):
    """Constants: gradient exactly 0 (difference form); fields linear in the
    plane: gradient, divergence and curl exact to FP64 rounding at every
    node, boundary included."""
    atlas = product[0]
    proj, kw = DOMAINS["lambert"]
    fvm = atlas.build_fvm_regional(proj, 41, 33, **kw)
    g = fvm.grid.arrays()
    c = torch.full((fvm.nnodes, 4), 2.75, dtype=torch.float32, device="cuda")
    gx, gy = fvm.gradient(c, 4)
    torch.cuda.synchronize()
    assert torch.count_nonzero(gx).item() == 0 and torch.count_nonzero(gy).item() == 0
    x, y, hx, hy = g["xy"][:, 0], g["xy"][:, 1], g["scale"][:, 0], g["scale"][:, 1]
    a, b, cc, d = 0.7, -1.3, 0.45, 2.1
    T = lambda z: torch.from_numpy(np.ascontiguousarray(np.repeat(z[:, None], 2, 1))).cuda()  # noqa: E731
    gx, gy = fvm.gradient(T(a * x + b * y), 2)
    dv = fvm.divergence(T((a * x + b * y) / hy), T((cc * x + d * y) / hx), 2)
    cu = fvm.curl(T((a * x + b * y) / hx), T((cc * x + d * y) / hy), 2)
    torch.cuda.synchronize()
    checks = [(gx, a / (R * hx)), (gy, b / (R * hy)), (dv, (a + d) / (R * hx * hy)), (cu, (cc - b) / (R * hx * hy))]
    for t, want in checks:
        assert _relmax(t[:, 0].cpu().numpy(), want) <= 1e-12


def test_lam_configuration_sampled(torch, product, oracle_mod):
    """The 1536 x 1440 x 90 Lambert configuration in FP32 (the benchmark's
    regional workload), checked on 600 sampled nodes: every corner and
    side, and random interior nodes."""
    atlas = product[0]
    proj, kw = LAM
    nx, ny, nlev, ld = LAM_NX, LAM_NY, LAM_NLEV, 92
    fvm = atlas.build_fvm_regional(proj, nx, ny, **kw)
    om = oracle_mod.RegionalMesh(proj, nx, ny, **kw)
    g = fvm.grid.arrays()
    f, u, v = _inputs(g, nlev, np.float32)
    tf, tu, tv = (torch.from_numpy(synthetic.padded(x, ld)).cuda() for x in (f, u, v))
    got = {}
    got["gx"], got["gy"] = fvm.gradient(tf, nlev)
    got["div"] = fvm.divergence(tu, tv, nlev)
    got["lap"] = fvm.laplacian(tf, nlev)
    got["curl"] = fvm.curl(tu, tv, nlev)
    torch.cuda.synchronize()
    rng = np.random.default_rng(5)
    V = nx * ny
    edge = [0, nx - 1, V - nx, V - 1, 1, nx, 2 * nx - 1, V - 2, nx + 1, V - nx - 2]
    sides = np.concatenate([rng.integers(1, nx - 1, 40), (ny - 1) * nx + rng.integers(1, nx - 1, 40),
                            nx * rng.integers(1, ny - 1, 40), nx * rng.integers(1, ny - 1, 40) + nx - 1])
    nodes = np.unique(np.concatenate([edge, sides, rng.integers(0, V, 430)])).astype(np.int64)
    want = {}
    want["gx"], want["gy"] = om.gradient(f, nlev, nodes)
    want["div"] = om.divergence(u, v, nlev, nodes)
    want["lap"] = om.laplacian(f, nlev, nodes)
    want["curl"] = om.curl(u, v, nlev, nodes)
    idx = torch.from_numpy(nodes).cuda()
    worst = {k: _relmax(got[k][idx, :nlev].double().cpu().numpy(), want[k]) for k in want}
    assert max(worst.values()) <= 1e-5, worst


def test_partitions_and_batches_equal_whole_grid(torch, product):
    from paper_1908_07038_gb300 import batch
    from paper_1908_07038_gb300.partition import Partition
    atlas = product[0]
    proj, kw = DOMAINS["rotated"]
    fvm = atlas.build_fvm_regional(proj, 97, 61, **kw)
    nlev, ld = 33, 36
    gen = torch.Generator(device="cuda").manual_seed(9)
    a, b = (torch.randn((fvm.nnodes, ld), generator=gen, device="cuda") for _ in range(2))
    for op, ins, nout in [("gradient", [a], 2), ("divergence", [a, b], 1), ("laplacian", [a], 1), ("curl", [a, b], 1)]:
        want = getattr(fvm, op)(*ins, nlev)
        want = list(want) if isinstance(want, tuple) else [want]
        halo = 2 if op == "laplacian" else 1
        got = [torch.full_like(want[0], float("nan")) for _ in range(nout)]
        for k in range(3):
            p = Partition(fvm, 3, k, halo)
            outs = [torch.empty((p.own_rows, ld), device="cuda") for _ in range(nout)]
            p.apply(op, [p.local_view(x).clone() for x in ins], outs, nlev)
            for g_, o in zip(got, outs):
                g_[p.own0:p.own1] = o
            p.close()
        torch.cuda.synchronize()
        for g_, w in zip(got, want):
            assert torch.equal(g_[:, :nlev], w[:, :nlev]), op
    jobs = [dict(op="gradient", fvm=fvm, ins=(a,), outs=(torch.zeros_like(a), torch.zeros_like(a)), nlev=nlev),
            dict(op="divergence", fvm=fvm, ins=(a, b), outs=(torch.zeros_like(a),), nlev=nlev)]
    bt = batch.Batch(jobs)
    bt.launch()
    ref = [tuple(torch.zeros_like(o) for o in j["outs"]) for j in jobs]
    fvm.gradient(a, nlev, out=ref[0])
    fvm.divergence(a, b, nlev, out=ref[1][0])
    torch.cuda.synchronize()
    for j, r in zip(jobs, ref):
        for o, w in zip(j["outs"], r):
            assert torch.equal(o, w)
    bt.close()


def test_autograd_dot_products(torch, product):
    atlas = product[0]
    proj, kw = DOMAINS["mercator"]
    fvm = atlas.build_fvm_regional(proj, 129, 97, **kw)
    V, L, ld = fvm.nnodes, 7, 8
    gen = torch.Generator(device="cuda").manual_seed(3)
    rnd = lambda g=False: torch.randn((V, ld), generator=gen, device="cuda", dtype=torch.float64,  # noqa: E731
                                      requires_grad=g)
    f, y0, y1 = rnd(True), rnd(), rnd()
    gx, gy = atlas.gradient_fn(f, fvm)
    (gx[:, :L] * y0[:, :L] + gy[:, :L] * y1[:, :L]).sum().backward()
    lhs = (gx[:, :L] * y0[:, :L] + gy[:, :L] * y1[:, :L]).sum().item()
    assert abs(lhs - (f[:, :L] * f.grad[:, :L]).sum().item()) <= 1e-12 * abs(lhs)
    u, v, z = rnd(True), rnd(True), rnd()
    d = atlas.divergence_fn(u, v, fvm)
    (d[:, :L] * z[:, :L]).sum().backward()
    lhs = (d[:, :L] * z[:, :L]).sum().item()
    rhs = ((u[:, :L] * u.grad[:, :L]).sum() + (v[:, :L] * v.grad[:, :L]).sum()).item()
    assert abs(lhs - rhs) <= 1e-12 * abs(lhs)


def test_edge_variant_refuses_regional(torch, product):
    atlas, capi = product
    proj, kw = DOMAINS["lambert"]
    fvm = atlas.build_fvm_regional(proj, 9, 7, **kw)
    f = torch.zeros((fvm.nnodes, 4), device="cuda")
    with pytest.raises(capi.AtlasError) as ei:
        fvm.gradient_edges(f, 4, ws=torch.empty(1 << 20, dtype=torch.uint8, device="cuda"))
    assert "global" in str(ei.value)


@pytest.mark.parametrize("dt,tol", [(np.float64, 1e-13), (np.float32, 1e-5)])
def test_remap_global_field_to_regional_grid(torch, product, omesh, dt, tol):
    """Boundary data for a limited-area grid: an O64 field interpolated to a
    97 x 73 Lambert grid on the GPU, against the oracle's located triangles
    and weights."""
    atlas = product[0]
    proj, kw = DOMAINS["lambert"]
    rg = atlas.Grid.regional(proj, 97, 73, **kw)
    r = atlas.Remap(atlas.Mesh(atlas.Grid(64)), rg)
    om = omesh(64)
    g = om.grid()
    nlev = 9
    f = synthetic.level_scalar(g["lon"], g["lat_node"], nlev, dt)
    out = r.apply(torch.from_numpy(synthetic.padded(f, 12)).cuda(), nlev)
    torch.cuda.synchronize()
    a = rg.arrays()
    want = om.remap(np.stack([a["lon"], a["lat_node"]], 1), f, nlev)
    assert _relmax(out[:, :nlev].double().cpu().numpy(), want) <= tol
    r.close()
