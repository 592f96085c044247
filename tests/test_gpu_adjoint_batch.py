"""GPU tests of the adjoint kernels behind torch.autograd, the persistent
batched launch (with CUDA-graph capture) and the autotuner."""
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


def test_dot_product_test_o320_137_fp64(torch, pfvm):
    """<G x, y> = <x, G^T y> and <D (u,v), d> = <(u,v), D^T d> to 1e-12 with
    seeded N(0,1) fields, FP64, through the adjoint kernels."""
    fvm = pfvm(320)
    V, L, ld = fvm.nnodes, 137, 138
    gen = torch.Generator(device="cuda")
    gen.manual_seed(1)
    rnd = lambda: torch.randn((V, ld), generator=gen, device="cuda", dtype=torch.float64)
    x, y0, y1, u, v, d = (rnd() for _ in range(6))
    gx, gy = fvm.gradient(x, L)
    gt = fvm.gradient_adjoint(y0, y1, L)
    lhs = (gx[:, :L] * y0[:, :L]).sum() + (gy[:, :L] * y1[:, :L]).sum()
    rhs = (x[:, :L] * gt[:, :L]).sum()
    assert abs((lhs - rhs).item()) <= 1e-12 * abs(lhs.item())
    dv = fvm.divergence(u, v, L)
    du_, dv_ = fvm.divergence_adjoint(d, L)
    lhs = (dv[:, :L] * d[:, :L]).sum()
    rhs = (u[:, :L] * du_[:, :L]).sum() + (v[:, :L] * dv_[:, :L]).sum()
    assert abs((lhs - rhs).item()) <= 1e-12 * abs(lhs.item())


def test_autograd_finite_differences_o16x4_fp64(torch, pfvm):
    """J(f) = sum_i V_i |grad f|_i^2 over 4 levels through GradientFn; the
    gradient from the adjoint kernel agrees with central differences (eps 1e-6,
    FP64; J is quadratic so only rounding separates them)."""
    from paper_1908_07038_gb300 import atlas
    fvm = pfvm(16)
    V = torch.from_numpy(fvm.arrays()["V"]).cuda()
    g = fvm.grid.arrays()
    f0 = synthetic.level_scalar(g["lon"], g["lat_node"], 4)
    f = torch.from_numpy(f0).cuda().requires_grad_(True)

    def J(ff):
        gx, gy = atlas.gradient_fn(ff, fvm)
        return (V[:, None] * (gx * gx + gy * gy)).sum()

    J(f).backward()
    grad = f.grad.cpu().numpy()
    eps = 1e-6
    with torch.no_grad():
        j0 = J(f).item()
        roundoff = 64 * np.finfo(float).eps * abs(j0) / (2 * eps)
        for i, k in [(0, 0), (7, 1), (fvm.nnodes // 2, 2), (fvm.nnodes - 1, 3), (333, 3)]:
            fp = f.detach().clone(); fp[i, k] += eps
            fm = f.detach().clone(); fm[i, k] -= eps
            fd = (J(fp).item() - J(fm).item()) / (2 * eps)
            assert abs(fd - grad[i, k]) <= 1e-9 * abs(grad[i, k]) + roundoff


def test_divergence_autograd_matches_adjoint(torch, pfvm):
    from paper_1908_07038_gb300 import atlas
    fvm = pfvm(32)
    gen = torch.Generator(device="cuda")
    gen.manual_seed(2)
    u = torch.randn((fvm.nnodes, 6), generator=gen, device="cuda", dtype=torch.float64, requires_grad=True)
    v = torch.randn((fvm.nnodes, 6), generator=gen, device="cuda", dtype=torch.float64, requires_grad=True)
    w = torch.randn((fvm.nnodes, 6), generator=gen, device="cuda", dtype=torch.float64)
    (atlas.divergence_fn(u, v, fvm) * w).sum().backward()
    du, dv = fvm.divergence_adjoint(w.contiguous())
    torch.cuda.synchronize()
    assert torch.equal(u.grad, du) and torch.equal(v.grad, dv)


@pytest.fixture(scope="module")
def batch_jobs(torch, pfvm):
    from paper_1908_07038_gb300 import batch
    fvms = {N: pfvm(N) for N in batch.GRIDS}
    return batch.make_jobs(fvms, 24, seed=3)


@pytest.mark.parametrize("plain_waves", [-1, 0, 8, 1])
def test_batched_launch_equals_plain_launches(torch, batch_jobs, plain_waves):
    """24 fields (grids O80..O640, levels {1,60,91,137}) in one persistent
    launch (plain_waves -1) give bitwise the results of 24 separate launches;
    the CUDA-graph replay does too.  With plain_waves, the fields of that
    many full waves run as plain launches inside the batched call (0: the
    default, 4 waves; 8: O160 x 137 and up; 1: nearly all), with the same
    results."""
    from paper_1908_07038_gb300 import batch
    jobs = batch_jobs
    b = batch.Batch(jobs, tune=dict(plain_waves=plain_waves))
    if plain_waves in (-1, 0):
        assert b.tiles > 0
    b.launch()
    torch.cuda.synchronize()
    got = [[o.clone() for o in j["outs"]] for j in jobs]
    for j in jobs:
        for o in j["outs"]:
            o.zero_()
    batch.plain(jobs)
    torch.cuda.synchronize()
    for j, gs in zip(jobs, got):
        for o, gcopy in zip(j["outs"], gs):
            assert torch.equal(o[:, :j["nlev"]], gcopy[:, :j["nlev"]])
    for j in jobs:
        for o in j["outs"]:
            o.zero_()
    b.capture()
    for j in jobs:
        for o in j["outs"]:
            o.zero_()
    b.replay()
    torch.cuda.synchronize()
    for j, gs in zip(jobs, got):
        for o, gcopy in zip(j["outs"], gs):
            assert torch.equal(o[:, :j["nlev"]], gcopy[:, :j["nlev"]])
    b.close()


def test_batched_results_match_oracle(torch, batch_jobs, omesh):
    from paper_1908_07038_gb300 import batch
    b = batch.Batch(batch_jobs, tune=dict(tile_items=2048, threads=256))
    b.launch()
    torch.cuda.synchronize()
    checked = 0
    for j in batch_jobs:
        if j["N"] != 80 or checked >= 3:
            continue
        om = omesh(80)
        L = j["nlev"]
        ins = [t[:, :L].cpu().numpy() for t in j["ins"]]
        if j["op"] == "gradient":
            want = om.gradient(ins[0])
        else:
            want = (om.divergence(ins[0], ins[1]),)
        for o, w in zip(j["outs"], want):
            got = o[:, :L].double().cpu().numpy()
            assert np.max(np.abs(got - w)) <= 1e-5 * np.max(np.abs(w))
        checked += 1
    b.close()
    assert checked > 0


def test_autotuner_installs_a_shape_and_keeps_results(torch, product, tmp_path, monkeypatch):
    atlas, _ = product
    from paper_1908_07038_gb300 import tune
    monkeypatch.setenv("ATLASGB_TUNE_CACHE", str(tmp_path / "tune.json"))
    fvm = atlas.build_fvm(64)
    gen = torch.Generator(device="cuda")
    gen.manual_seed(5)
    f = torch.randn((fvm.nnodes, 140), generator=gen, device="cuda")
    ref = [t.clone() for t in fvm.gradient(f, 137)]
    best = tune.tune_fvm(fvm, nlev=137, ld=140, ops=("gradient", "laplacian"), reps=2)
    assert set(best) == {"gradient", "laplacian"} and best["gradient"]["ms"] > 0
    gx, gy = fvm.gradient(f, 137)
    torch.cuda.synchronize()
    assert torch.equal(gx[:, :137], ref[0][:, :137]) and torch.equal(gy[:, :137], ref[1][:, :137])
    assert (tmp_path / "tune.json").exists()
    best2 = tune.tune_fvm(fvm, nlev=137, ld=140, ops=("gradient",), reps=2)  # from the cache
    assert best2["gradient"]["vec"] == best["gradient"]["vec"]
