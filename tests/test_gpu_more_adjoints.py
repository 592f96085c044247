"""GPU: the adjoints of the curl and of the fused Laplacian, as autograd
backward passes built from the hand-written divergence and gradient adjoint
kernels.  Dot-product test <A x, y> = <x, A^T y> in FP64 (1e-12, seeded
N(0,1) fields, O320 x 137 as for the gradient and divergence), and central
finite differences of a quadratic loss (O16 x 4, eps 1e-6, FP64)."""
import numpy as np
import pytest

import synthetic

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    t = pytest.importorskip("torch")
    if not t.cuda.is_available():
        pytest.skip("no CUDA device")
    return t


def test_dot_product_tests_o320_137(torch, pfvm):
    from paper_1908_07038_gb300 import atlas
    fvm = pfvm(320)
    V, L, ld = fvm.nnodes, 137, 138
    gen = torch.Generator(device="cuda")
    gen.manual_seed(5)
    rnd = lambda g=False: torch.randn((V, ld), generator=gen, device="cuda", dtype=torch.float64,  # noqa: E731
                                      requires_grad=g)
    # curl: <curl(u, v), z> = <(u, v), curl^T z>
    u, v, z = rnd(True), rnd(True), rnd()
    c = atlas.curl_fn(u, v, fvm)
    (c[:, :L] * z[:, :L]).sum().backward()
    lhs = (c[:, :L] * z[:, :L]).sum().item()
    rhs = ((u[:, :L] * u.grad[:, :L]).sum() + (v[:, :L] * v.grad[:, :L]).sum()).item()
    assert abs(lhs - rhs) <= 1e-12 * abs(lhs)
    # Laplacian: <L f, y> = <f, L^T y>
    f, y = rnd(True), rnd()
    lap = atlas.laplacian_fn(f, fvm)
    (lap[:, :L] * y[:, :L]).sum().backward()
    lhs = (lap[:, :L] * y[:, :L]).sum().item()
    rhs = (f[:, :L] * f.grad[:, :L]).sum().item()
    assert abs(lhs - rhs) <= 1e-12 * abs(lhs)


@pytest.mark.parametrize("which", ["curl", "laplacian"])
def test_finite_differences_o16x4(torch, pfvm, which):
    from paper_1908_07038_gb300 import atlas
    fvm = pfvm(16)
    Vol = torch.from_numpy(fvm.arrays()["V"]).cuda()
    g = fvm.grid.arrays()
    if which == "curl":
        u0, v0 = synthetic.level_vector(g["lon"], g["lat_node"], 4)
        x = [torch.from_numpy(u0).cuda().requires_grad_(True), torch.from_numpy(v0).cuda().requires_grad_(True)]

        def J(a, b):
            z = atlas.curl_fn(a, b, fvm)
            return (Vol[:, None] * z * z).sum()
    else:
        f0 = synthetic.level_scalar(g["lon"], g["lat_node"], 4)
        x = [torch.from_numpy(f0).cuda().requires_grad_(True)]

        def J(a):
            lap = atlas.laplacian_fn(a, fvm)
            return (Vol[:, None] * lap * lap).sum()

    J(*x).backward()
    grads = [t.grad.cpu().numpy() for t in x]
    eps = 1e-6
    with torch.no_grad():
        j0 = J(*x).item()
        roundoff = 64 * np.finfo(float).eps * abs(j0) / (2 * eps)
        for m, t in enumerate(x):
            for i, k in [(0, 0), (7, 1), (fvm.nnodes // 2, 2), (fvm.nnodes - 1, 3)]:
                xp = [s.detach().clone() for s in x]
                xm = [s.detach().clone() for s in x]
                xp[m][i, k] += eps
                xm[m][i, k] -= eps
                fd = (J(*xp).item() - J(*xm).item()) / (2 * eps)
                assert abs(fd - grads[m][i, k]) <= 1e-8 * abs(grads[m][i, k]) + roundoff, (which, m, i, k)
