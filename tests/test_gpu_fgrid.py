"""GPU parity of every operator on the regular Gaussian grid F<N> with the
FP64 oracle's F-grid mesh (same seeded inputs; tolerances FP64 1e-13,
FP32 1e-5 relative max-norm per output component)."""
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
    den = np.max(np.abs(b))
    return np.max(np.abs(np.asarray(a, np.float64) - b)) / (den if den > 0 else 1.0)


@pytest.mark.parametrize("N,nlev,ld,dt", [(8, 1, 2, np.float64), (8, 5, 8, np.float32), (40, 137, 138, np.float64),
                                          (40, 137, 140, np.float32)])
def test_all_operators_on_f_grids(torch, product, N, nlev, ld, dt):
    from oracle.oracle import Mesh
    atlas = product[0]
    fvm = atlas.build_fvm(N, regular=True)
    om = Mesh(N, R, regular=True)
    g = om.grid()
    f = synthetic.level_scalar(g["lon"], g["lat_node"], nlev, dt)
    u, v = synthetic.level_vector(g["lon"], g["lat_node"], nlev, dt)
    tf, tu, tv = (torch.from_numpy(synthetic.padded(x, ld)).cuda() for x in (f, u, v))
    got = {}
    got["gx"], got["gy"] = fvm.gradient(tf, nlev)
    got["div"] = fvm.divergence(tu, tv, nlev)
    got["lap"] = fvm.laplacian(tf, nlev)
    got["ga"] = fvm.gradient_adjoint(tu, tv, nlev)
    got["du"], got["dv"] = fvm.divergence_adjoint(tf, nlev)
    got["curl"] = fvm.curl(tu, tv, nlev)
    got["ux"], got["uy"], got["vx"], got["vy"] = fvm.vector_gradient(tu, tv, nlev)
    torch.cuda.synchronize()
    want = {}
    want["gx"], want["gy"] = om.gradient(f, nlev)
    want["div"] = om.divergence(u, v, nlev)
    want["lap"] = om.laplacian(f, nlev)
    want["ga"] = om.gradient_adjoint(u, v, nlev)
    want["du"], want["dv"] = om.divergence_adjoint(f, nlev)
    want["curl"] = om.curl(u, v, nlev)
    want["ux"], want["uy"], want["vx"], want["vy"] = om.vector_gradient(u, v, nlev)
    tol = 1e-13 if dt == np.float64 else 1e-5
    worst = {k: _relmax(got[k][:, :nlev].double().cpu().numpy(), want[k]) for k in want}
    assert max(worst.values()) <= tol, worst
