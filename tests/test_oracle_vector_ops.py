"""Pins of the oracle's curl (vertical vorticity) and vector gradient.

Closed forms (checked symbolically when written):
* solid-body rotation about an axis tilted by alpha,
  (u, v) = (cos lat cos a + sin lat cos lon sin a, -sin lon sin a),
  has vorticity 2 (sin lat cos a - cos lat cos lon sin a) / R;
* the non-divergent flow of a streamfunction psi,
  (u, v) = (-d_lat psi / R, d_lon psi / (R cos lat)), has vorticity
  Laplacian(psi), which for a spherical harmonic Y_l^m is -l(l+1)/R^2 Y;
* the projection onto the sphere of the constant Cartesian vector e_x,
  (u, v) = (-sin lon, -sin lat cos lon), is a gradient field (its curl is 0);
  its components have the gradients (-cos lon / (R cos lat), 0) and
  (sin lat sin lon / (R cos lat), -cos lat cos lon / R).
Invariant: the circulations of all cells add up to zero over the closed
sphere (every regular face is shared by two cells with opposite normals).
Convergence is asserted on the volume-weighted L2 error over |lat| < 60 deg,
as for the scalar operators.
"""
import numpy as np
import pytest

R = 6371220.0


def _l2(V, e, mask):
    return np.sqrt(np.sum(V[mask] * e[mask] ** 2) / np.sum(V[mask]))


def _slopes(errs):
    return [np.log2(errs[i] / errs[i + 1]) for i in range(len(errs) - 1)]


def _bulk_order_ok(errs):
    s = _slopes(errs)
    return min(s) >= 1.2 and s[-1] >= 1.35


def _geo(m):
    g = m.grid()
    return g["lon"], g["lat_node"], m.dual()["V"], g["pl"]


@pytest.mark.parametrize("alpha", [0.0, np.pi / 4])
def test_curl_of_solid_body_rotation(omesh, alpha):
    errs = []
    for N in (16, 32, 64):
        m = omesh(N)
        lam, phi, V, _ = _geo(m)
        u = np.cos(phi) * np.cos(alpha) + np.sin(phi) * np.cos(lam) * np.sin(alpha)
        v = -np.sin(lam) * np.sin(alpha)
        z = m.curl(u[:, None], v[:, None])[:, 0] * R
        want = 2 * (np.sin(phi) * np.cos(alpha) - np.cos(phi) * np.cos(lam) * np.sin(alpha))
        errs.append(_l2(V, z - want, np.abs(phi) < np.radians(60)))
    assert _bulk_order_ok(errs), errs


def _sph(l, mm, lam, phi):
    from scipy.special import lpmv
    P = lpmv(abs(mm), l, np.sin(phi))
    return P * (np.cos(mm * lam) if mm >= 0 else np.sin(-mm * lam))


@pytest.mark.parametrize("l,mm", [(2, 1), (3, -2), (4, 3)])
def test_curl_of_streamfunction_flow_is_its_laplacian(omesh, l, mm):
    """(u, v) from psi = Y_l^m (derivatives by central differences of the
    closed form, step 1e-6 rad): curl -> -l(l+1)/R^2 psi; the relative bulk
    error falls monotonically and is below 5% at O64."""
    rel = []
    h = 1e-6
    for N in (16, 32, 64):
        m = omesh(N)
        lam, phi, V, _ = _geo(m)
        dpsi_dlat = (_sph(l, mm, lam, phi + h) - _sph(l, mm, lam, phi - h)) / (2 * h)
        dpsi_dlon = (_sph(l, mm, lam + h, phi) - _sph(l, mm, lam - h, phi)) / (2 * h)
        u = -dpsi_dlat  # in units of 1/R
        v = dpsi_dlon / np.cos(phi)
        z = m.curl(u[:, None], v[:, None])[:, 0] * R
        want = -l * (l + 1) * _sph(l, mm, lam, phi)
        bulk = np.abs(phi) < np.radians(60)
        rel.append(_l2(V, z - want, bulk) / _l2(V, want, bulk))
    assert rel[0] > rel[1] > rel[2], rel
    assert rel[2] < 0.05, rel


@pytest.mark.parametrize("N", [16, 32])
def test_total_circulation_vanishes(omesh, N):
    m = omesh(N)
    rng = np.random.default_rng(7)
    u = rng.standard_normal((m.nnodes, 3))
    v = rng.standard_normal((m.nnodes, 3))
    V = m.dual()["V"]
    z = m.curl(u, v)
    for k in range(3):
        t = V * z[:, k]
        assert abs(np.sum(t)) <= 1e-12 * np.sum(np.abs(t))


def test_curl_of_gradient_field_converges_to_zero(omesh):
    """e_x projected on the sphere is R grad(cos lat cos lon): its discrete curl
    tends to 0 in the bulk (first order: the scheme's curl and gradient are
    not mimetic)."""
    errs = []
    for N in (16, 32, 64):
        m = omesh(N)
        lam, phi, _, _ = _geo(m)
        z = m.curl(-np.sin(lam)[:, None], (-np.sin(phi) * np.cos(lam))[:, None])[:, 0] * R
        errs.append(np.max(np.abs(z[np.abs(phi) < np.radians(60)])))
    assert errs[0] > errs[1] > errs[2] and errs[2] < 0.01, errs


def test_curl_agrees_with_divergence_of_the_rotated_field(omesh):
    """The circulation of (u, v) is the flux of (v, -u cos lat), the field the
    divergence integrates for the vector (v, -u): curl(u, v) = div(v, -u)
    with the same face means.  curl_node and div_node are separate code, so
    this cross-checks signs and operand order."""
    m = omesh(16)
    rng = np.random.default_rng(3)
    u = rng.standard_normal((m.nnodes, 2))
    v = rng.standard_normal((m.nnodes, 2))
    z = m.curl(u, v)
    d = m.divergence(v, -u)
    assert np.max(np.abs(z - d)) <= 1e-13 * np.max(np.abs(d))


def test_vector_gradient_converges(omesh):
    errs = {c: [] for c in range(4)}
    for N in (16, 32, 64):
        m = omesh(N)
        lam, phi, V, _ = _geo(m)
        u = -np.sin(lam)
        v = -np.sin(phi) * np.cos(lam)
        out = m.vector_gradient(u[:, None], v[:, None])
        want = (-np.cos(lam) / np.cos(phi), 0 * lam, np.sin(phi) * np.sin(lam) / np.cos(phi),
                -np.cos(phi) * np.cos(lam))
        bulk = np.abs(phi) < np.radians(60)
        for c in range(4):
            errs[c].append(_l2(V, out[c][:, 0] * R - want[c], bulk))
    # the d_lat u component (exact value 0) starts at first order (O16 -> O32,
    # slope 1.06) before reaching the scheme's bulk rate: assert the mean
    # order over O16 -> O64 and the last step
    for c in range(4):
        s = _slopes(errs[c])
        assert np.mean(s) >= 1.2 and s[-1] >= 1.35, (c, errs[c])


def test_vector_gradient_reverses_the_antipode_on_pole_faces(omesh):
    """u = -sin lon (e_x's east component) has d_lat u = 0.  On the polar rows
    the vector rule's pole faces see the antipode's component reversed
    (face value u_i) and the error stays below 0.2/R; the scalar gradient of
    the same numbers averages u with -u there (face value 0) and is off by
    about |u|/(R dlat), more than 50 times as much.  Off the polar rows both
    are the same arithmetic, bitwise."""
    for N in (16, 32):
        m = omesh(N)
        lam, phi, _, pl = _geo(m)
        u = (-np.sin(lam))[:, None]
        v = (-np.sin(phi) * np.cos(lam))[:, None]
        ux, uy, vx, vy = m.vector_gradient(u, v)
        sx, sy = m.gradient(u)
        polar = np.zeros(m.nnodes, bool)
        polar[:pl[0]] = True
        polar[-pl[-1]:] = True
        vec_err = np.max(np.abs(uy[polar, 0])) * R
        sca_err = np.max(np.abs(sy[polar, 0])) * R
        assert vec_err < 0.2 and sca_err > 50 * vec_err, (vec_err, sca_err)
        assert np.array_equal(ux[~polar], sx[~polar]) and np.array_equal(uy[~polar], sy[~polar])
        tx, ty = m.gradient(v)
        assert np.array_equal(vx[~polar], tx[~polar]) and np.array_equal(vy[~polar], ty[~polar])


def test_vector_ops_node_subsets_and_float32(omesh):
    m = omesh(16)
    rng = np.random.default_rng(5)
    u = rng.standard_normal((m.nnodes, 3)).astype(np.float32)
    v = rng.standard_normal((m.nnodes, 3)).astype(np.float32)
    nodes = np.array([0, 5, m.nnodes // 2, m.nnodes - 1])
    z = m.curl(u, v)
    assert np.array_equal(m.curl(u, v, nodes=nodes), z[nodes])
    assert np.array_equal(z, m.curl(u.astype(np.float64), v.astype(np.float64)))
    full = m.vector_gradient(u, v)
    sub = m.vector_gradient(u, v, nodes=nodes)
    for a, b in zip(full, sub):
        assert np.array_equal(a[nodes], b)


# ------------------------------------------------------------ curl adjoint
def test_curl_adjoint_is_the_dense_transpose_on_o2(omesh):
    """O2 brute force: the curl's matrix, column by column from orc_curl on
    unit fields, transposed and applied, against curl_adjoint."""
    m = omesh(2)
    V = m.nnodes
    C = np.zeros((V, 2 * V))
    for k in range(V):
        e = np.zeros((V, 1))
        e[k] = 1.0
        C[:, k] = m.curl(e, np.zeros((V, 1)))[:, 0]
        C[:, V + k] = m.curl(np.zeros((V, 1)), e)[:, 0]
    rng = np.random.default_rng(21)
    z = rng.standard_normal((V, 3))
    xu, xv = m.curl_adjoint(z)
    want = C.T @ z
    scale = np.max(np.abs(want))
    assert np.max(np.abs(xu - want[:V])) <= 1e-13 * scale
    assert np.max(np.abs(xv - want[V:])) <= 1e-13 * scale


def test_curl_adjoint_dot_product_o16(omesh):
    """<C (u, v), z> = <(u, v), C^T z> to 1e-12 with N(0,1) fields."""
    m = omesh(16)
    rng = np.random.default_rng(22)
    u, v, z = (rng.standard_normal((m.nnodes, 4)) for _ in range(3))
    lhs = np.sum(m.curl(u, v) * z)
    xu, xv = m.curl_adjoint(z)
    rhs = np.sum(u * xu) + np.sum(v * xv)
    assert abs(lhs - rhs) <= 1e-12 * (np.sum(np.abs(m.curl(u, v) * z)))


def test_curl_adjoint_node_subset(omesh):
    m = omesh(8)
    rng = np.random.default_rng(23)
    z = rng.standard_normal((m.nnodes, 2))
    nodes = np.array([0, 5, 17, m.nnodes - 1], dtype=np.int64)
    fu, fv = m.curl_adjoint(z)
    su, sv = m.curl_adjoint(z, nodes=nodes)
    assert np.array_equal(su, fu[nodes]) and np.array_equal(sv, fv[nodes])
