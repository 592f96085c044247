"""Pins of the oracle's nabla operators: exact zeros, conservation, closed
forms and convergence, spherical-harmonic Laplacians, and the adjoints
against brute-force transposes and finite differences.

Operators named in the paper (Sec. 2.3): gradient, divergence, Laplacian.

Convergence reading.  The median-dual cells of the octahedral grid are
smooth inside each octant, and there the scheme converges at second order;
along the octant seams (the meridians at multiples of 90 deg and the
equator, where the row triangulation turns) and in the polar rows the cells
are not symmetric and pointwise errors decay at first order only.  Seams
are lines, so over a band that contains them the volume-weighted L2 error
decays at about order 1.5.  The floors asserted below sit 0.03 to 0.09 under
the measured orders (O16 -> O32 -> O64; measured, O32 -> O64: gradient 1.78
and divergence 1.95 in the octant interiors, 1.47 and 1.59 over the band
|lat| < 60 deg, 0.99 for the gradient over the whole sphere), so a mistake
that costs half an order fails them (two such mutants are planted in the
mutant tests).
"""
import numpy as np
import pytest

R = 6371220.0


def _l2(V, e, mask=None):
    if mask is None:
        mask = np.ones_like(V, bool)
    return np.sqrt(np.sum(V[mask] * e[mask] ** 2) / np.sum(V[mask]))


def _slopes(errs):
    return [np.log2(errs[i] / errs[i + 1]) for i in range(len(errs) - 1)]


# floors: (each refinement, the last refinement O32 -> O64)
FLOORS = {"gradient_interior": (1.5, 1.7), "divergence_interior": (1.8, 1.9),
          "gradient_band": (1.3, 1.4), "divergence_band": (1.5, 1.55), "rotation_band": (1.25, 1.4),
          "gradient_sphere": (0.95, 0.95)}


def _bulk_order_ok(errs, floor=(1.25, 1.4)):
    s = _slopes(errs)
    return min(s) >= floor[0] and s[-1] >= floor[1]


def octant_interior(lam, phi, margin_deg=3.0):
    """Nodes of the band |lat| < 60 deg at least margin_deg from the octant
    seams (the meridians at multiples of 90 deg and the equator)."""
    dl = np.degrees(np.abs((lam + np.pi / 4) % (np.pi / 2) - np.pi / 4))
    return (np.abs(phi) < np.radians(60)) & (dl >= margin_deg) & (np.degrees(np.abs(phi)) >= margin_deg)


def convergence_orders(mesh_of):
    """Orders of the volume-weighted L2 errors of the closed-form gradient
    (f = cos lat cos lon) and divergence ((u, v) = (cos lat, 0.1 sin lon cos
    lat)) on O16, O32, O64, over the octant interiors, the band
    |lat| < 60 deg and (gradient) the whole sphere; mesh_of(N) gives the
    oracle mesh."""
    errs = {k: [] for k in FLOORS if k != "rotation_band"}
    for N in (16, 32, 64):
        m = mesh_of(N)
        lam, phi, V = _fields(m)
        band, inner = np.abs(phi) < np.radians(60), octant_interior(lam, phi)
        gx, gy = m.gradient(np.cos(phi) * np.cos(lam))
        e = np.hypot(gx[:, 0] + np.sin(lam) / R, gy[:, 0] + np.sin(phi) * np.cos(lam) / R) * R
        errs["gradient_interior"].append(_l2(V, e, inner))
        errs["gradient_band"].append(_l2(V, e, band))
        errs["gradient_sphere"].append(_l2(V, e))
        d = m.divergence(np.cos(phi), 0.1 * np.sin(lam) * np.cos(phi))[:, 0] * R
        e = d + 0.2 * np.sin(lam) * np.sin(phi)
        errs["divergence_interior"].append(_l2(V, e, inner))
        errs["divergence_band"].append(_l2(V, e, band))
    return {k: _slopes(v) for k, v in errs.items()}


def orders_meet_floors(orders):
    return all(min(s) >= FLOORS[k][0] and s[-1] >= FLOORS[k][1] for k, s in orders.items())


def test_gradient_of_constant_is_exactly_zero(omesh):
    m = omesh(16)
    f = np.full((m.nnodes, 3), 3.7)
    gx, gy = m.gradient(f)
    assert np.all(gx == 0) and np.all(gy == 0)
    f32 = np.full((m.nnodes, 2), -1.25, np.float32)
    gx, gy = m.gradient(f32)
    assert np.all(gx == 0) and np.all(gy == 0)


def _fields(m):
    g = m.grid()
    return g["lon"], g["lat_node"], m.dual()["V"]


def test_gradient_and_divergence_convergence(omesh):
    """Second order in the octant interiors, about 1.5 over the band, first
    order over the whole sphere (the polar rows)."""
    orders = convergence_orders(omesh)
    for k, s in orders.items():
        assert min(s) >= FLOORS[k][0] and s[-1] >= FLOORS[k][1], (k, s)


@pytest.mark.parametrize("alpha", [0.0, np.pi / 4])
def test_solid_body_rotation_divergence_free(omesh, alpha):
    errs = []
    for N in (16, 32, 64):
        m = omesh(N)
        lam, phi, V = _fields(m)
        u = np.cos(phi) * np.cos(alpha) + np.sin(phi) * np.cos(lam) * np.sin(alpha)
        v = -np.sin(lam) * np.sin(alpha)
        d = m.divergence(u, v)[:, 0] * R
        errs.append(_l2(V, d, np.abs(phi) < np.radians(60)))
    if alpha == 0.0:
        assert max(errs) <= 1e-13  # zonal flow: exact to rounding
    else:
        assert _bulk_order_ok(errs, FLOORS["rotation_band"]), _slopes(errs)


def test_divergence_closed_form(omesh):
    """(u, v) = (cos lat, 0.1 sin lon cos lat): div = -0.2 sin lon sin lat / R."""
    errs = []
    for N in (16, 32, 64):
        m = omesh(N)
        lam, phi, V = _fields(m)
        d = m.divergence(np.cos(phi), 0.1 * np.sin(lam) * np.cos(phi))[:, 0] * R
        errs.append(_l2(V, d + 0.2 * np.sin(lam) * np.sin(phi), np.abs(phi) < np.radians(60)))
    assert _bulk_order_ok(errs, FLOORS["divergence_band"]), _slopes(errs)


def _real_sph_harm(l, m_, lam, phi):
    """Real spherical harmonic (unnormalised): P_l^|m|(sin lat) cos/sin(m lon)."""
    from scipy.special import lpmv
    x = np.sin(phi)
    P = lpmv(abs(m_), l, x)
    return P * (np.cos(m_ * lam) if m_ >= 0 else np.sin(-m_ * lam))


@pytest.mark.parametrize("l,m_", [(1, 0), (2, 1), (3, -2), (4, 3)])
def test_laplacian_of_spherical_harmonics(omesh, l, m_):
    """Laplacian of Y_l^m approaches -l(l+1)/R^2 Y: the relative L2 error over
    |lat| < 60 deg falls monotonically from O16 to O64 and is below 5% at O64."""
    rel = []
    for N in (16, 32, 64):
        m = omesh(N)
        lam, phi, V = _fields(m)
        Y = _real_sph_harm(l, m_, lam, phi)
        lap = m.laplacian(Y)[:, 0] * R * R
        want = -l * (l + 1) * Y
        bulk = np.abs(phi) < np.radians(60)
        rel.append(_l2(V, lap - want, bulk) / _l2(V, want, bulk))
    assert rel[0] > rel[1] > rel[2]
    assert rel[2] < 0.05


@pytest.mark.parametrize("N", [16, 32])
def test_divergence_conservation(omesh, N):
    m = omesh(N)
    rng = np.random.default_rng(1)
    u = rng.standard_normal((m.nnodes, 3))
    v = rng.standard_normal((m.nnodes, 3))
    V = m.dual()["V"]
    d = m.divergence(u, v)
    for k in range(3):
        t = V * d[:, k]
        assert abs(np.sum(t)) <= 1e-12 * np.sum(np.abs(t))


def _dense(op, m, nin):
    """Dense matrix of a forward operator by applying it to unit vectors."""
    V = m.nnodes
    cols = []
    for c in range(nin * V):
        x = np.zeros((nin, V, 1))
        x[c // V, c % V, 0] = 1.0
        cols.append(np.concatenate([o[:, 0] for o in op(*x)]))
    return np.stack(cols, axis=1)


def test_adjoints_are_bruteforce_transposes(omesh):
    m = omesh(2)
    rng = np.random.default_rng(2)
    G = _dense(lambda f: m.gradient(f), m, 1)             # (2V, V)
    D = _dense(lambda u, v: (m.divergence(u, v),), m, 2)  # (V, 2V)
    V = m.nnodes
    y = rng.standard_normal((2, V, 2))
    x = m.gradient_adjoint(y[0], y[1])
    want = G.T @ np.concatenate([y[0], y[1]])
    assert np.max(np.abs(x - want)) <= 1e-13 * np.max(np.abs(want))
    d = rng.standard_normal((V, 2))
    xu, xv = m.divergence_adjoint(d)
    want = D.T @ d
    assert np.max(np.abs(np.concatenate([xu, xv]) - want)) <= 1e-13 * np.max(np.abs(want))
    # the COO triplets are the same matrices
    from scipy.sparse import coo_matrix
    r, c, val = m.triplets("gradient")
    Gs = coo_matrix((val, (r, c)), shape=(2 * V, V)).toarray()
    assert np.max(np.abs(Gs - G)) <= 1e-13 * np.max(np.abs(G))
    r, c, val = m.triplets("divergence")
    Ds = coo_matrix((val, (r, c)), shape=(V, 2 * V)).toarray()
    assert np.max(np.abs(Ds - D)) <= 1e-13 * np.max(np.abs(D))


@pytest.mark.parametrize("N", [16, 32])
def test_dot_product_test(omesh, N):
    m = omesh(N)
    rng = np.random.default_rng(3)
    L = 4
    x = rng.standard_normal((m.nnodes, L))
    y0 = rng.standard_normal((m.nnodes, L))
    y1 = rng.standard_normal((m.nnodes, L))
    gx, gy = m.gradient(x)
    lhs = np.sum(gx * y0) + np.sum(gy * y1)
    rhs = np.sum(x * m.gradient_adjoint(y0, y1))
    assert abs(lhs - rhs) <= 1e-12 * abs(lhs)
    u, v, d = (rng.standard_normal((m.nnodes, L)) for _ in range(3))
    lhs = np.sum(m.divergence(u, v) * d)
    xu, xv = m.divergence_adjoint(d)
    rhs = np.sum(u * xu) + np.sum(v * xv)
    assert abs(lhs - rhs) <= 1e-12 * abs(lhs)


def test_finite_difference_of_weighted_gradient_loss(omesh):
    """J(f) = sum_i V_i |grad f|_i^2 (all levels); dJ/df = 2 G^T (V g)."""
    m = omesh(16)
    L = 4
    rng = np.random.default_rng(4)
    g = m.grid()
    f = np.cos(g["lat_node"])[:, None] * np.cos(g["lon"])[:, None] * (1 + 0.1 * np.arange(L)) + \
        0.01 * rng.standard_normal((m.nnodes, L))
    V = m.dual()["V"]

    def J(ff):
        gx, gy = m.gradient(ff)
        return np.sum(V[:, None] * (gx * gx + gy * gy))

    gx, gy = m.gradient(f)
    grad = 2.0 * m.gradient_adjoint(V[:, None] * gx, V[:, None] * gy)
    eps = 1e-6
    # J is quadratic, so central differences are exact up to the rounding of J
    roundoff = 64 * np.finfo(float).eps * J(f) / (2 * eps)
    for i, k in [(0, 0), (5, 1), (m.nnodes // 2, 2), (m.nnodes - 1, 3), (777, 0)]:
        fp = f.copy(); fp[i, k] += eps
        fm = f.copy(); fm[i, k] -= eps
        fd = (J(fp) - J(fm)) / (2 * eps)
        assert abs(fd - grad[i, k]) <= 1e-9 * abs(grad[i, k]) + roundoff


def test_node_subsets_match_full_evaluation(omesh):
    m = omesh(8)
    rng = np.random.default_rng(6)
    f, u, v = (rng.standard_normal((m.nnodes, 3)) for _ in range(3))
    nodes = np.array([0, 3, 19, 20, 150, m.nnodes - 1, m.nnodes - 11], np.int64)
    gx, gy = m.gradient(f)
    sx, sy = m.gradient(f, nodes=nodes)
    assert np.array_equal(sx, gx[nodes]) and np.array_equal(sy, gy[nodes])
    assert np.array_equal(m.divergence(u, v, nodes=nodes), m.divergence(u, v)[nodes])
    assert np.array_equal(m.laplacian(f, nodes=nodes), m.laplacian(f)[nodes])
    assert np.array_equal(m.gradient_adjoint(u, v, nodes=nodes), m.gradient_adjoint(u, v)[nodes])
    xu, xv = m.divergence_adjoint(f)
    su, sv = m.divergence_adjoint(f, nodes=nodes)
    assert np.array_equal(su, xu[nodes]) and np.array_equal(sv, xv[nodes])


def test_float32_inputs_are_upcast_exactly(omesh):
    m = omesh(8)
    rng = np.random.default_rng(7)
    f32 = rng.standard_normal((m.nnodes, 5)).astype(np.float32)
    # padded leading dimension
    buf = np.zeros((m.nnodes, 8), np.float32)
    buf[:, :5] = f32
    gx, gy = m.gradient(buf, nlev=5)
    hx, hy = m.gradient(f32.astype(np.float64))
    assert np.array_equal(gx, hx) and np.array_equal(gy, hy)
