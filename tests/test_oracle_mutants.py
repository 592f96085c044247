"""The oracle's pins catch plausible mistakes: each case plants one bug in a
copy of the oracle's C source (a wrong tie rule, a dropped metric factor, a
sign, a formula) or in one function of its Python module, builds it, and
checks that a named pin passes on the real oracle and fails on the mutant.
Mutants are built in a temporary directory (C) or a private namespace
(Python) and used only inside their test; the oracle itself is never
changed.  Several pins are the oracle's own tests, called directly."""
import contextlib
import ctypes
import inspect
import os
import subprocess

import numpy as np
import pytest

from oracle import oracle
from test_oracle_dual import _dual_by_quadrature
from test_oracle_grid import _zipper_bruteforce
from test_oracle_grid import test_latitudes_match_legendre_roots as _latitudes_test
from test_oracle_integral import test_exact_against_fractions as _fractions_test
from test_oracle_operators import test_adjoints_are_bruteforce_transposes as _transposes_test
from test_oracle_operators import test_node_subsets_match_full_evaluation as _subsets_test
from test_oracle_operators import convergence_orders, orders_meet_floors
from test_oracle_regional import test_scale_factors_and_orthogonality_from_chords as _chords_test
from test_oracle_regional import test_cell_areas_and_closure as _areas_test
from test_oracle_regional import test_linear_fields_are_exact_everywhere as _linear_test
from test_oracle_integral import test_residual_after_cancelling_the_rounded_sum as _residual_test
from test_oracle_remap import test_weights_are_barycentric_coordinates_of_the_ray_crossing as _barycentric_test
from test_oracle_remap import test_targets_on_source_nodes_take_the_node_values as _on_nodes_test
from test_oracle_vector_ops import test_curl_of_solid_body_rotation as _curl_test
from test_oracle_vector_ops import test_vector_gradient_reverses_the_antipode_on_pole_faces as _antipode_test
from synthetic.regional import DOMAINS

HERE = os.path.dirname(os.path.abspath(__file__))
SOURCES = {"global": os.path.join(HERE, "..", "oracle", "atlas_oracle.c"),
           "regional": os.path.join(HERE, "..", "oracle", "regional_oracle.c")}
R = oracle.R_EARTH


def _build(tmp, which, old, new):
    texts = {k: open(p).read() for k, p in SOURCES.items()}
    assert texts[which].count(old) == 1, "mutation site not found once: %r" % old
    texts[which] = texts[which].replace(old, new)
    files = []
    for k, t in texts.items():
        path = os.path.join(tmp, k + ".c")
        with open(path, "w") as fh:
            fh.write(t)
        files.append(path)
    so = os.path.join(tmp, "mutant.so")
    subprocess.check_call(["gcc", *oracle.CFLAGS, "-o", so, *files, "-lm"])
    return ctypes.CDLL(so)


@contextlib.contextmanager
def _oracle_lib(lib):
    saved = oracle._load()
    oracle._lib = oracle._configure(lib)
    try:
        yield
    finally:
        oracle._lib = saved


# ------------------------------------------------------------------ pins
def pin_zipper():
    m = oracle.Mesh(3)
    d, pl = m.mesh(), m.grid()["pl"]
    got = {}
    for t in range(m.ntri):
        r = int(d["tri_r"][t].min())
        got.setdefault(r, []).append(tuple((int(d["tri_r"][t, k]) - r, int(d["tri_j"][t, k])) for k in range(3)))
    return all(got[r] == _zipper_bruteforce(int(pl[r]), int(pl[r + 1])) for r in range(5))


def pin_closure():
    res, ab = oracle.Mesh(8).closure()
    return np.max(np.abs(res).max(1) / ab) <= 1e-14


def pin_gradient_closed_form():
    m = oracle.Mesh(32)
    g = m.grid()
    lam, phi = g["lon"], g["lat_node"]
    gx, gy = m.gradient(np.cos(phi) * np.cos(lam))
    e = np.hypot(gx[:, 0] + np.sin(lam) / R, gy[:, 0] + np.sin(phi) * np.cos(lam) / R) * R
    return e[np.abs(phi) < np.radians(60)].max() <= 0.05  # 0.014 for the scheme


def pin_convergence_orders():
    return orders_meet_floors(convergence_orders(oracle.Mesh))


def pin_sphere_area():
    V = oracle.Mesh(16).dual()["V"]
    return abs(V.sum() - 4 * np.pi * R ** 2) <= 1e-12 * 4 * np.pi * R ** 2


def pin_volumes_by_quadrature():
    m = oracle.Mesh(4)
    Vq, _ = _dual_by_quadrature(m)
    return np.max(np.abs(m.dual()["V"] - Vq) / Vq) <= 1e-13


def pin_conservation():
    m = oracle.Mesh(16)
    rng = np.random.default_rng(2)
    u, v = rng.standard_normal((m.nnodes, 2)), rng.standard_normal((m.nnodes, 2))
    Vd = m.dual()["V"][:, None] * m.divergence(u, v)
    return np.all(np.abs(Vd.sum(0)) <= 1e-12 * np.abs(Vd).sum(0))


def _regional(name, **over):
    proj, kw = DOMAINS[name]
    return oracle.RegionalMesh(proj, 17, 11, **dict(kw, **over))


def pin_regional_linear(name="rotated"):
    m = _regional(name)
    g = m.geometry()
    x, y, hx, hy = g["x"], g["y"], g["hx"], g["hy"]
    gx, gy = m.gradient((0.7 * x - 1.3 * y)[:, None])
    ok = np.allclose(gx[:, 0], 0.7 / (R * hx), rtol=1e-12, atol=0) and np.allclose(gy[:, 0], -1.3 / (R * hy),
                                                                                    rtol=1e-12, atol=0)
    cur = m.curl(((0.7 * x - 1.3 * y) / hx)[:, None], ((0.45 * x + 2.1 * y) / hy)[:, None])[:, 0]
    return ok and np.allclose(cur, (0.45 + 1.3) / (R * hx * hy), rtol=1e-12, atol=0)


def pin_lambert_scale_from_chords():
    proj, kw = DOMAINS["lambert"]
    kw = dict(kw, xmin=2e5 - 1.0, xmax=2e5 + 1.0, ymin=1e5 - 1.0, ymax=1e5 + 1.0)
    g = oracle.RegionalMesh(proj, 3, 3, **kw).geometry()
    P = np.stack([np.cos(g["lat"]) * np.cos(g["lon"]), np.cos(g["lat"]) * np.sin(g["lon"]), np.sin(g["lat"])], 1)
    h = np.linalg.norm(P[5] - P[3]) / (2.0 / R)
    return abs(h - g["hx"][4]) <= 1e-6 * g["hx"][4]


def pin_rotated_pole_distance():
    g = _regional("rotated").geometry()
    sp = DOMAINS["rotated"][1]["south_pole"]
    P = np.stack([np.cos(g["lat"]) * np.cos(g["lon"]), np.cos(g["lat"]) * np.sin(g["lon"]), np.sin(g["lat"])], 1)
    lon_n, lat_n = np.radians(sp[0] + 180.0), np.radians(-sp[1])
    north = np.array([np.cos(lat_n) * np.cos(lon_n), np.cos(lat_n) * np.sin(lon_n), np.sin(lat_n)])
    ang = np.arctan2(np.linalg.norm(np.cross(P, north), axis=1), P @ north)
    return np.max(np.abs(ang - (np.pi / 2 - g["y"]))) <= 1e-12


def _meshes(N):
    return oracle.Mesh(N, R)


def _passes(test, *args):
    """A test of the oracle used as a pin: True when its assertions hold."""
    try:
        test(*args)
    except AssertionError:
        return False
    return True


def pin_latitudes():
    return _passes(_latitudes_test, oracle, 64)


def pin_barycentric():
    return _passes(_barycentric_test, _meshes, 16, 8)


def pin_curl_solid_body():
    return _passes(_curl_test, _meshes, 0.0)


def pin_antipode():
    return _passes(_antipode_test, _meshes)


def pin_transposes():
    return _passes(_transposes_test, _meshes)


def pin_subsets():
    return _passes(_subsets_test, _meshes)


def pin_remap_on_nodes():
    return _passes(_on_nodes_test, _meshes)


def pin_chords(name):
    return lambda: _passes(_chords_test, name)


def pin_areas(name):
    return lambda: _passes(_areas_test, name)


def pin_linear(name):
    return lambda: _passes(_linear_test, name)


def pin_exact_sums():
    return _passes(_fractions_test) and _passes(_residual_test)


MUTANTS = [
    ("tie rule reversed", "global", "else north = (n1 <= n2);", "else north = (n1 > n2);", pin_zipper),
    ("pole faces signed like regular faces", "global",
     "double s = m->is_pole[e] ? 1.0 : (double)m->n2e_sign[p];", "double s = (double)m->n2e_sign[p];", pin_closure),
    ("cos metric dropped from the gradient", "global",
     "      double d = 0.5 * (fld(f, f32, ld, j, k) - fi);\n      acc_add_prod(&al, nl, d);\n"
     "      acc_add_prod(&ap, np, d);\n    }\n    gx[k] = acc_val(&al) / m->V[i];\n"
     "    gy[k] = m->coslat[i] * acc_val(&ap) / m->V[i];",
     "      double d = 0.5 * (fld(f, f32, ld, j, k) - fi);\n      acc_add_prod(&al, nl, d);\n"
     "      acc_add_prod(&ap, np, d);\n    }\n    gx[k] = acc_val(&al) / m->V[i];\n"
     "    gy[k] = acc_val(&ap) / m->V[i];", pin_gradient_closed_form),
    ("cross-row edge midpoints at a third of the row spacing (first-order volumes)", "global",
     "double mphi = (tr[ia] == tr[ib]) ? phia : 0.5 * (m->lat[r] + m->lat[s]);",
     "double mphi = (tr[ia] == tr[ib]) ? phia : (2.0 * m->lat[r] + m->lat[s]) / 3.0;", pin_convergence_orders),
    ("centroid latitude as the mean of two rows (order pin)", "global",
     "double cphi = ((m->lat[p] + m->lat[p]) + m->lat[qq]) / 3.0;",
     "double cphi = (m->lat[p] + m->lat[qq]) / 2.0;", pin_convergence_orders),
    ("pole segment dropped from the volumes", "global",
     "acc_add(&vacc[m->off[rr] + j], ipole);", "(void)ipole;", pin_sphere_area),
    ("centroid latitude as the mean of two rows", "global",
     "double cphi = ((m->lat[p] + m->lat[p]) + m->lat[qq]) / 3.0;",
     "double cphi = (m->lat[p] + m->lat[qq]) / 2.0;", pin_volumes_by_quadrature),
    ("neighbour's cos replaced by the node's in the divergence", "global",
     "double dv = 0.5 * diff_of_products(fld(v, f32, ld, j, k), m->coslat[j], vi, ci);",
     "double dv = 0.5 * diff_of_products(fld(v, f32, ld, j, k), ci, vi, ci);", pin_conservation),
    ("pole flux sign flipped in the divergence", "global",
     "      two_prod(vi, ci, &pv, &ev);\n      acc_add_prod(&a, -m->pole_nphi[i], pv);\n"
     "      acc_add_prod(&a, -m->pole_nphi[i], ev);\n    }\n    out[k] = acc_val(&a) / m->V[i];",
     "      two_prod(vi, ci, &pv, &ev);\n      acc_add_prod(&a, m->pole_nphi[i], pv);\n"
     "      acc_add_prod(&a, m->pole_nphi[i], ev);\n    }\n    out[k] = acc_val(&a) / m->V[i];", pin_conservation),
    ("boundary half-edge weighted (3 f_i + f_j)/4", "regional",
     "(int32_t)i, j, 5.0 / 6.0, 1.0 / 6.0};", "(int32_t)i, j, 0.75, 0.25};", pin_regional_linear),
    ("h_y in place of h_x in the gradient", "regional",
     "gx[l] = r_val(&ax) / (g->A[i] * g->hx[i]);", "gx[l] = r_val(&ax) / (g->A[i] * g->hy[i]);",
     pin_regional_linear),
    ("curl with the wrong sign of -h_x u", "regional",
     "reg_flux_node(g, seg, ns, i, v, u, f32, ld, l, 1.0, -1.0)", "reg_flux_node(g, seg, ns, i, v, u, f32, ld, l, 1.0, 1.0)",
     pin_regional_linear),
    ("Lambert scale factor k instead of 1/k", "regional", "*hx = *hy = 1.0 / k;", "*hx = *hy = k;",
     pin_lambert_scale_from_chords),
    ("rotated frame turned the wrong way", "regional", "double b = -(0.5 * RPI + pp);",
     "double b = (0.5 * RPI + pp);", pin_rotated_pole_distance),
    ("Legendre series coefficients g_k g_k instead of g_k g_(n-k)", "global", "c[k] = g[k] * g[n - k];",
     "c[k] = g[k] * g[k];", pin_latitudes),
    ("remap weights given to the wrong vertices", "global", "bw[0] = w0; bw[1] = u; bw[2] = v;",
     "bw[0] = u; bw[1] = w0; bw[2] = v;", pin_barycentric),
    ("remap accepts the triangle on the far side of the sphere", "global",
     "if (tt <= 0) continue; /* the far side of the sphere */", "(void)tt;", pin_barycentric),
    ("curl with the sign of the (u cos) term flipped", "global", "acc_add_prod(&a, -np, duc);",
     "acc_add_prod(&a, np, duc);", pin_curl_solid_body),
    ("vector gradient treats pole faces like scalar ones", "global",
     "double d = m->is_pole[e] ? -0.5 * (fj + fi) : 0.5 * (fj - fi);", "double d = 0.5 * (fj - fi);",
     pin_antipode),
    ("divergence adjoint with the node's cos in place of the neighbour's", "global",
     "ent[nent].c1 = np * m->coslat[j] / (2.0 * m->V[i]);", "ent[nent].c1 = np * ci / (2.0 * m->V[i]);",
     pin_transposes),
    ("gradient adjoint reads y_lambda for both components", "global",
     "acc_add_prod(&acc[l], ent[t].c1, fld(y1, f32, ld, i, l));",
     "acc_add_prod(&acc[l], ent[t].c1, fld(y0, f32, ld, i, l));", pin_transposes),
    ("node-subset Laplacian takes the node's gradient for its neighbours'", "global",
     "double uj = gx[(1 + p - p0) * nlev + k], vj = gy[(1 + p - p0) * nlev + k];",
     "double uj = gx[k], vj = gy[k];", pin_subsets),
    ("remap applies the first weight to all three vertices", "global",
     "acc_add_prod(&a, w[3 * t + q], fld(f, f32, ld, nodes[3 * t + q], k));",
     "acc_add_prod(&a, w[3 * t], fld(f, f32, ld, nodes[3 * t + q], k));", pin_remap_on_nodes),
    ("Mercator scale factor 1/cos instead of cos", "regional", "*hx = *hy = cos(*lat);",
     "*hx = *hy = 1.0 / cos(*lat);", pin_chords("mercator")),
    ("polar stereographic scale factor inverted", "regional", "*hx = *hy = 4.0 / (4.0 + r2);",
     "*hx = *hy = (4.0 + r2) / 4.0;", pin_chords("polar")),
    ("polar stereographic plane mirrored", "regional", "atan2(x, -north * y);", "atan2(x, north * y);",
     pin_chords("polar")),
    ("right side of the rectangle not seen as boundary", "regional",
     "if (ca == cb && (ca == 0 || ca == g->nx - 1)) return 1;", "if (ca == cb && ca == 0) return 1;",
     pin_areas("rotated")),
    ("triangle area shared in halves instead of thirds", "regional",
     "g->A[v[k]] += R * R * (0.5 * ar) / 3.0;", "g->A[v[k]] += R * R * (0.5 * ar) / 2.0;", pin_areas("lambert")),
    ("Lambert longitude without the cone constant", "regional", "*lon = p[5] * RPI / 180.0 + th / n;",
     "*lon = p[5] * RPI / 180.0 + th;", pin_chords("lambert")),
    ("flux form without the h_y factor on its first component", "regional",
     "double d1 = s1 * rdiff(g->hy[cb], rfld(p, f32, ld, cb, l), g->hy[i], pi);",
     "double d1 = s1 * (rfld(p, f32, ld, cb, l) - pi);", pin_linear("mercator")),
]

# mistakes planted in the Python part of the oracle (the exact sums)
PY_MUTANTS = [
    ("low x low product dropped", "integral", "vh * xh, vh * xl, vl * xh, vl * xl", "vh * xh, vh * xl, vl * xh",
     pin_exact_sums),
    ("Veltkamp constant 2^26 + 1 (halves too wide for exact products)", "_split", "134217729.0", "67108865.0",
     pin_exact_sums),
    ("sum rounded term by term instead of exactly", "integral", "math.fsum(", "sum(", pin_exact_sums),
]


@pytest.mark.parametrize("what,which,old,new,pin", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_pin_catches_planted_mistake(tmp_path, what, which, old, new, pin):
    if not pytest.importorskip("shutil").which("gcc"):
        pytest.skip("gcc missing")
    assert pin(), "the pin fails on the real oracle"
    lib = _build(str(tmp_path), which, old, new)
    with _oracle_lib(lib):
        caught = not pin()
    assert caught, "the planted mistake (%s) passed the pin %s" % (what, pin.__name__)


@pytest.mark.parametrize("what,name,old,new,pin", PY_MUTANTS, ids=[m[0] for m in PY_MUTANTS])
def test_pin_catches_planted_python_mistake(monkeypatch, what, name, old, new, pin):
    assert pin(), "the pin fails on the real oracle"
    src = inspect.getsource(getattr(oracle, name))
    assert src.count(old) == 1, "mutation site not found once: %r" % old
    ns = dict(vars(oracle))
    exec(compile(src.replace(old, new), "<mutant of oracle.%s>" % name, "exec"), ns)
    monkeypatch.setattr(oracle, name, ns[name])
    caught = not pin()
    monkeypatch.undo()
    assert caught, "the planted mistake (%s) passed the pin %s" % (what, pin.__name__)
