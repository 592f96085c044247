"""ctypes front end of the FP64 CPU oracle (``atlas_oracle.c``).

TEST INFRASTRUCTURE. Only ``tests/``, ``__graft_entry__`` (``build()``
compiles it, ``smoke()`` checks against it) and the CPU legs of ``bench.py``
(its CPU baseline and its ``--impl reference`` arm) import this module. It
imports nothing from the product package and the product never imports it.

The oracle computes, in plain FP64 C, the octahedral reduced Gaussian grid,
its zipper triangulation with pole edges, the median-dual geometry and the
nabla operators (gradient, divergence, Laplacian, the adjoints of gradient
and divergence, curl and the gradient of a tangent vector field) that Atlas
supplies (paper Sec. 2.3).  The formulas and the
readings they follow are stated beside each function in ``atlas_oracle.c``.
Every function here is pinned by ``tests/test_oracle_*.py``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "atlas_oracle.c")
_SRC_REGIONAL = os.path.join(_HERE, "regional_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None

R_EARTH = 6371220.0

CFLAGS = ["-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off", "-fno-fast-math"]


def build(force: bool = False) -> str:
    """Compile the oracle into ``oracle/_build/liboracle.so`` (gcc, no GPU)."""
    os.makedirs(_BUILD, exist_ok=True)
    srcs = [_SRC, _SRC_REGIONAL]
    if force or not os.path.exists(_LIB) or any(os.path.getmtime(_LIB) < os.path.getmtime(x) for x in srcs):
        tmp = _LIB + ".%d.tmp" % os.getpid()
        subprocess.check_call(["gcc", *CFLAGS, "-o", tmp, *srcs, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def _configure(lib):
    """Declare the C signatures on a loaded oracle library."""
    P = ctypes.c_void_p
    i64 = ctypes.c_int64
    lib.orc_build.restype = P
    lib.orc_build.argtypes = [ctypes.c_int, ctypes.c_double]
    lib.orc_build_grid.restype = P
    lib.orc_build_grid.argtypes = [ctypes.c_int, ctypes.c_double, ctypes.c_int]
    lib.orc_free.argtypes = [P]
    lib.orc_counts.argtypes = [P, P]
    lib.orc_gauss_colatitudes.argtypes = [ctypes.c_int, P]
    lib.orc_get_grid.argtypes = [P, P, P, P, P]
    lib.orc_get_mesh.argtypes = [P] * 9
    lib.orc_get_dual.argtypes = [P] * 5
    lib.orc_gradient.argtypes = [P, P, ctypes.c_int, i64, ctypes.c_int, P, i64, P, P]
    lib.orc_gradient_adjoint.argtypes = [P, P, P, ctypes.c_int, i64, ctypes.c_int, P, i64, P]
    lib.orc_divergence.argtypes = [P, P, P, ctypes.c_int, i64, ctypes.c_int, P, i64, P]
    lib.orc_laplacian.argtypes = [P, P, ctypes.c_int, i64, ctypes.c_int, P, i64, P]
    lib.orc_divergence_adjoint.argtypes = [P, P, ctypes.c_int, i64, ctypes.c_int, P, i64, P, P]
    lib.orc_curl.argtypes = [P, P, P, ctypes.c_int, i64, ctypes.c_int, P, i64, P]
    lib.orc_curl_adjoint.argtypes = [P, P, ctypes.c_int, i64, ctypes.c_int, P, i64, P, P]
    lib.orc_remap.argtypes = [P, P, i64, P, P]
    lib.orc_remap_apply.argtypes = [P, P, i64, P, ctypes.c_int, i64, ctypes.c_int, P]
    lib.orc_vector_gradient.argtypes = [P, P, P, ctypes.c_int, i64, ctypes.c_int, P, i64, P, P, P, P]
    lib.orc_gradient_triplets.restype = i64
    lib.orc_gradient_triplets.argtypes = [P, P, P, P]
    lib.orc_divergence_triplets.restype = i64
    lib.orc_divergence_triplets.argtypes = [P, P, P, P]
    lib.orc_gradient_averaged.argtypes = [P, P, ctypes.c_int, i64, ctypes.c_int, P, P]
    lib.orc_closure.argtypes = [P, P, P]
    lib.orc_reg_build.restype = P
    lib.orc_reg_build.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, P, ctypes.c_double]
    lib.orc_reg_free.argtypes = [P]
    lib.orc_reg_counts.argtypes = [P, P]
    lib.orc_reg_get.argtypes = [P] * 6
    lib.orc_reg_closure.argtypes = [P, P, P]
    lib.orc_reg_gradient.argtypes = [P, P, ctypes.c_int, i64, ctypes.c_int, P, i64, P, P]
    lib.orc_reg_divergence.argtypes = [P, P, P, ctypes.c_int, i64, ctypes.c_int, P, i64, P]
    lib.orc_reg_curl.argtypes = [P, P, P, ctypes.c_int, i64, ctypes.c_int, P, i64, P]
    lib.orc_reg_laplacian.argtypes = [P, P, ctypes.c_int, i64, ctypes.c_int, P, i64, P]
    lib.orc_reg_gradient_adjoint.argtypes = [P, P, P, ctypes.c_int, i64, ctypes.c_int, P, i64, P]
    lib.orc_reg_divergence_adjoint.argtypes = [P, P, ctypes.c_int, i64, ctypes.c_int, P, i64, P, P]
    lib.orc_reg_gradient_averaged.argtypes = [P, P, ctypes.c_int, i64, ctypes.c_int, P, P]
    for name in ("orc_reg_gradient", "orc_reg_divergence", "orc_reg_curl", "orc_reg_laplacian",
                 "orc_reg_gradient_adjoint", "orc_reg_divergence_adjoint", "orc_reg_gradient_averaged"):
        getattr(lib, name).restype = ctypes.c_int
    for name in ("orc_gradient", "orc_divergence", "orc_laplacian", "orc_gradient_adjoint",
                 "orc_divergence_adjoint", "orc_gradient_averaged", "orc_gauss_colatitudes", "orc_curl",
                 "orc_curl_adjoint",
                 "orc_vector_gradient", "orc_remap", "orc_remap_apply"):
        getattr(lib, name).restype = ctypes.c_int
    return lib


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        _lib = _configure(ctypes.CDLL(build()))
        return _lib


def _ptr(a):
    return a.ctypes.data_as(ctypes.c_void_p) if a is not None else None


def gauss_colatitudes(n: int) -> np.ndarray:
    """Colatitudes (radians, ascending from the north pole) of the n roots of P_n."""
    out = np.empty(n, dtype=np.float64)
    if _load().orc_gauss_colatitudes(int(n), _ptr(out)) != 0:
        raise ValueError("invalid n")
    return out


def _field(x):
    """Accept a 2-D float32/float64 array [node][level] (any leading dim)."""
    x = np.asarray(x)
    if x.ndim == 1:
        x = x[:, None]
    if x.dtype not in (np.float32, np.float64):
        raise TypeError("oracle fields are float32 or float64")
    if x.strides[1] != x.itemsize:
        x = np.ascontiguousarray(x)
    ld = x.strides[0] // x.itemsize
    return x, int(x.dtype == np.float32), ld


class Mesh:
    """Oracle grid + mesh + median dual for the octahedral grid O<N>."""

    def __init__(self, N: int, R: float = R_EARTH, regular: bool = False):
        """Octahedral grid O<N>, or with regular=True the regular Gaussian
        grid F<N> (4N points per row), meshed and dualised the same way."""
        lib = _load()
        h = lib.orc_build_grid(int(N), float(R), int(bool(regular)))
        if not h:
            raise ValueError("oracle mesh build failed for N=%r" % (N,))
        self._h = ctypes.c_void_p(h)
        self._lib = lib
        self.R = float(R)
        c = np.zeros(6, dtype=np.int64)
        lib.orc_counts(self._h, _ptr(c))
        self.N, self.nlat, self.nnodes, self.ntri, self.nedges, self.nnz = (int(v) for v in c)

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and h.value:
            self._lib.orc_free(h)
            self._h = None

    # ---------------------------------------------------------------- data
    def grid(self):
        pl = np.empty(self.nlat, np.int32)
        lat = np.empty(self.nlat)
        colat = np.empty(self.nlat)
        lonlat = np.empty((self.nnodes, 2))
        self._lib.orc_get_grid(self._h, _ptr(pl), _ptr(lat), _ptr(colat), _ptr(lonlat))
        return dict(pl=pl, lat=lat, colat=colat, lon=lonlat[:, 0].copy(), lat_node=lonlat[:, 1].copy())

    def mesh(self):
        T, E, V = self.ntri, self.nedges, self.nnodes
        d = dict(tri=np.empty((T, 3), np.int32), tri_r=np.empty((T, 3), np.int32),
                 tri_j=np.empty((T, 3), np.int32), e2n=np.empty((E, 2), np.int32),
                 is_pole=np.empty(E, np.uint8), n2e_ptr=np.empty(V + 1, np.int32),
                 n2e=np.empty(2 * E, np.int32), n2e_sign=np.empty(2 * E, np.int8))
        self._lib.orc_get_mesh(self._h, *(_ptr(d[k]) for k in
                                          ("tri", "tri_r", "tri_j", "e2n", "is_pole", "n2e_ptr", "n2e", "n2e_sign")))
        return d

    def dual(self):
        d = dict(S=np.empty((self.nedges, 2)), V=np.empty(self.nnodes), coslat=np.empty(self.nnodes),
                 pole_nphi=np.empty(self.nnodes))
        self._lib.orc_get_dual(self._h, _ptr(d["S"]), _ptr(d["V"]), _ptr(d["coslat"]), _ptr(d["pole_nphi"]))
        return d

    def closure(self):
        res = np.empty((self.nnodes, 2))
        ab = np.empty(self.nnodes)
        self._lib.orc_closure(self._h, _ptr(res), _ptr(ab))
        return res, ab

    # ----------------------------------------------------------- operators
    def _nodes(self, nodes):
        if nodes is None:
            return None, self.nnodes
        nodes = np.ascontiguousarray(nodes, dtype=np.int64)
        return nodes, int(nodes.shape[0])

    def gradient(self, f, nlev=None, nodes=None):
        f, f32, ld = _field(f)
        nlev = f.shape[1] if nlev is None else nlev
        nodes, n = self._nodes(nodes)
        gx = np.empty((n, nlev)); gy = np.empty((n, nlev))
        rc = self._lib.orc_gradient(self._h, _ptr(f), f32, ld, nlev, _ptr(nodes), n, _ptr(gx), _ptr(gy))
        if rc:
            raise ValueError("orc_gradient rc=%d" % rc)
        return gx, gy

    def divergence(self, u, v, nlev=None, nodes=None):
        u, f32, ld = _field(u)
        v, f32v, ldv = _field(v)
        if (f32, ld) != (f32v, ldv):
            raise ValueError("u and v need the same dtype and leading dimension")
        nlev = u.shape[1] if nlev is None else nlev
        nodes, n = self._nodes(nodes)
        out = np.empty((n, nlev))
        rc = self._lib.orc_divergence(self._h, _ptr(u), _ptr(v), f32, ld, nlev, _ptr(nodes), n, _ptr(out))
        if rc:
            raise ValueError("orc_divergence rc=%d" % rc)
        return out

    def curl(self, u, v, nlev=None, nodes=None):
        """Vertical vorticity of the tangent vector (u, v) (Stokes on the dual cell)."""
        u, f32, ld = _field(u)
        v, f32v, ldv = _field(v)
        if (f32, ld) != (f32v, ldv):
            raise ValueError("u and v need the same dtype and leading dimension")
        nlev = u.shape[1] if nlev is None else nlev
        nodes, n = self._nodes(nodes)
        out = np.empty((n, nlev))
        rc = self._lib.orc_curl(self._h, _ptr(u), _ptr(v), f32, ld, nlev, _ptr(nodes), n, _ptr(out))
        if rc:
            raise ValueError("orc_curl rc=%d" % rc)
        return out

    def vector_gradient(self, u, v, nlev=None, nodes=None):
        """Gradients of both components of a tangent vector field, with the
        antipode's component reversed on the pole faces: (ux, uy, vx, vy)."""
        u, f32, ld = _field(u)
        v, f32v, ldv = _field(v)
        if (f32, ld) != (f32v, ldv):
            raise ValueError("u and v need the same dtype and leading dimension")
        nlev = u.shape[1] if nlev is None else nlev
        nodes, n = self._nodes(nodes)
        o = [np.empty((n, nlev)) for _ in range(4)]
        rc = self._lib.orc_vector_gradient(self._h, _ptr(u), _ptr(v), f32, ld, nlev, _ptr(nodes), n,
                                           *(_ptr(x) for x in o))
        if rc:
            raise ValueError("orc_vector_gradient rc=%d" % rc)
        return tuple(o)

    def remap_weights(self, lonlat):
        """(nodes [T][3], weights [T][3]) locating each target (lon, lat) in
        radians in this mesh (linear interpolation in three-dimensional space
        over the sphere); raises if a target lies in no triangle."""
        lonlat = np.ascontiguousarray(lonlat, dtype=np.float64)
        T = lonlat.shape[0]
        nodes = np.empty((T, 3), np.int32)
        w = np.empty((T, 3))
        rc = self._lib.orc_remap(self._h, _ptr(lonlat), T, _ptr(nodes), _ptr(w))
        if rc:
            raise ValueError("orc_remap rc=%d" % rc)
        return nodes, w

    def remap(self, lonlat, f, nlev=None):
        """Field f on this mesh's nodes remapped to the target points."""
        nodes, w = self.remap_weights(lonlat)
        f, f32, ld = _field(f)
        nlev = f.shape[1] if nlev is None else nlev
        out = np.empty((nodes.shape[0], nlev))
        rc = self._lib.orc_remap_apply(_ptr(nodes), _ptr(w), nodes.shape[0], _ptr(f), f32, ld, nlev, _ptr(out))
        if rc:
            raise ValueError("orc_remap_apply rc=%d" % rc)
        return out

    def laplacian(self, f, nlev=None, nodes=None):
        f, f32, ld = _field(f)
        nlev = f.shape[1] if nlev is None else nlev
        nodes, n = self._nodes(nodes)
        out = np.empty((n, nlev))
        rc = self._lib.orc_laplacian(self._h, _ptr(f), f32, ld, nlev, _ptr(nodes), n, _ptr(out))
        if rc:
            raise ValueError("orc_laplacian rc=%d" % rc)
        return out

    def gradient_adjoint(self, y0, y1, nlev=None, nodes=None):
        y0, f32, ld = _field(y0)
        y1, f32b, ldb = _field(y1)
        if (f32, ld) != (f32b, ldb):
            raise ValueError("y0 and y1 need the same dtype and leading dimension")
        nlev = y0.shape[1] if nlev is None else nlev
        nodes, n = self._nodes(nodes)
        out = np.empty((n, nlev))
        rc = self._lib.orc_gradient_adjoint(self._h, _ptr(y0), _ptr(y1), f32, ld, nlev, _ptr(nodes), n, _ptr(out))
        if rc:
            raise ValueError("orc_gradient_adjoint rc=%d" % rc)
        return out

    def divergence_adjoint(self, d, nlev=None, nodes=None):
        d, f32, ld = _field(d)
        nlev = d.shape[1] if nlev is None else nlev
        nodes, n = self._nodes(nodes)
        xu = np.empty((n, nlev)); xv = np.empty((n, nlev))
        rc = self._lib.orc_divergence_adjoint(self._h, _ptr(d), f32, ld, nlev, _ptr(nodes), n, _ptr(xu), _ptr(xv))
        if rc:
            raise ValueError("orc_divergence_adjoint rc=%d" % rc)
        return xu, xv

    def curl_adjoint(self, z, nlev=None, nodes=None):
        """(u_bar, v_bar) = C^T z: the transpose of the curl's matrix rows."""
        z, f32, ld = _field(z)
        nlev = z.shape[1] if nlev is None else nlev
        nodes, n = self._nodes(nodes)
        xu = np.empty((n, nlev)); xv = np.empty((n, nlev))
        rc = self._lib.orc_curl_adjoint(self._h, _ptr(z), f32, ld, nlev, _ptr(nodes), n, _ptr(xu), _ptr(xv))
        if rc:
            raise ValueError("orc_curl_adjoint rc=%d" % rc)
        return xu, xv

    def gradient_averaged(self, f):
        f, f32, ld = _field(f)
        nlev = f.shape[1]
        gx = np.empty((self.nnodes, nlev)); gy = np.empty((self.nnodes, nlev))
        self._lib.orc_gradient_averaged(self._h, _ptr(f), f32, ld, nlev, _ptr(gx), _ptr(gy))
        return gx, gy

    def triplets(self, op: str):
        fn = {"gradient": self._lib.orc_gradient_triplets, "divergence": self._lib.orc_divergence_triplets}[op]
        n = int(fn(self._h, None, None, None))
        rows = np.empty(n, np.int64); cols = np.empty(n, np.int64); vals = np.empty(n)
        fn(self._h, _ptr(rows), _ptr(cols), _ptr(vals))
        return rows, cols, vals


PROJECTIONS = {"rotated_lonlat": 0, "mercator": 1, "lambert_conformal": 2, "polar_stereographic": 3}


class RegionalMesh:
    """Oracle regional grid (a rectangle of a projection's plane, two
    triangles per quad), its plane median dual and the operators with the
    projection's scale factors (``regional_oracle.c``)."""

    def __init__(self, projection: str, nx: int, ny: int, xmin: float, xmax: float, ymin: float, ymax: float, *,
                 radius: float = R_EARTH, lon0: float = 0.0, lat0: float = 45.0, south_pole=(0.0, -90.0)):
        lib = _load()
        code = PROJECTIONS[projection]
        if code == 0:
            tail = [float(south_pole[0]), float(south_pole[1]), 0.0, 0.0]
        else:
            tail = [float(radius), float(lon0), float(lat0), 0.0]
        prm = np.array([xmin, xmax, ymin, ymax, *tail], dtype=np.float64)
        h = lib.orc_reg_build(code, int(nx), int(ny), _ptr(prm), float(radius))
        if not h:
            raise ValueError("oracle regional grid build failed")
        self._h = ctypes.c_void_p(h)
        self._lib = lib
        self.R = float(radius)
        self.nx, self.ny = int(nx), int(ny)
        c = np.zeros(2, dtype=np.int64)
        lib.orc_reg_counts(self._h, _ptr(c))
        self.nnodes, self.ntri = int(c[0]), int(c[1])

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and h.value:
            self._lib.orc_reg_free(h)
            self._h = None

    def geometry(self):
        """lon, lat (radians), x, y (unit-sphere plane), hx, hy, area (R^2 x plane), tri [T][3]."""
        V, T = self.nnodes, self.ntri
        ll = np.empty((V, 2)); xy = np.empty((V, 2)); h = np.empty((V, 2)); A = np.empty(V)
        tri = np.empty((T, 3), np.int32)
        self._lib.orc_reg_get(self._h, _ptr(ll), _ptr(xy), _ptr(h), _ptr(A), _ptr(tri))
        return dict(lon=ll[:, 0].copy(), lat=ll[:, 1].copy(), x=xy[:, 0].copy(), y=xy[:, 1].copy(),
                    hx=h[:, 0].copy(), hy=h[:, 1].copy(), area=A, tri=tri)

    def closure(self):
        res = np.empty((self.nnodes, 2))
        ab = np.empty(self.nnodes)
        self._lib.orc_reg_closure(self._h, _ptr(res), _ptr(ab))
        return res, ab

    def _nodes(self, nodes):
        if nodes is None:
            return None, self.nnodes
        nodes = np.ascontiguousarray(nodes, dtype=np.int64)
        return nodes, int(nodes.shape[0])

    def _pair(self, a, b):
        a, f32, ld = _field(a)
        b, f32b, ldb = _field(b)
        if (f32, ld) != (f32b, ldb):
            raise ValueError("both inputs need the same dtype and leading dimension")
        return a, b, f32, ld

    def gradient(self, f, nlev=None, nodes=None):
        f, f32, ld = _field(f)
        nlev = f.shape[1] if nlev is None else nlev
        nodes, n = self._nodes(nodes)
        gx = np.empty((n, nlev)); gy = np.empty((n, nlev))
        if self._lib.orc_reg_gradient(self._h, _ptr(f), f32, ld, nlev, _ptr(nodes), n, _ptr(gx), _ptr(gy)):
            raise ValueError("orc_reg_gradient failed")
        return gx, gy

    def vector_gradient(self, u, v, nlev=None, nodes=None):
        ux, uy = self.gradient(u, nlev, nodes)
        vx, vy = self.gradient(v, nlev, nodes)
        return ux, uy, vx, vy

    def divergence(self, u, v, nlev=None, nodes=None):
        u, v, f32, ld = self._pair(u, v)
        nlev = u.shape[1] if nlev is None else nlev
        nodes, n = self._nodes(nodes)
        out = np.empty((n, nlev))
        if self._lib.orc_reg_divergence(self._h, _ptr(u), _ptr(v), f32, ld, nlev, _ptr(nodes), n, _ptr(out)):
            raise ValueError("orc_reg_divergence failed")
        return out

    def curl(self, u, v, nlev=None, nodes=None):
        u, v, f32, ld = self._pair(u, v)
        nlev = u.shape[1] if nlev is None else nlev
        nodes, n = self._nodes(nodes)
        out = np.empty((n, nlev))
        if self._lib.orc_reg_curl(self._h, _ptr(u), _ptr(v), f32, ld, nlev, _ptr(nodes), n, _ptr(out)):
            raise ValueError("orc_reg_curl failed")
        return out

    def laplacian(self, f, nlev=None, nodes=None):
        f, f32, ld = _field(f)
        nlev = f.shape[1] if nlev is None else nlev
        nodes, n = self._nodes(nodes)
        out = np.empty((n, nlev))
        if self._lib.orc_reg_laplacian(self._h, _ptr(f), f32, ld, nlev, _ptr(nodes), n, _ptr(out)):
            raise ValueError("orc_reg_laplacian failed")
        return out

    def gradient_adjoint(self, y0, y1, nlev=None, nodes=None):
        y0, y1, f32, ld = self._pair(y0, y1)
        nlev = y0.shape[1] if nlev is None else nlev
        nodes, n = self._nodes(nodes)
        out = np.empty((n, nlev))
        if self._lib.orc_reg_gradient_adjoint(self._h, _ptr(y0), _ptr(y1), f32, ld, nlev, _ptr(nodes), n, _ptr(out)):
            raise ValueError("orc_reg_gradient_adjoint failed")
        return out

    def gradient_averaged(self, f):
        """The averaged form sum n (wa f_i + wb f_j) / (A h), every node."""
        f, f32, ld = _field(f)
        nlev = f.shape[1]
        gx = np.empty((self.nnodes, nlev)); gy = np.empty((self.nnodes, nlev))
        if self._lib.orc_reg_gradient_averaged(self._h, _ptr(f), f32, ld, nlev, _ptr(gx), _ptr(gy)):
            raise ValueError("orc_reg_gradient_averaged failed")
        return gx, gy

    def divergence_adjoint(self, d, nlev=None, nodes=None):
        d, f32, ld = _field(d)
        nlev = d.shape[1] if nlev is None else nlev
        nodes, n = self._nodes(nodes)
        xu = np.empty((n, nlev)); xv = np.empty((n, nlev))
        if self._lib.orc_reg_divergence_adjoint(self._h, _ptr(d), f32, ld, nlev, _ptr(nodes), n, _ptr(xu), _ptr(xv)):
            raise ValueError("orc_reg_divergence_adjoint failed")
        return xu, xv


def _split(a):
    """Veltkamp splitting: a = hi + lo with hi, lo of at most 26 significant
    bits, so that every product of two halves is exact in FP64."""
    c = a * 134217729.0  # 2^27 + 1
    hi = c - (c - a)
    return hi, a - hi


def integral(V, x, nlev=None):
    """Volume-weighted sums I_k = sum_i V_i x[i, k], correctly rounded: every
    product V_i x_ik is taken exactly as the sum of the four products of the
    operands' 26-bit halves (Dekker 1971) and all of them are added by
    ``math.fsum`` (exact summation, one final rounding).  V: [n] FP64 dual
    volumes; x: [n, >= nlev] (float32 values are upcast exactly)."""
    import math
    V = np.asarray(V, dtype=np.float64)
    x = np.asarray(x)
    if x.ndim == 1:
        x = x[:, None]
    nlev = x.shape[1] if nlev is None else int(nlev)
    vh, vl = _split(V)
    out = np.empty(nlev)
    for k in range(nlev):
        xk = x[:, k].astype(np.float64)
        xh, xl = _split(xk)
        out[k] = math.fsum(np.concatenate([vh * xh, vh * xl, vl * xh, vl * xl]).tolist())
    return out
